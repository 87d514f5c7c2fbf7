// Euler implicit heat kernel (the alternative approximation of H_t that Sec. 4 cites): K backward
// Euler steps of the heat equation, Y = (I + (t/K) L)^{-K} V, each step one solve of the symmetric
// positive definite system (I + h L) x = b, h = t/K, by conjugate gradients on all B columns at
// once.  With L = I - P the matrix is (1 + h) I - h P; P's spectrum lies in [-1, 1], so the
// condition number is at most 1 + 2h and a handful of iterations reach FP32 accuracy.
//
// Every CG iteration is five stream-ordered launches with the scalars on the device (no host
// synchronisation): q = A p with a per-block partial of p.q; alpha = rr / pq per column; x += alpha
// p, r -= alpha q with a partial of r.r; beta (and the column's convergence) per column; p = r +
// beta p.  Partial sums are taken in a fixed order, so results repeat bit for bit.  A column whose
// residual has dropped below tol |b| keeps alpha = 0 from then on.  The graph is used in the
// caller's node order (rowptr / col / pval of the CSR).
#include "gs_internal.cuh"

namespace {

constexpr int kCgThreads = 256;

// per-column state: [0] rr, [1] pq, [2] alpha, [3] beta, [4] bb (|b|^2), [5] done
constexpr int kColState = 6;

// q = (1 + h) p - h P p for the [n, B] block p; partial[blk][c] = sum over the block's elements of
// column c of p * q (elements e = row * B + c, 256 consecutive elements per block)
__global__ void __launch_bounds__(kCgThreads) cg_matvec(int64_t n, int B, const int* __restrict__ rowptr,
                                                        const int* __restrict__ col, const float* __restrict__ pval,
                                                        float h, const float* __restrict__ p, float* __restrict__ q,
                                                        double* __restrict__ partial)
{
    __shared__ double vals[kCgThreads];
    const int64_t e = (int64_t)blockIdx.x * kCgThreads + threadIdx.x;
    double pq = 0.0;
    if (e < n * B) {
        const int64_t row = e / B;
        const int c = (int)(e - row * B);
        float s = 0.f;
        for (int k = rowptr[row]; k < rowptr[row + 1]; ++k) s = fmaf(pval[k], p[(int64_t)col[k] * B + c], s);
        const float pe = p[e];
        const float qe = fmaf(1.f + h, pe, -h * s);
        q[e] = qe;
        pq = (double)pe * (double)qe;
    }
    vals[threadIdx.x] = pq;
    __syncthreads();
    // column c collects the block's elements with (e0 + j) % B == c, in increasing j
    if ((int)threadIdx.x < B) {
        const int64_t e0 = (int64_t)blockIdx.x * kCgThreads;
        const int c = threadIdx.x;
        const int j0 = (int)((c - e0 % B + B) % B);
        double acc = 0.0;
        for (int j = j0; j < kCgThreads; j += B) acc += vals[j];
        partial[(int64_t)blockIdx.x * B + c] = acc;
    }
}

// x += alpha p, r -= alpha q per column; partial of r.r
__global__ void __launch_bounds__(kCgThreads) cg_update(int64_t n, int B, const double* __restrict__ st,
                                                        const float* __restrict__ p, const float* __restrict__ q,
                                                        float* __restrict__ x, float* __restrict__ r,
                                                        double* __restrict__ partial)
{
    __shared__ double vals[kCgThreads];
    const int64_t e = (int64_t)blockIdx.x * kCgThreads + threadIdx.x;
    double rr = 0.0;
    if (e < n * B) {
        const int c = (int)(e % B);
        const float a = (float)st[c * kColState + 2];
        x[e] = fmaf(a, p[e], x[e]);
        const float re = fmaf(-a, q[e], r[e]);
        r[e] = re;
        rr = (double)re * (double)re;
    }
    vals[threadIdx.x] = rr;
    __syncthreads();
    if ((int)threadIdx.x < B) {
        const int64_t e0 = (int64_t)blockIdx.x * kCgThreads;
        const int c = threadIdx.x;
        const int j0 = (int)((c - e0 % B + B) % B);
        double acc = 0.0;
        for (int j = j0; j < kCgThreads; j += B) acc += vals[j];
        partial[(int64_t)blockIdx.x * B + c] = acc;
    }
}

// p = r + beta p
__global__ void __launch_bounds__(kCgThreads) cg_direction(int64_t n, int B, const double* __restrict__ st,
                                                           const float* __restrict__ r, float* __restrict__ p)
{
    const int64_t e = (int64_t)blockIdx.x * kCgThreads + threadIdx.x;
    if (e >= n * B) return;
    const int c = (int)(e % B);
    p[e] = fmaf((float)st[c * kColState + 3], p[e], r[e]);
}

// Column scalars from the block partials (summed over blocks in order), one thread per column.
//   which 0: start of a solve: rr = bb = sum partial (r = p = b), done = 0
//   which 1: alpha = rr / pq (0 once done)
//   which 2: rr_new; done when rr_new <= tol^2 bb; beta = rr_new / rr (0 once done)
__global__ void cg_scalars(int B, int nblk, const double* __restrict__ partial, double* __restrict__ st, int which,
                           double tol2)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= B) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * B + c];
    double* o = st + c * kColState;
    if (which == 0) {
        o[0] = s;
        o[4] = s;
        o[5] = s == 0.0 ? 1.0 : 0.0;
        o[2] = o[3] = 0.0;
    } else if (which == 1) {
        o[1] = s;
        o[2] = (o[5] != 0.0 || !(s > 0.0)) ? 0.0 : o[0] / s;
    } else {
        const double rr = o[0];
        if (o[5] == 0.0 && s <= tol2 * o[4]) o[5] = 1.0;
        o[3] = (o[5] != 0.0 || !(rr > 0.0)) ? 0.0 : s / rr;
        o[0] = s;
    }
}

// partial of b.b for the start of a solve (b already copied into r and p)
__global__ void __launch_bounds__(kCgThreads) cg_norm(int64_t n, int B, const float* __restrict__ b,
                                                      double* __restrict__ partial)
{
    __shared__ double vals[kCgThreads];
    const int64_t e = (int64_t)blockIdx.x * kCgThreads + threadIdx.x;
    vals[threadIdx.x] = e < n * B ? (double)b[e] * (double)b[e] : 0.0;
    __syncthreads();
    if ((int)threadIdx.x < B) {
        const int64_t e0 = (int64_t)blockIdx.x * kCgThreads;
        const int c = threadIdx.x;
        const int j0 = (int)((c - e0 % B + B) % B);
        double acc = 0.0;
        for (int j = j0; j < kCgThreads; j += B) acc += vals[j];
        partial[(int64_t)blockIdx.x * B + c] = acc;
    }
}

}  // namespace

gs_status gs_heat_apply_implicit_impl(gs_ctx* ctx, const gs_graph* g, double t, int K, const float* V, int B,
                                      float* Y, double tol, int iters)
{
    const int64_t n = g->n, count = n * (int64_t)B;
    const int nblk = (int)((count + kCgThreads - 1) / kCgThreads);
    WsPlan plan;
    const size_t blk = sizeof(float) * (size_t)count;
    const size_t ix = plan.add(blk), ib = plan.add(blk), ir = plan.add(blk), ip = plan.add(blk), iq = plan.add(blk),
                 ipart = plan.add(sizeof(double) * (size_t)nblk * B), ist = plan.add(sizeof(double) * kColState * B);
    gs_status st = gs_ws_ensure(ctx, plan.total);
    if (st != GS_OK) return st;
    float* x = ws_at<float>(ctx, plan, ix);
    float* b = ws_at<float>(ctx, plan, ib);
    float* r = ws_at<float>(ctx, plan, ir);
    float* p = ws_at<float>(ctx, plan, ip);
    float* q = ws_at<float>(ctx, plan, iq);
    double* part = ws_at<double>(ctx, plan, ipart);
    double* cs = ws_at<double>(ctx, plan, ist);
    cudaStream_t s = ctx->stream;
    const float h = (float)(t / K);
    const double tol2 = tol * tol;
    const unsigned cb = (unsigned)((B + 127) / 128);
    cudaMemcpyAsync(b, V, blk, cudaMemcpyDeviceToDevice, s);
    for (int step = 0; step < K; ++step) {
        // solve (I + h L) x = b from x = 0: r = p = b
        cudaMemsetAsync(x, 0, blk, s);
        cudaMemcpyAsync(r, b, blk, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(p, b, blk, cudaMemcpyDeviceToDevice, s);
        cg_norm<<<nblk, kCgThreads, 0, s>>>(n, B, b, part);
        cg_scalars<<<cb, 128, 0, s>>>(B, nblk, part, cs, 0, tol2);
        for (int it = 0; it < iters; ++it) {
            cg_matvec<<<nblk, kCgThreads, 0, s>>>(n, B, g->rowptr, g->col, g->pval, h, p, q, part);
            cg_scalars<<<cb, 128, 0, s>>>(B, nblk, part, cs, 1, tol2);
            cg_update<<<nblk, kCgThreads, 0, s>>>(n, B, cs, p, q, x, r, part);
            cg_scalars<<<cb, 128, 0, s>>>(B, nblk, part, cs, 2, tol2);
            cg_direction<<<nblk, kCgThreads, 0, s>>>(n, B, cs, r, p);
        }
        gs_count(ctx, 2 + 5 * iters);
        std::swap(x, b);  // this step's solution is the next step's right-hand side
    }
    cudaMemcpyAsync(Y, b, blk, cudaMemcpyDeviceToDevice, s);
    return gs_cuda_check(ctx, cudaGetLastError(), "implicit heat kernel");
}
