// Reverse mode of the unrolled Sinkhorn loop (Algorithm 1) and of the barycenter iteration
// (Sec. 3.3), with checkpoints every `ck` iterations.
//
// The filter is its own adjoint: p_K(L, t) is a polynomial in the symmetric matrix L, so every
// transposed apply in the reverse sweep is the forward fused-order kernel again.  Forward state
// is kept only at checkpoints; each segment is swept backwards from a tape of its filter outputs,
// which the forward pass writes directly for the last segment and the reverse sweep recomputes
// from the checkpoint for the others.  Reductions over nodes (the distance, the
// barycenter weights' gradient) accumulate in FP64.
//
// Notation (the library's names; the paper's in brackets): a, b [mu, nu] marginals, u, v [v, w]
// scalings, vol [a] vertex weights.  Forward iteration j:
//     s_j = H(vol v_{j-1}),  u_j = a / s_j,  r_j = H(vol u_j),  v_j = b / r_j
// and W^2 = 4t sum vol (a ln u_T + b ln v_T).
#include <math.h>

#include <vector>

#include "gs_internal.cuh"

namespace {

inline unsigned nb(int64_t work, int per) { return (unsigned)((work + per - 1) / per); }
constexpr int kColBlocks = 1184;  // fixed grid of the barycenter reverse kernel (8 x 148)

__device__ __forceinline__ float div0(float num, float den) { return num == 0.f ? 0.f : num / den; }

__global__ void scale_fill(int64_t count, int B, const float* __restrict__ vol,
                           const float* __restrict__ src, float* __restrict__ dst)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float s = src ? src[i] : 1.f;
    dst[i] = vol ? vol[i / B] * s : s;
}

// Output adjoints of W^2 = 4t sum vol (a ln u + b ln v).
__global__ void sk_out_adj(int64_t n, double t4, const float* __restrict__ a, const float* __restrict__ b,
                           const float* __restrict__ vol, const float* __restrict__ u,
                           const float* __restrict__ v, float* __restrict__ ubar,
                           float* __restrict__ vbar, float* __restrict__ ga, float* __restrict__ gb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double w = t4 * (vol ? (double)vol[i] : 1.0);
    ubar[i] = a[i] != 0.f ? (float)(w * a[i] / u[i]) : 0.f;
    vbar[i] = b[i] != 0.f ? (float)(w * b[i] / v[i]) : 0.f;
    ga[i] = (a[i] != 0.f && u[i] > 0.f) ? (float)(w * log((double)u[i])) : 0.f;
    gb[i] = (b[i] != 0.f && v[i] > 0.f) ? (float)(w * log((double)v[i])) : 0.f;
}

// v_j = b / r_j:  gb += vbar / r_j ;  x = rbar = -vbar v_j / r_j
__global__ void sk_adj_v(int64_t n, const float* __restrict__ vbar, const float* __restrict__ r,
                         const float* __restrict__ v, float* __restrict__ gb, float* __restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    gb[i] += vbar[i] / r[i];
    x[i] = -vbar[i] * v[i] / r[i];
}

// r_j = H(vol u_j):  ubar = ubar_in + vol f ;  u_j = a / s_j:  ga += ubar / s_j ; x = -ubar u_j / s_j
__global__ void sk_adj_u(int64_t n, const float* __restrict__ f, const float* __restrict__ vol,
                         const float* __restrict__ ubar_in, const float* __restrict__ s,
                         const float* __restrict__ u, float* __restrict__ ga, float* __restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float ub = (ubar_in ? ubar_in[i] : 0.f) + (vol ? vol[i] : 1.f) * f[i];
    ga[i] += ub / s[i];
    x[i] = -ub * u[i] / s[i];
}

// s_j = H(vol v_{j-1}):  vbar_{j-1} = vol f
__global__ void sk_adj_s(int64_t n, const float* __restrict__ f, const float* __restrict__ vol,
                         float* __restrict__ vbar)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    vbar[i] = (vol ? vol[i] : 1.f) * f[i];
}

// ---------------------------------------------------------------- barycenter reverse kernels
// One warp per row (grid-stride over rows, fixed grid): undo v_i <- v_i mu / d_i and
// mu = exp(sum alpha_i ln d_i) and d_i = v_i r_i for iteration j.
//   in : Vbar (adjoint of V^j), Vp = V^{j-1}, R, mu^j, Mbar_in (adjoint of mu^j from the output)
//   out: Vbar <- vpbar (partial), X <- Rbar = Dbar Vp, partials[block][i] += sum_rows Lbar ln d_i
__global__ void __launch_bounds__(256) by_adj_pre(int64_t n, int m, float* __restrict__ Vbar,
                                                  const float* __restrict__ Vp,
                                                  const float* __restrict__ R,
                                                  const float* __restrict__ mu,
                                                  const float* __restrict__ Mbar_in,
                                                  const double* __restrict__ alpha,
                                                  float* __restrict__ X, double* __restrict__ partials)
{
    extern __shared__ double colacc[];  // [warps][m]: each warp sums its own rows, no atomics
    const int nw = (int)(blockDim.x >> 5);
    for (int c = threadIdx.x; c < nw * m; c += blockDim.x) colacc[c] = 0.0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    double* wacc = colacc + (threadIdx.x >> 5) * m;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < n;
         row += warps) {
        const float muj = mu[row];
        const float* vp = Vp + row * m;
        const float* rr = R + row * m;
        float* vb = Vbar + row * m;
        float msum = 0.f;
        for (int c = lane; c < m; c += 32) {
            const float d = vp[c] * rr[c];
            msum += vb[c] * vp[c] / d;
        }
        for (int off = 16; off > 0; off >>= 1) msum += __shfl_xor_sync(0xffffffffu, msum, off);
        const float Mb = (Mbar_in ? Mbar_in[row] : 0.f) + msum;
        const float Lb = Mb * muj;
        for (int c = lane; c < m; c += 32) {
            const float d = vp[c] * rr[c];
            const float vn = div0(vp[c] * muj, d);
            const float vbc = vb[c];
            float dbar = -vbc * vn / d + Lb * (float)alpha[c] / d;
            float vpb = vbc * muj / d + dbar * rr[c];
            wacc[c] += (double)Lb * (double)logf(d);  // lane c of this warp only
            vb[c] = vpb;
            X[row * m + c] = dbar * vp[c];
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += colacc[w * m + c];  // warps in order: repeatable sums
        partials[(int64_t)blockIdx.x * m + c] += t;
    }
}

// r_i = H(vol w_i) and w_i = mu_i / s_i:  Wbar = vol f ; X = Sbar = -Wbar w_i / s_i
__global__ void by_adj_mid(int64_t count, int m, const float* __restrict__ f,
                           const float* __restrict__ vol, const float* __restrict__ M,
                           const float* __restrict__ S, float* __restrict__ X)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float wb = (vol ? vol[i / m] : 1.f) * f[i];
    const float w = div0(M[i], S[i]);
    X[i] = -wb * w / S[i];
}

// s_i = H(vol v_i^{j-1}):  Vbar += vol f
__global__ void by_adj_post(int64_t count, int m, const float* __restrict__ f,
                            const float* __restrict__ vol, float* __restrict__ Vbar)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    Vbar[i] += (vol ? vol[i / m] : 1.f) * f[i];
}

__global__ void col_final(int nblocks, int m, const double* __restrict__ partials,
                          double* __restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[(int64_t)b * m + c];
    out[c] = s;
}

}  // namespace

// ------------------------------------------------------------------------------ Sinkhorn
gs_status gs_sinkhorn_grad_impl(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b,
                                const float* vol, double t, int K, int iters, int ck,
                                double* dist, float* grad_a_user, float* grad_b_user)
{
    const bool perm = g->perm != nullptr;  // work in the filter's node order
    std::vector<double> c((size_t)K + 1);
    gs_heat_coefficients(t, K, c.data());
    const int64_t n = g->n;
    const int nseg = (iters + ck - 1) / ck;
    const size_t vec = sizeof(float) * (size_t)n;
    WsPlan plan;
    const size_t ix = plan.add(vec), iA = plan.add(vec), iy = plan.add(vec), iu = plan.add(vec),
                 iv = plan.add(vec), iub = plan.add(vec), ivb = plan.add(vec), if_ = plan.add(vec),
                 ick = plan.add(vec * (size_t)nseg), itape = plan.add(vec * 4 * (size_t)ck),
                 ipart = plan.add(sizeof(double) * gs_reduce_blocks());
    const size_t iap = perm ? plan.add(vec) : 0, ibp = perm ? plan.add(vec) : 0,
                 ivp = (perm && vol) ? plan.add(vec) : 0, iga = perm ? plan.add(vec) : 0,
                 igb = perm ? plan.add(vec) : 0;
    gs_status st = gs_ws_ensure(ctx, plan.total);
    if (st != GS_OK) return st;
    float* grad_a = perm ? ws_at<float>(ctx, plan, iga) : grad_a_user;
    float* grad_b = perm ? ws_at<float>(ctx, plan, igb) : grad_b_user;
    if (perm) {
        float* ap = ws_at<float>(ctx, plan, iap);
        float* bp = ws_at<float>(ctx, plan, ibp);
        gs_permute_rows(ctx, n, 1, g->perm, a, ap, true);
        gs_permute_rows(ctx, n, 1, g->perm, b, bp, true);
        a = ap;
        b = bp;
        if (vol) {
            float* vp = ws_at<float>(ctx, plan, ivp);
            gs_permute_rows(ctx, n, 1, g->perm, vol, vp, true);
            vol = vp;
        }
    }
    float* x = ws_at<float>(ctx, plan, ix);
    float* A = ws_at<float>(ctx, plan, iA);
    float* y = ws_at<float>(ctx, plan, iy);
    float* u = ws_at<float>(ctx, plan, iu);
    float* v = ws_at<float>(ctx, plan, iv);
    float* ubar = ws_at<float>(ctx, plan, iub);
    float* vbar = ws_at<float>(ctx, plan, ivb);
    float* f = ws_at<float>(ctx, plan, if_);
    float* cks = ws_at<float>(ctx, plan, ick);
    float* tape = ws_at<float>(ctx, plan, itape);
    double* partials = ws_at<double>(ctx, plan, ipart);
    cudaStream_t s = ctx->stream;

    auto half = [&](const float* num, float* out, float* fsave) -> gs_status {
        Epilogue e;
        e.kind = EPI_DIVIDE;
        e.num = num;
        e.vol = vol;
        e.out = out;
        e.fsave = fsave;
        e.xnext_to_scratch = true;
        float* scratch = nullptr;
        gs_status r = gs_filter_enqueue(ctx, g, c.data(), K, 1, x, true, A, nullptr, y, e, nullptr, &scratch);
        if (scratch != x) std::swap(x, A);
        return r;
    };
    auto apply = [&](float* in, float* out) -> gs_status {  // out = H(in); in is clobbered
        Epilogue e;
        e.kind = EPI_STORE;
        e.out = out;
        return gs_filter_enqueue(ctx, g, c.data(), K, 1, in, true, A, nullptr, y, e, nullptr, nullptr);
    };

    // forward with checkpoints of v_{j0}, j0 = 0, ck, 2ck, ...; the last segment's states go
    // straight to the tape, so the reverse sweep does not recompute that segment
    float* ts = tape;                       // s_j
    float* tu = tape + (size_t)ck * n;      // u_j
    float* tr = tape + (size_t)2 * ck * n;  // r_j
    float* tv = tape + (size_t)3 * ck * n;  // v_j
    const int j0_last = (nseg - 1) * ck;
    scale_fill<<<nb(n, 256), 256, 0, s>>>(n, 1, nullptr, nullptr, cks);  // v_0 = 1
    scale_fill<<<nb(n, 256), 256, 0, s>>>(n, 1, vol, nullptr, x);
    gs_count(ctx, 2);
    for (int j = 1; j <= iters && st == GS_OK; ++j) {
        if (j > j0_last) {
            const size_t l = (size_t)(j - 1 - j0_last);
            st = half(a, tu + l * n, ts + l * n);
            if (st == GS_OK) st = half(b, tv + l * n, tr + l * n);
        } else {
            st = half(a, u, nullptr);
            if (st == GS_OK) st = half(b, v, nullptr);
        }
        if (st == GS_OK && j % ck == 0 && j < iters)
            cudaMemcpyAsync(cks + (size_t)(j / ck) * n, v, vec, cudaMemcpyDeviceToDevice, s);
    }
    if (st != GS_OK) return st;
    u = tu + (size_t)(iters - 1 - j0_last) * n;  // the last iteration's scalings
    v = tv + (size_t)(iters - 1 - j0_last) * n;
    if ((st = gs_distance_enqueue(ctx, n, a, b, vol, u, v, t, partials, dist)) != GS_OK) return st;
    sk_out_adj<<<nb(n, 256), 256, 0, s>>>(n, 4.0 * t, a, b, vol, u, v, ubar, vbar, grad_a, grad_b);
    gs_count(ctx, 1);

    // reverse sweep, one segment at a time
    for (int seg = nseg - 1; seg >= 0 && st == GS_OK; --seg) {
        const int j0 = seg * ck;
        const int len = (iters - j0) < ck ? (iters - j0) : ck;
        if (seg < nseg - 1) {  // recompute the segment from its checkpoint (the last one is on tape)
            scale_fill<<<nb(n, 256), 256, 0, s>>>(n, 1, vol, cks + (size_t)seg * n, x);
            gs_count(ctx, 1);
            for (int l = 0; l < len && st == GS_OK; ++l) {
                st = half(a, tu + (size_t)l * n, ts + (size_t)l * n);
                if (st == GS_OK) st = half(b, tv + (size_t)l * n, tr + (size_t)l * n);
            }
        }
        for (int l = len - 1; l >= 0 && st == GS_OK; --l) {
            const bool last = (seg == nseg - 1) && (l == len - 1);
            sk_adj_v<<<nb(n, 256), 256, 0, s>>>(n, vbar, tr + (size_t)l * n, tv + (size_t)l * n, grad_b, x);
            gs_count(ctx, 1);
            if ((st = apply(x, f)) != GS_OK) break;
            sk_adj_u<<<nb(n, 256), 256, 0, s>>>(n, f, vol, last ? ubar : nullptr, ts + (size_t)l * n,
                                                 tu + (size_t)l * n, grad_a, x);
            gs_count(ctx, 1);
            if ((st = apply(x, f)) != GS_OK) break;
            sk_adj_s<<<nb(n, 256), 256, 0, s>>>(n, f, vol, vbar);
            gs_count(ctx, 1);
        }
    }
    if (st != GS_OK) return st;
    if (perm) {
        gs_permute_rows(ctx, n, 1, g->perm, grad_a, grad_a_user, false);
        gs_permute_rows(ctx, n, 1, g->perm, grad_b, grad_b_user, false);
    }
    return gs_cuda_check(ctx, cudaGetLastError(), "Sinkhorn reverse sweep");
}

// ---------------------------------------------------------------------------- barycenter
gs_status gs_barycenter_grad_impl(gs_ctx* ctx, const gs_graph* g, const float* M, int m,
                                  const double* alpha, const float* vol, double t, int K, int iters,
                                  int ck, const float* mubar, float* mu_user, double* grad_alpha)
{
    const bool perm = g->perm != nullptr;  // work in the filter's node order
    std::vector<double> c((size_t)K + 1);
    gs_heat_coefficients(t, K, c.data());
    const int64_t n = g->n;
    const int64_t nm = n * (int64_t)m;
    const int nseg = (iters + ck - 1) / ck;
    const size_t blk = sizeof(float) * (size_t)nm;
    WsPlan plan;
    const size_t ix = plan.add(blk), iA = plan.add(blk), iy = plan.add(blk), iV = plan.add(blk),
                 iVb = plan.add(blk), iF = plan.add(blk), ick = plan.add(blk * (size_t)nseg),
                 itp = plan.add(blk * (size_t)ck), its = plan.add(blk * (size_t)ck),
                 itr = plan.add(blk * (size_t)ck), imu = plan.add(sizeof(float) * (size_t)n * ck),
                 ipart = plan.add(sizeof(double) * (size_t)kColBlocks * m);
    const size_t vecb = sizeof(float) * (size_t)n;
    const size_t iMp = perm ? plan.add(blk) : 0, imb = perm ? plan.add(vecb) : 0,
                 imo = plan.add(vecb), ivp = (perm && vol) ? plan.add(vecb) : 0;
    gs_status st = gs_ws_ensure(ctx, plan.total);
    if (st != GS_OK) return st;
    float* mu_out = ws_at<float>(ctx, plan, imo);
    if (perm) {
        float* Mp = ws_at<float>(ctx, plan, iMp);
        float* mbp = ws_at<float>(ctx, plan, imb);
        gs_permute_rows(ctx, n, m, g->perm, M, Mp, true);
        gs_permute_rows(ctx, n, 1, g->perm, mubar, mbp, true);
        M = Mp;
        mubar = mbp;
        if (vol) {
            float* vp = ws_at<float>(ctx, plan, ivp);
            gs_permute_rows(ctx, n, 1, g->perm, vol, vp, true);
            vol = vp;
        }
    }
    float* x = ws_at<float>(ctx, plan, ix);
    float* A = ws_at<float>(ctx, plan, iA);
    float* y = ws_at<float>(ctx, plan, iy);
    float* V = ws_at<float>(ctx, plan, iV);
    float* Vbar = ws_at<float>(ctx, plan, iVb);
    float* F = ws_at<float>(ctx, plan, iF);
    float* cks = ws_at<float>(ctx, plan, ick);
    float* tVp = ws_at<float>(ctx, plan, itp);
    float* tS = ws_at<float>(ctx, plan, its);
    float* tR = ws_at<float>(ctx, plan, itr);
    float* tmu = ws_at<float>(ctx, plan, imu);
    double* partials = ws_at<double>(ctx, plan, ipart);
    cudaStream_t s = ctx->stream;

    auto iterate = [&](float* Vp_save, float* S_save, float* R_save, float* mu_dst) -> gs_status {
        if (Vp_save) cudaMemcpyAsync(Vp_save, V, blk, cudaMemcpyDeviceToDevice, s);
        Epilogue e1;
        e1.kind = EPI_DIVIDE;
        e1.num = M;
        e1.vol = vol;
        e1.fsave = S_save;
        e1.xnext_to_scratch = true;
        float* scratch = nullptr;
        gs_status r = gs_filter_enqueue(ctx, g, c.data(), K, m, x, true, A, nullptr, y, e1, nullptr, &scratch);
        if (scratch != x) std::swap(x, A);
        if (r != GS_OK) return r;
        Epilogue e2;
        e2.kind = EPI_BARY_V;
        e2.vol = vol;
        e2.V = V;
        e2.alpha = alpha;
        e2.mu = mu_dst;
        e2.fsave = R_save;
        e2.xnext_to_scratch = true;
        r = gs_filter_enqueue(ctx, g, c.data(), K, m, x, true, A, nullptr, y, e2, nullptr, &scratch);
        if (scratch != x) std::swap(x, A);
        return r;
    };

    // forward with checkpoints of V; the last segment's states go straight to the tape, so the
    // reverse sweep does not recompute that segment
    const int j0_last = (nseg - 1) * ck;
    scale_fill<<<nb(nm, 256), 256, 0, s>>>(nm, m, nullptr, nullptr, V);
    scale_fill<<<nb(nm, 256), 256, 0, s>>>(nm, m, vol, nullptr, x);
    gs_count(ctx, 2);
    for (int j = 0; j < iters && st == GS_OK; ++j) {
        if (j % ck == 0) cudaMemcpyAsync(cks + (size_t)(j / ck) * nm, V, blk, cudaMemcpyDeviceToDevice, s);
        if (j >= j0_last) {
            const size_t l = (size_t)(j - j0_last);
            st = iterate(tVp + l * nm, tS + l * nm, tR + l * nm, tmu + l * n);
        } else {
            st = iterate(nullptr, nullptr, nullptr, mu_out);
        }
    }
    if (st != GS_OK) return st;
    cudaMemcpyAsync(mu_out, tmu + (size_t)(iters - 1 - j0_last) * n, vecb, cudaMemcpyDeviceToDevice, s);

    cudaFuncSetAttribute(by_adj_pre, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double) * 8 * m));
    cudaMemsetAsync(partials, 0, sizeof(double) * (size_t)kColBlocks * m, s);
    cudaMemsetAsync(Vbar, 0, blk, s);
    const unsigned rgrid = (unsigned)std::min<int64_t>(kColBlocks, (n + 7) / 8);
    for (int seg = nseg - 1; seg >= 0 && st == GS_OK; --seg) {
        const int j0 = seg * ck;
        const int len = (iters - j0) < ck ? (iters - j0) : ck;
        if (seg < nseg - 1) {  // recompute the segment from its checkpoint (the last one is on tape)
            cudaMemcpyAsync(V, cks + (size_t)seg * nm, blk, cudaMemcpyDeviceToDevice, s);
            scale_fill<<<nb(nm, 256), 256, 0, s>>>(nm, m, vol, V, x);
            gs_count(ctx, 1);
            for (int l = 0; l < len && st == GS_OK; ++l)
                st = iterate(tVp + (size_t)l * nm, tS + (size_t)l * nm, tR + (size_t)l * nm, tmu + (size_t)l * n);
        }
        for (int l = len - 1; l >= 0 && st == GS_OK; --l) {
            const bool last = (seg == nseg - 1) && (l == len - 1);
            by_adj_pre<<<rgrid, 256, sizeof(double) * 8 * m, s>>>(n, m, Vbar, tVp + (size_t)l * nm,
                                                               tR + (size_t)l * nm, tmu + (size_t)l * n,
                                                               last ? mubar : nullptr, alpha, x, partials);
            gs_count(ctx, 1);
            Epilogue e;
            e.kind = EPI_STORE;
            e.out = F;
            if ((st = gs_filter_enqueue(ctx, g, c.data(), K, m, x, true, A, nullptr, y, e, nullptr, nullptr)) != GS_OK)
                break;
            by_adj_mid<<<nb(nm, 256), 256, 0, s>>>(nm, m, F, vol, M, tS + (size_t)l * nm, x);
            gs_count(ctx, 1);
            if ((st = gs_filter_enqueue(ctx, g, c.data(), K, m, x, true, A, nullptr, y, e, nullptr, nullptr)) != GS_OK)
                break;
            by_adj_post<<<nb(nm, 256), 256, 0, s>>>(nm, m, F, vol, Vbar);
            gs_count(ctx, 1);
        }
    }
    if (st != GS_OK) return st;
    col_final<<<nb(m, 128), 128, 0, s>>>((int)rgrid, m, partials, grad_alpha);
    gs_count(ctx, 1);
    if (mu_user) {
        if (perm) gs_permute_rows(ctx, n, 1, g->perm, mu_out, mu_user, false);
        else cudaMemcpyAsync(mu_user, mu_out, vecb, cudaMemcpyDeviceToDevice, s);
    }
    return gs_cuda_check(ctx, cudaGetLastError(), "barycenter reverse sweep");
}
