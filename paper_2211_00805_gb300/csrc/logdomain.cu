// Log-domain Geodesic Sinkhorn: Algorithm 1 with the scalings held as FP64 potentials ln u, ln v
// instead of FP32 values, for the small diffusion times where u and v leave the FP32 range (on a
// sphere graph at t = 1 they span e^{-170} .. e^{130}).
//
// With the potentials absorbed into the kernel, H (vol * v) becomes a sum whose terms span the same
// range, and the Chebyshev recurrence of Sec. 3.5 carries them through K orders of signed sums.
// Every vector of the recurrence is therefore held in an extended-range form: an FP32 mantissa m
// and an int32 binary exponent e, value m 2^e (m = 0 for zero).  One order over a row takes the
// largest exponent E of the terms it adds, scales every term by the exact power of two 2^{e - E},
// adds the mantissas in FP32 and renormalises the sum (frexpf).  The sums carry FP32 rounding only
// (no exponentials per nonzero); a term more than 2^126 below the row's largest one is dropped.
// Coefficients c_k are split the same way on the host, so c_K below the FP32 range is no problem.
//
// Per Sinkhorn half-step (one application of p_K), K launches over the caller-order CSR of P:
//   order 0     : x1 = P x0;                y = c0 x0 + c1 x1
//   order k >= 1: x_{k+1} = 2 P x_k - x_{k-1};  y += c_{k+1} x_{k+1}
// and the last order ends with the division of Algorithm 1 in the log domain,
//   ln u_i = ln a_i - ln y_i  (-inf where a_i = 0; NaN and GS_FLAG_NONFINITE where a_i > 0 and
//   y_i <= 0), and writes the next half-step's input vol_i u_i in the extended form.
// Then W^2 = 4t sum_i vol_i (a_i ln u_i + b_i ln v_i) from the potentials, in FP64.
#include <math.h>

#include <vector>

#include "gs_internal.cuh"

namespace {

constexpr int kZeroExp = -(1 << 30);  // exponent stored with a zero mantissa
constexpr int kLanes = 8;             // lanes summing one row
constexpr int kXrThreads = 256;
constexpr int kRowsPerBlock = kXrThreads / kLanes;
constexpr int kRedThreads = 1024;
constexpr double kLn2 = 0.69314718055994530942;

// m 2^d for d <= 1: an exact power of two for d >= -126; the term is dropped below that
__device__ __forceinline__ float scale_pow2(float m, int d)
{
    return d < -126 ? 0.f : m * __int_as_float((d + 127) << 23);
}

// s 2^E as a normalised (m, e): m in [0.5, 1) in magnitude, or m = 0
__device__ __forceinline__ void xr_normalise(float s, int E, float& m, int& e)
{
    if (s == 0.f || E == kZeroExp) {
        m = 0.f;
        e = kZeroExp;
        return;
    }
    int ee;
    m = frexpf(s, &ee);
    e = E + ee;
}

// (m1, e1) += (m2, e2)
__device__ __forceinline__ void xr_add(float& m1, int& e1, float m2, int e2)
{
    if (m2 == 0.f) return;
    if (m1 == 0.f) {
        m1 = m2;
        e1 = e2;
        return;
    }
    const int E = max(e1, e2);
    xr_normalise(scale_pow2(m1, e1 - E) + scale_pow2(m2, e2 - E), E, m1, e1);
}

// ln|value| parts -> extended form of exp(z) (z = -inf gives zero)
__device__ __forceinline__ void xr_from_log(double z, float& m, int& e)
{
    if (z == -INFINITY) {
        m = 0.f;
        e = kZeroExp;
        return;
    }
    const double f = floor(z / kLn2);
    m = (float)(0.5 * exp(z - f * kLn2));  // in [0.5, 1)
    e = (int)f + 1;
}

struct XrOrder {
    int64_t n;
    const int* rowptr;
    const int* col;
    const float* pval;
    const float* xm;  // T_k x, gathered
    const int* xe;
    const float* zm;  // T_{k-1} x, own row only; null in order 0
    const int* ze;
    float* om;  // T_{k+1} x (not written by the last order)
    int* oe;
    float* ym;  // accumulator y, own row only
    int* ye;
    float c0m;  // order 0: coefficient of T_0 (mantissa, exponent)
    int c0e;
    float cm;  // coefficient of T_{k+1}
    int ce;
    int twice;  // 0: P x (order 0), 1: 2 P x
    int last;   // last order: division epilogue instead of storing y and T_{k+1} x
    const float* marg;  // a (or b) of the division
    const float* vol;   // vertex weights or null
    double* logout;     // ln u (or ln v)
    float* nm;          // next half-step's input vol * u
    int* ne;
    int* flags;
};

__global__ void __launch_bounds__(kXrThreads) xr_order(XrOrder p)
{
    const int64_t row = (int64_t)blockIdx.x * kRowsPerBlock + (threadIdx.x / kLanes);
    const int lane = threadIdx.x & (kLanes - 1);
    if (row >= p.n) return;  // whole lane groups leave together
    const unsigned gmask = 0xffu << (threadIdx.x & 24);
    const int beg = p.rowptr[row], end = p.rowptr[row + 1];
    // pass 1: largest exponent of the row's terms
    int E = kZeroExp;
    for (int k = beg + lane; k < end; k += kLanes) {
        const int j = p.col[k];
        if (p.xm[j] != 0.f) E = max(E, p.xe[j]);
    }
    for (int off = kLanes / 2; off > 0; off >>= 1) E = max(E, __shfl_xor_sync(gmask, E, off));
    float zm = 0.f;
    int ze = kZeroExp;
    if (p.zm) {
        zm = p.zm[row];
        ze = p.ze[row];
        if (zm != 0.f) E = max(E, ze);
    }
    // pass 2: mantissas aligned to 2^E, summed in FP32 (lane partials, then a fixed butterfly)
    float s = 0.f;
    if (E != kZeroExp) {
        for (int k = beg + lane; k < end; k += kLanes) {
            const int j = p.col[k];
            const float m = p.xm[j];
            if (m != 0.f) s = fmaf(p.pval[k], scale_pow2(m, p.xe[j] - E + p.twice), s);
        }
    }
    for (int off = kLanes / 2; off > 0; off >>= 1) s += __shfl_xor_sync(gmask, s, off);
    if (zm != 0.f) s -= scale_pow2(zm, ze - E);
    float xm1;
    int xe1;
    xr_normalise(s, E, xm1, xe1);
    if (lane != 0) return;
    // accumulator
    float ym;
    int ye;
    if (p.zm) {
        ym = p.ym[row];
        ye = p.ye[row];
    } else {  // order 0: y = c0 x0
        const float x0 = p.xm[row];
        ym = 0.f;
        ye = kZeroExp;
        if (x0 != 0.f && p.c0m != 0.f) {
            int ee;
            ym = frexpf(p.c0m * x0, &ee);
            ye = p.c0e + p.xe[row] + ee;
        }
    }
    if (xm1 != 0.f) {
        int ee;
        const float pm = frexpf(p.cm * xm1, &ee);
        xr_add(ym, ye, pm, p.ce + xe1 + ee);
    }
    if (!p.last) {
        p.om[row] = xm1;
        p.oe[row] = xe1;
        p.ym[row] = ym;
        p.ye[row] = ye;
        return;
    }
    // division epilogue (Algorithm 1) in the log domain
    const float a = p.marg[row];
    double lu;
    if (a == 0.f) {
        lu = -INFINITY;
    } else if (ym > 0.f) {
        lu = log((double)a) - (log((double)ym) + (double)ye * kLn2);
    } else {
        lu = NAN;
        atomicOr(p.flags, GS_FLAG_NONFINITE);
    }
    p.logout[row] = lu;
    const double z = lu + (p.vol ? log((double)p.vol[row]) : 0.0);
    float m;
    int e;
    xr_from_log(z == z ? z : -INFINITY, m, e);
    p.nm[row] = m;
    p.ne[row] = e;
}

// x0 = vol * 1 (the first half-step's input, v = 1)
__global__ void xr_init(int64_t n, const float* __restrict__ vol, float* __restrict__ m, int* __restrict__ e)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float mm;
    int ee;
    xr_from_log(vol ? log((double)vol[i]) : 0.0, mm, ee);
    m[i] = mm;
    e[i] = ee;
}

// W^2 = 4t sum_i vol_i (a_i ln u_i + b_i ln v_i) (0 ln 0 := 0), one block, fixed summation order
__global__ void __launch_bounds__(kRedThreads) xr_distance(int64_t n, const float* __restrict__ a,
                                                           const float* __restrict__ b, const float* __restrict__ vol,
                                                           const double* __restrict__ lu, const double* __restrict__ lv,
                                                           double t, double* __restrict__ dist, int* __restrict__ flags)
{
    __shared__ double red[kRedThreads / 32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kRedThreads) {
        double term = 0.0;
        if (a[i] != 0.f) term += (double)a[i] * lu[i];
        if (b[i] != 0.f) term += (double)b[i] * lv[i];
        s += (vol ? (double)vol[i] : 1.0) * term;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double tot = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) tot += red[w];
    const double W2 = 4.0 * t * tot;
    if (!isfinite(W2)) atomicOr(flags, GS_FLAG_NONFINITE);
    dist[0] = W2;
    dist[1] = W2 >= 0.0 ? sqrt(W2) : NAN;
}

}  // namespace

gs_status gs_sinkhorn_log_impl(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b, const float* vol,
                               double t, int K, int iters, double* log_u, double* log_v, double* dist)
{
    const int64_t n = g->n;
    WsPlan plan;
    const size_t fb = sizeof(float) * (size_t)n, ib = sizeof(int) * (size_t)n;
    size_t im[6], ie[6];
    for (int i = 0; i < 6; ++i) {  // two inputs (ping-pong), three recurrence vectors, accumulator
        im[i] = plan.add(fb);
        ie[i] = plan.add(ib);
    }
    gs_status st = gs_ws_ensure(ctx, plan.total);
    if (st != GS_OK) return st;
    float* M[6];
    int* E[6];
    for (int i = 0; i < 6; ++i) {
        M[i] = ws_at<float>(ctx, plan, im[i]);
        E[i] = ws_at<int>(ctx, plan, ie[i]);
    }
    std::vector<double> c((size_t)K + 1);
    gs_heat_coefficients(t, K, c.data());
    std::vector<float> cm((size_t)K + 1);
    std::vector<int> ce((size_t)K + 1);
    for (int k = 0; k <= K; ++k) {
        int ee;
        cm[k] = (float)frexp(c[k], &ee);
        ce[k] = ee;
    }
    cudaStream_t s = ctx->stream;
    const unsigned grid = (unsigned)((n + kRowsPerBlock - 1) / kRowsPerBlock);
    xr_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, vol, M[0], E[0]);
    int in = 0;  // the current input is buffer `in`, the next one 1 - in; 2..4 recurrence, 5 y
    for (int it = 0; it < 2 * iters; ++it) {
        const bool half_u = (it & 1) == 0;
        XrOrder p{};
        p.n = n;
        p.rowptr = g->rowptr;
        p.col = g->col;
        p.pval = g->pval;
        p.ym = M[5];
        p.ye = E[5];
        p.c0m = cm[0];
        p.c0e = ce[0];
        p.marg = half_u ? a : b;
        p.vol = vol;
        p.logout = half_u ? log_u : log_v;
        p.nm = M[1 - in];
        p.ne = E[1 - in];
        p.flags = ctx->flags;
        for (int k = 0; k < K; ++k) {
            // gathers x_k, subtracts x_{k-1}, writes x_{k+1}: x_0 is the input, x_j (j >= 1) is 2 + (j - 1) % 3
            const int xk = k == 0 ? in : 2 + (k - 1) % 3;
            const int zk = k == 0 ? -1 : (k == 1 ? in : 2 + (k - 2) % 3);
            const int ok = 2 + k % 3;
            p.xm = M[xk];
            p.xe = E[xk];
            p.zm = zk < 0 ? nullptr : M[zk];
            p.ze = zk < 0 ? nullptr : E[zk];
            p.om = M[ok];
            p.oe = E[ok];
            p.cm = cm[k + 1];
            p.ce = ce[k + 1];
            p.twice = k == 0 ? 0 : 1;
            p.last = k == K - 1;
            xr_order<<<grid, kXrThreads, 0, s>>>(p);
        }
        in = 1 - in;
    }
    gs_count(ctx, 1 + 2 * (int64_t)iters * K);
    if (dist) {
        xr_distance<<<1, kRedThreads, 0, s>>>(n, a, b, vol, log_u, log_v, t, dist, ctx->flags);
        gs_count(ctx, 1);
    }
    return gs_cuda_check(ctx, cudaGetLastError(), "log-domain Sinkhorn");
}
