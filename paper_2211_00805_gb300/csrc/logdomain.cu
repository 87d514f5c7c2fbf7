// Log-domain Geodesic Sinkhorn: Algorithm 1 with the scalings held as FP64 potentials ln u, ln v
// instead of FP32 values, for the small diffusion times where u and v leave the FP32 range (on a
// sphere graph at t = 1 they span e^{-170} .. e^{130}).
//
// With the potentials absorbed into the kernel, H (vol * v) becomes a sum whose terms span the same
// range, and the Chebyshev recurrence of Sec. 3.5 carries them through K orders of signed sums.
// Every vector of the recurrence is therefore held in an extended-range form: an FP32 mantissa m
// and an int32 binary exponent e, value m 2^e (m = 0 for zero), packed in 8 bytes.  Over a row,
// each lane keeps its partial sum as s 2^E and raises E when a larger term arrives (the partial
// is rescaled by an exact power of two); terms are scaled by 2^{e - E} and added in FP32, the
// lanes' partials are aligned the same way, and the row's sum is renormalised (frexpf).  The sums
// carry FP32 rounding only (no exponentials per nonzero); a term more than 2^126 below the row's
// largest one is dropped.  Coefficients c_k are split the same way on the host, so c_K below the
// FP32 range is no problem.
//
// Per Sinkhorn half-step (one application of p_K), K launches over the CSR of P in the graph's
// locality order (marginals, weights and potentials are read and written through the node
// permutation inside the kernels):
//   order 0     : x1 = P x0;                y = c0 x0 + c1 x1
//   order k >= 1: x_{k+1} = 2 P x_k - x_{k-1};  y += c_{k+1} x_{k+1}
// and the last order ends with the division of Algorithm 1 in the log domain,
//   ln u_i = ln a_i - ln y_i  (-inf where a_i = 0; NaN and GS_FLAG_NONFINITE where a_i > 0 and
//   y_i <= 0), and writes the next half-step's input vol_i u_i in the extended form.  One
// iteration's 2K launches are captured once and replayed (the loop is launch-bound on small graphs).
// Then W^2 = 4t sum_i vol_i (a_i ln u_i + b_i ln v_i) from the potentials, in FP64.
//
// Persistent form (default where the graph carries the persistent loop's gather-cache tables):
// the whole fixed-count loop in one cooperative launch over that partition, one 1024-thread block
// per SM, like the FP32 loop.  Each block keeps its slice of P and the distinct-column list in
// shared memory and its rows' recurrence entries (T_k, T_{k-1}, y, the half-step input) in
// registers; every order it stages its distinct neighbour entries into a shared-memory cache and
// sums each row from there in the extended-range arithmetic above (one thread per row, the row's
// entries in the sliced-ELL order, aligned to the row's largest exponent found in a first pass).
// Entries other blocks need are exchanged as 8-byte words
// (FP32 mantissa whose last bit carries the stage parity, int32 exponent) in three rotating
// slots; a reader re-reads a word until its parity is the wanted one (bounded wait, then
// GS_FLAG_TIMEOUT).  The owner keeps the exact mantissa, so the exchanged entries differ from the
// per-order kernels' by at most one unit in the last place.
#include <math.h>

#include <algorithm>
#include <vector>

#include "cache_slices.cuh"
#include "gs_internal.cuh"
#include "sell_row.cuh"

namespace {

constexpr int kZeroExp = -(1 << 30);  // exponent stored with a zero mantissa
constexpr int kLanes = 4;             // lanes summing one row
constexpr int kXrThreads = 256;
constexpr int kRowsPerBlock = kXrThreads / kLanes;
constexpr int kRedThreads = 1024;
constexpr double kLn2 = 0.69314718055994530942;

// One vector entry, value m 2^e; packed so that a gather is one 8-byte load.
struct __align__(8) Xr {
    float m;  // |m| in [0.5, 1), or 0
    int e;    // kZeroExp when m = 0
};

// m 2^d for d <= 0: an exact power of two for d >= -126; the term is dropped below that
__device__ __forceinline__ float scale_pow2(float m, int d)
{
    return d < -126 ? 0.f : m * __int_as_float((d + 127) << 23);
}

// keep the value s 2^E while raising E to at least e (exact: a power-of-two scaling)
__device__ __forceinline__ void xr_raise(float& s, int& E, int e)
{
    if (e > E) {
        s = scale_pow2(s, E - e);
        E = e;
    }
}

// s 2^E as a normalised entry
__device__ __forceinline__ Xr xr_normalise(float s, int E)
{
    if (s == 0.f || E == kZeroExp) return Xr{0.f, kZeroExp};
    int ee;
    const float m = frexpf(s, &ee);
    return Xr{m, E + ee};
}

// y + (m, e) for a nonzero m in [0.25, 1)
__device__ __forceinline__ Xr xr_add(Xr y, float m, int e)
{
    if (y.m == 0.f) return xr_normalise(m, e);
    float s = y.m;
    int E = y.e;
    xr_raise(s, E, e);
    return xr_normalise(s + scale_pow2(m, e - E), E);
}

// the extended form of exp(z) (z = -inf gives zero)
__device__ __forceinline__ Xr xr_from_log(double z)
{
    if (!(z > -INFINITY)) return Xr{0.f, kZeroExp};  // -inf, or NaN (already flagged)
    const double f = floor(z / kLn2);
    return Xr{(float)(0.5 * exp(z - f * kLn2)), (int)f + 1};  // mantissa in [0.5, 1)
}

struct XrOrder {
    int64_t n;
    const int* rowptr;  // the filter's CSR of P (node order of the graph's locality ordering)
    const int* col;
    const float* pval;
    const int* perm;  // filter position -> caller's node index, or null
    const Xr* x;      // T_k x, gathered
    const Xr* z;      // T_{k-1} x, own row only; null in order 0
    Xr* out;          // T_{k+1} x (not written by the last order)
    Xr* y;            // accumulator, own row only
    float c0m;        // order 0: coefficient of T_0 (mantissa, exponent)
    int c0e;
    float cm;  // coefficient of T_{k+1}
    int ce;
    float twice;  // 1: P x (order 0), 2: 2 P x
    int last;     // last order: division epilogue instead of storing y and T_{k+1} x
    const float* marg;  // a (or b) of the division, caller order
    const float* vol;   // vertex weights or null, caller order
    double* logout;     // ln u (or ln v), caller order
    Xr* next;           // next half-step's input vol * u, filter order
    int* flags;
    const int* done;     // eps stop: the loop's early-exit flag, or null
    double* err;         // eps check (last order): adds sum_i |u_i y_i - a_i|, u the committed scaling
    const double* lold;  // eps check: the committed ln u, caller order
};

__global__ void __launch_bounds__(kXrThreads) xr_order(XrOrder p)
{
    if (p.done != nullptr && *p.done) return;
    const int64_t row = (int64_t)blockIdx.x * kRowsPerBlock + (threadIdx.x / kLanes);
    const int lane = threadIdx.x & (kLanes - 1);
    if (row >= p.n) return;  // whole lane groups leave together
    const unsigned gmask = ((1u << kLanes) - 1u) << (threadIdx.x & 31 & ~(kLanes - 1));
    const int beg = p.rowptr[row], end = p.rowptr[row + 1];
    // each lane: s 2^E over its entries, E raised as larger terms arrive
    // (the lane's entries in CSR order; four gathers are issued before the first is summed)
    float s = 0.f;
    int E = kZeroExp;
    int k = beg + lane;
    for (; k + 3 * kLanes < end; k += 4 * kLanes) {
        int c[4];
        float w[4];
        Xr x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = __ldg(p.col + k + u * kLanes);
            w[u] = __ldg(p.pval + k + u * kLanes);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = p.x[c[u]];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (x[u].m != 0.f) {
                xr_raise(s, E, x[u].e);
                s = fmaf(p.twice * w[u], scale_pow2(x[u].m, x[u].e - E), s);
            }
        }
    }
    for (; k < end; k += kLanes) {
        const Xr x = p.x[__ldg(p.col + k)];
        if (x.m != 0.f) {
            xr_raise(s, E, x.e);
            s = fmaf(p.twice * __ldg(p.pval + k), scale_pow2(x.m, x.e - E), s);
        }
    }
    // lane partials combined by a fixed butterfly (both partners compute the same sum)
    for (int off = kLanes / 2; off > 0; off >>= 1) {
        const float so = __shfl_xor_sync(gmask, s, off);
        const int Eo = __shfl_xor_sync(gmask, E, off);
        const int Em = max(E, Eo);
        s = scale_pow2(s, E - Em) + scale_pow2(so, Eo - Em);
        E = Em;
    }
    if (lane != 0) return;
    if (p.z) {
        const Xr z = p.z[row];
        if (z.m != 0.f) {
            xr_raise(s, E, z.e);
            s -= scale_pow2(z.m, z.e - E);
        }
    }
    const Xr xn = xr_normalise(s, E);
    Xr y{0.f, kZeroExp};
    if (p.z) {
        y = p.y[row];
    } else {  // order 0: y = c0 x0
        const Xr x0 = p.x[row];
        if (x0.m != 0.f && p.c0m != 0.f) {
            int ee;
            const float m = frexpf(p.c0m * x0.m, &ee);
            y = Xr{m, p.c0e + x0.e + ee};
        }
    }
    if (xn.m != 0.f && p.cm != 0.f) y = xr_add(y, p.cm * xn.m, p.ce + xn.e);
    if (!p.last) {
        p.out[row] = xn;
        p.y[row] = y;
        return;
    }
    // division epilogue (Algorithm 1) in the log domain
    const int64_t node = p.perm ? p.perm[row] : row;
    const float a = p.marg[node];
    double lu;
    if (a == 0.f) {
        lu = -INFINITY;
    } else if (y.m > 0.f) {
        lu = log((double)a) - (log((double)y.m) + (double)y.e * kLn2);
    } else {
        lu = NAN;
        atomicOr(p.flags, GS_FLAG_NONFINITE);
    }
    p.logout[node] = lu;
    p.next[row] = xr_from_log(lu + (p.vol ? log((double)p.vol[node]) : 0.0));
    if (p.err != nullptr && a != 0.f)  // u_old y - a = a (u_old / u_new - 1), as ln u_new = ln a - ln y
        atomicAdd(p.err, (double)a * fabs(expm1(p.lold[node] - lu)));
}

__global__ void xr_eps_init(int* done, int32_t* iters_done, int iters)
{
    if (done) *done = 0;
    if (iters_done) *iters_done = iters;
}

// After a checked u half-step (new ln u in lalt, error of the committed ln u in *err): stop at
// iteration j keeping the committed scalings, or commit the new ln u.
__global__ void xr_eps_check(int64_t n, const double* err, double eps, int* done, int32_t* iters_done, int j,
                             double* __restrict__ lu, const double* __restrict__ lalt, int commit)
{
    if (*done) return;
    if (*err < eps) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            *done = 1;
            if (iters_done) *iters_done = j;
        }
        return;
    }
    if (!commit) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        lu[i] = lalt[i];
}

__global__ void xr_eps_finalize(const int* done, int* flags)
{
    if (!*done) atomicOr(flags, GS_FLAG_NOT_CONVERGED);
}

// x0 = vol * 1 (the first half-step's input, v = 1), filter order
__global__ void xr_init(int64_t n, const int* __restrict__ perm, const float* __restrict__ vol, Xr* __restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = xr_from_log(vol ? log((double)vol[perm ? perm[i] : i]) : 0.0);
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

// ------------------------------------------------------------------------- persistent loop
constexpr int kLoopThreads = 1024;
constexpr long long kLoopBudget = 4000000000ll;  // clock cycles a wait may take (~2 s)
// Self-test (GS_OPT_BARRIER_SELFTEST): every staging wait looks for a parity no word carries, so
// each runs out after this much shorter budget and the launch ends with GS_FLAG_TIMEOUT.
constexpr long long kLoopSelfTestBudget = 20000000ll;

struct XrLoopArgs {
    int n;
    const int* sptr;  // sliced ELL of P (locality order) and the gather-cache tables
    const float* sval;
    const uint16_t* xc_lidx;
    const int* xc_ucol;
    const int* xc_ucnt;
    const int* xc_rows;
    int xc_max_e, xc_max_u;
    const int* perm;    // filter position -> caller's node (null: identity)
    const float* a;     // caller order
    const float* b;
    const float* vol;
    double* log_u;      // caller order
    double* log_v;
    const float* cm;    // [K + 1] coefficient mantissas / exponents
    const int* ce;
    int K, iters;
    unsigned long long* words;  // [3][n] exchange words
    int* flags;
    long long budget;   // clock cycles a wait may take
    int selftest;       // wait for a parity no word carries (bounded-wait self-test)
};

__device__ __forceinline__ unsigned long long xr_pack(Xr v, unsigned parity)
{
    return ((unsigned long long)(unsigned)v.e << 32) | (unsigned long long)((__float_as_uint(v.m) & ~1u) | parity);
}
__device__ __forceinline__ Xr xr_unpack(unsigned long long w)
{
    const float m = __uint_as_float((unsigned)w & ~1u);
    return m == 0.f ? Xr{0.f, kZeroExp} : Xr{m, (int)(w >> 32)};
}
__device__ __forceinline__ unsigned long long xr_ld(const unsigned long long* a)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ void xr_st(unsigned long long* a, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;\n" ::"l"(a), "l"(v) : "memory");
}

// Algorithm 1's division in the log domain for one row: ln u = ln a - ln y (FP64); returns the
// next half-step's input vol * u in the extended form.
__device__ __forceinline__ Xr xr_divide(float a, Xr y, double lvol, double* logout, int* flags)
{
    double lu;
    if (a == 0.f) {
        lu = -INFINITY;
    } else if (y.m > 0.f) {
        lu = log((double)a) - (log((double)y.m) + (double)y.e * kLn2);
    } else {
        lu = NAN;
        atomicOr(flags, GS_FLAG_NONFINITE);
    }
    *logout = lu;
    return xr_from_log(lu + lvol);
}

template <int RPT, bool GROUP>
__global__ void __launch_bounds__(kLoopThreads) xr_loop(const XrLoopArgs p)
{
    __shared__ int s_ok;
    __shared__ __align__(8) unsigned long long s_mbar;
    extern __shared__ __align__(128) unsigned char x_smem[];
    if (threadIdx.x == 0) s_ok = 1;
    __syncthreads();
    const int r0 = __ldg(p.xc_rows + blockIdx.x), r1 = __ldg(p.xc_rows + blockIdx.x + 1);
    const int emax = (p.xc_max_e + 31) / 32 * 32, umax = (p.xc_max_u + 31) / 32 * 32;
    float* sval_s = reinterpret_cast<float*>(x_smem);
    uint16_t* lidx_s = reinterpret_cast<uint16_t*>(x_smem + (size_t)emax * 4);
    int* ucol_s = reinterpret_cast<int*>(x_smem + (size_t)emax * 6);
    Xr* xc = reinterpret_cast<Xr*>(x_smem + (size_t)emax * 6 + (size_t)umax * 4);
    int e0 = 0, ucnt = 0;
    bool timed_out = false;
    if (!gs_load_cache_tables(p.sptr, p.sval, p.xc_lidx, p.xc_ucol, p.xc_ucnt, (int)blockIdx.x, r0, r1, kLoopBudget,
                              sval_s, lidx_s, ucol_s, &e0, &ucnt, &s_mbar, &timed_out))
        s_ok = 0;
    if (timed_out) atomicOr(p.flags, GS_FLAG_TIMEOUT);
    __syncthreads();
    if (!s_ok || r0 >= r1) return;
    const size_t n = (size_t)p.n;

    int off[RPT], width[RPT], node[RPT];
    float av[RPT], bv[RPT];
    double lvol[RPT];
    Xr x0[RPT], xk[RPT], xkm1[RPT], y[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int row = r0 + (int)threadIdx.x + j * kLoopThreads;
        off[j] = width[j] = node[j] = 0;
        av[j] = bv[j] = 0.f;
        lvol[j] = 0.0;
        x0[j] = xk[j] = xkm1[j] = y[j] = Xr{0.f, kZeroExp};
        if (row < r1) {
            const int sl = row / 32;
            const int beg = __ldg(p.sptr + sl);
            width[j] = (__ldg(p.sptr + sl + 1) - beg) / 32;
            off[j] = beg - e0 + row % 32;
            node[j] = p.perm ? __ldg(p.perm + row) : row;
            av[j] = __ldg(p.a + node[j]);
            bv[j] = __ldg(p.b + node[j]);
            lvol[j] = p.vol ? log((double)__ldg(p.vol + node[j])) : 0.0;
            x0[j] = xr_from_log(lvol[j]);  // vol * (v = 1)
            xr_st(p.words + row, xr_pack(x0[j], 0u));  // stage 0 in slot 0
        }
    }
    unsigned stage = 0;
    int rslot = 0, wslot = 1;
    const int K = p.K;
    for (int it = 0; it < p.iters; ++it) {
        for (int h = 0; h < 2; ++h) {
            for (int k = 0; k < K; ++k) {
                ++stage;
                const unsigned long long* src = p.words + (size_t)rslot * n;
                unsigned long long* dst = p.words + (size_t)wslot * n;
                const unsigned want = p.selftest ? 2u : ((stage - 1u) & 1u);
                for (int i0 = threadIdx.x; i0 < ucnt; i0 += 8 * kLoopThreads) {
                    unsigned long long w[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int i = i0 + u * kLoopThreads;
                        w[u] = i < ucnt ? xr_ld(src + ucol_s[i]) : 0ull;
                    }
                    // words not yet carrying the wanted parity are re-read together (GROUP: one
                    // round trip per retry round) or one at a time, as in the FP32 loop
                    if (GROUP) {
                        unsigned pending = 0;
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (i0 + u * kLoopThreads < ucnt && ((unsigned)w[u] & 1u) != want) pending |= 1u << u;
                        if (pending) {
                            const long long t0 = clock64();
                            do {
#pragma unroll
                                for (int u = 0; u < 8; ++u)
                                    if (pending & (1u << u)) w[u] = xr_ld(src + ucol_s[i0 + u * kLoopThreads]);
#pragma unroll
                                for (int u = 0; u < 8; ++u)
                                    if ((pending & (1u << u)) && ((unsigned)w[u] & 1u) == want) pending &= ~(1u << u);
                                if (pending && clock64() - t0 > p.budget) {
                                    atomicOr(p.flags, GS_FLAG_TIMEOUT);
                                    s_ok = 0;
                                    break;
                                }
                            } while (pending);
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int i = i0 + u * kLoopThreads;
                            if (i < ucnt) xc[i] = xr_unpack(w[u]);
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int i = i0 + u * kLoopThreads;
                            if (i >= ucnt) break;
                            if (((unsigned)w[u] & 1u) != want) {
                                const long long t0 = clock64();
                                do {
                                    w[u] = xr_ld(src + ucol_s[i]);
                                    if (clock64() - t0 > p.budget) {
                                        atomicOr(p.flags, GS_FLAG_TIMEOUT);
                                        s_ok = 0;
                                        break;
                                    }
                                } while (((unsigned)w[u] & 1u) != want);
                            }
                            xc[i] = xr_unpack(w[u]);
                        }
                    }
                }
                __syncthreads();
                if (!s_ok) return;
                const float twice = k == 0 ? 1.f : 2.f;
                const float cm = p.cm[k + 1];
                const int ce = p.ce[k + 1];
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const int row = r0 + (int)threadIdx.x + j * kLoopThreads;
                    if (row >= r1) continue;
                    // the row's sum s 2^E over its stored entries (padding entries have weight 0):
                    // first the largest exponent E of the row's terms, then the terms aligned to it
                    const float* vp = sval_s + off[j];
                    const int r = (int)threadIdx.x & 31;
                    const uint16_t* lp = lidx_s + off[j] - r;  // the slice's paired local indices
                    int E = (k > 0 && xkm1[j].m != 0.f) ? xkm1[j].e : kZeroExp;
                    gs_cached_lidx_each(lp, r, width[j], [&](int q, unsigned li) {
                        const Xr x = xc[li];
                        if (vp[q * 32] != 0.f && x.m != 0.f) E = max(E, x.e);
                    });
                    float s = 0.f;
                    gs_cached_lidx_each(lp, r, width[j], [&](int q, unsigned li) {
                        const float v = vp[q * 32];
                        const Xr x = xc[li];
                        if (v != 0.f && x.m != 0.f) s = fmaf(twice * v, scale_pow2(x.m, x.e - E), s);
                    });
                    if (k > 0 && xkm1[j].m != 0.f)  // T_{k+1} = 2 P T_k - T_{k-1}
                        s -= scale_pow2(xkm1[j].m, xkm1[j].e - E);
                    const Xr xn = xr_normalise(s, E);
                    if (k == 0) {  // y = c0 x0
                        y[j] = Xr{0.f, kZeroExp};
                        if (x0[j].m != 0.f && p.cm[0] != 0.f) {
                            int ee;
                            const float m = frexpf(p.cm[0] * x0[j].m, &ee);
                            y[j] = Xr{m, p.ce[0] + x0[j].e + ee};
                        }
                    }
                    if (xn.m != 0.f && cm != 0.f) y[j] = xr_add(y[j], cm * xn.m, ce + xn.e);
                    Xr pub;
                    if (k < K - 1) {
                        xkm1[j] = k == 0 ? x0[j] : xk[j];
                        xk[j] = xn;
                        pub = xn;
                    } else {
                        x0[j] = xr_divide(h == 0 ? av[j] : bv[j], y[j], lvol[j],
                                          (h == 0 ? p.log_u : p.log_v) + node[j], p.flags);
                        xk[j] = x0[j];
                        pub = x0[j];
                    }
                    xr_st(dst + row, xr_pack(pub, stage & 1u));
                }
                __syncthreads();  // xc is refilled by the next order
                rslot = wslot;
                wslot = wslot == 2 ? 0 : wslot + 1;
            }
        }
    }
}

// The whole loop as one cooperative launch; GS_ERR_UNSUPPORTED (nothing enqueued) when the
// graph has no gather-cache partition of one block per SM, its tables do not fit in shared
// memory, or the device cannot co-schedule the grid.
gs_status xr_loop_launch(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b, const float* vol,
                         const float* cmd, const int* ced, int K, int iters, double* log_u, double* log_v,
                         unsigned long long* words)
{
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    if (!coop || !g->xc_ok || !g->sptr || ctx->num_sms < 1 || g->xc_blocks != ctx->num_sms || g->n >= (1ll << 31))
        return GS_ERR_UNSUPPORTED;
    const int rpt = (g->xc_rpb + kLoopThreads - 1) / kLoopThreads;
    const size_t emax = (size_t)(g->xc_max_e + 31) / 32 * 32, umax = (size_t)(g->xc_max_u + 31) / 32 * 32;
    const size_t smem = emax * 6 + umax * 12;
    if (rpt < 1 || rpt > 2 || smem > 200 * 1024) return GS_ERR_UNSUPPORTED;
    // staging re-reads as the FP32 loop takes them on this graph (grouped where blocks are large)
    const int form = gs_persist_sync_setting(ctx, g);
    const bool group = form == 2 || (form != 4 && gs_tagged_form(g) == 2);
    void (*kern)(XrLoopArgs) = rpt == 1 ? (group ? xr_loop<1, true> : xr_loop<1, false>)
                                        : (group ? xr_loop<2, true> : xr_loop<2, false>);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_UNSUPPORTED;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLoopThreads, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return GS_ERR_UNSUPPORTED;
    }
    XrLoopArgs p;
    p.n = (int)g->n;
    p.sptr = g->sptr;
    p.sval = g->sval;
    p.xc_lidx = g->xc_lidx;
    p.xc_ucol = g->xc_ucol;
    p.xc_ucnt = g->xc_ucnt;
    p.xc_rows = g->xc_rows;
    p.xc_max_e = g->xc_max_e;
    p.xc_max_u = g->xc_max_u;
    p.perm = g->perm;
    p.a = a;
    p.b = b;
    p.vol = vol;
    p.log_u = log_u;
    p.log_v = log_v;
    p.cm = cmd;
    p.ce = ced;
    p.K = K;
    p.iters = iters;
    p.words = words;
    p.flags = ctx->flags;
    p.budget = ctx->barrier_selftest ? kLoopSelfTestBudget : kLoopBudget;
    p.selftest = ctx->barrier_selftest;
    // slot k must not start with stage k's parity: slots 0 and 2 odd, slot 1 even
    const size_t bytes = sizeof(unsigned long long) * (size_t)g->n;
    cudaMemsetAsync(words, 0x01, bytes, ctx->stream);
    cudaMemsetAsync(words + g->n, 0x00, bytes, ctx->stream);
    cudaMemsetAsync(words + 2 * g->n, 0x01, bytes, ctx->stream);
    void* params[] = {&p};
    const cudaError_t e = cudaLaunchCooperativeKernel((void*)kern, dim3((unsigned)g->xc_blocks), dim3(kLoopThreads),
                                                      params, smem, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_UNSUPPORTED;
    }
    ctx->barrier_selftest = 0;  // the self-test applies to one launch
    gs_count(ctx, 1);
    return GS_OK;
}

// Runs body() once under stream capture on the context's private capture stream (ctx->stream
// points there meanwhile, and launches are not counted) and instantiates the graph.
template <class F>
gs_status capture_iteration(gs_ctx* ctx, F&& body, cudaGraphExec_t* out)
{
    if (!ctx->cap) {
        gs_status st = gs_cuda_check(ctx, cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking),
                                     "capture stream");
        if (st != GS_OK) return st;
    }
    cudaStream_t user = ctx->stream;
    ctx->stream = ctx->cap;
    ctx->capturing = true;
    cudaError_t e = cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal);
    const gs_status st = e == cudaSuccess ? body() : GS_OK;
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(ctx->cap, &graph) : e;
    ctx->stream = user;
    ctx->capturing = false;
    if (st != GS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    gs_status st2 = gs_cuda_check(ctx, e2, "graph capture");
    if (st2 != GS_OK) return st2;
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    return gs_cuda_check(ctx, e, "graph instantiate");
}

}  // namespace

gs_status gs_sinkhorn_log_impl(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b, const float* vol,
                               double t, int K, double eps, int iters, double* log_u, double* log_v, double* dist,
                               int32_t* iters_done)
{
    const int64_t n = g->n;
    const bool reordered = g->perm && g->prowptr;
    const FilterCsr fc = reordered ? gs_filter_csr(g) : FilterCsr{g->rowptr, g->col, g->pval};
    const bool use_eps = eps > 0.0;
    WsPlan plan;
    size_t ix[6];
    for (int i = 0; i < 6; ++i) ix[i] = plan.add(sizeof(Xr) * (size_t)n);  // two inputs, three vectors, y
    // eps stop: the checked half-step's ln u, the error and the early-exit flag
    const size_t ialt = use_eps ? plan.add(sizeof(double) * (size_t)n) : 0;
    const size_t ierr = use_eps ? plan.add(sizeof(double) + sizeof(int)) : 0;
    gs_status st = gs_ws_ensure(ctx, plan.total);
    if (st != GS_OK) return st;
    Xr* X[6];
    for (int i = 0; i < 6; ++i) X[i] = ws_at<Xr>(ctx, plan, ix[i]);
    double* lalt = use_eps ? ws_at<double>(ctx, plan, ialt) : nullptr;
    double* err = use_eps ? ws_at<double>(ctx, plan, ierr) : nullptr;
    int* done = use_eps ? reinterpret_cast<int*>(err + 1) : nullptr;
    std::vector<double> c((size_t)K + 1);
    gs_heat_coefficients(t, K, c.data());
    std::vector<float> cm((size_t)K + 1);
    std::vector<int> ce((size_t)K + 1);
    for (int k = 0; k <= K; ++k) {
        int ee;
        cm[k] = (float)frexp(c[k], &ee);
        ce[k] = ee;
    }
    const unsigned grid = (unsigned)((n + kRowsPerBlock - 1) / kRowsPerBlock);
    // one half-step of K orders: half 0 reads buffer 0 and writes the next input to buffer 1, half 1
    // the other way round; chk: write ln u to lalt and add its marginal error to *err
    auto half_step = [&](int half, bool chk) -> gs_status {
        const int in = half;
        XrOrder p{};
        p.n = n;
        p.rowptr = fc.rowptr;
        p.col = fc.col;
        p.pval = fc.pval;
        p.perm = reordered ? g->perm : nullptr;
        p.y = X[5];
        p.c0m = cm[0];
        p.c0e = ce[0];
        p.marg = half == 0 ? a : b;
        p.vol = vol;
        p.logout = chk ? lalt : (half == 0 ? log_u : log_v);
        p.next = X[1 - in];
        p.flags = ctx->flags;
        p.done = done;
        p.err = chk ? err : nullptr;
        p.lold = chk ? log_u : nullptr;
        for (int k = 0; k < K; ++k) {
            // x_0 is the input; x_j (j >= 1) lives in buffer 2 + (j - 1) % 3
            p.x = X[k == 0 ? in : 2 + (k - 1) % 3];
            p.z = k == 0 ? nullptr : X[k == 1 ? in : 2 + (k - 2) % 3];
            p.out = X[2 + k % 3];
            p.cm = cm[k + 1];
            p.ce = ce[k + 1];
            p.twice = k == 0 ? 1.f : 2.f;
            p.last = k == K - 1;
            xr_order<<<grid, kXrThreads, 0, ctx->stream>>>(p);
        }
        return gs_cuda_check(ctx, cudaGetLastError(), "log-domain Sinkhorn order");
    };
    auto iteration = [&]() -> gs_status {
        const gs_status s0 = half_step(0, false);
        return s0 != GS_OK ? s0 : half_step(1, false);
    };
    cudaStream_t s = ctx->stream;
    xr_eps_init<<<1, 1, 0, s>>>(done, iters_done, iters);
    gs_count(ctx, 1);
    if (!use_eps && ctx->loop_mode != 1 && reordered) {
        // the whole loop in one persistent launch (GS_OPT_LOOP 1 keeps the per-order launches)
        WsPlan lp;
        const size_t icm = lp.add(sizeof(float) * (size_t)(K + 1)), ice = lp.add(sizeof(int) * (size_t)(K + 1)),
                     iw = lp.add(sizeof(unsigned long long) * 3 * (size_t)n);
        if ((st = gs_ws_ensure(ctx, plan.total + lp.total + 256)) != GS_OK) return st;
        for (int i = 0; i < 6; ++i) X[i] = ws_at<Xr>(ctx, plan, ix[i]);
        char* base = static_cast<char*>(ctx->ws) + ((plan.total + 255) & ~(size_t)255);
        float* cmd = reinterpret_cast<float*>(base + lp.offs[icm]);
        int* ced = reinterpret_cast<int*>(base + lp.offs[ice]);
        unsigned long long* words = reinterpret_cast<unsigned long long*>(base + lp.offs[iw]);
        cudaMemcpyAsync(cmd, cm.data(), sizeof(float) * (size_t)(K + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(ced, ce.data(), sizeof(int) * (size_t)(K + 1), cudaMemcpyHostToDevice, s);
        st = xr_loop_launch(ctx, g, a, b, vol, cmd, ced, K, iters, log_u, log_v, words);
        if (st == GS_OK) {
            if (dist) {
                xr_distance<<<1, kRedThreads, 0, s>>>(n, a, b, vol, log_u, log_v, t, dist, ctx->flags);
                gs_count(ctx, 1);
            }
            return gs_cuda_check(ctx, cudaGetLastError(), "log-domain Sinkhorn");
        }
        if (st != GS_ERR_UNSUPPORTED) return st;
    }
    xr_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, reordered ? g->perm : nullptr, vol, X[0]);
    if (use_eps) {
        // the eps stop of gs_sinkhorn: at the start of iteration j (j - 1 a multiple of 10) the u
        // half-step also measures the marginal error of the committed u; below eps the loop stops
        // there (later launches return at once), otherwise the new u is committed
        const unsigned cgrid = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
        for (int j = 1; j <= iters && st == GS_OK; ++j) {
            if (j > 1 && (j - 1) % 10 == 0) {
                cudaMemsetAsync(err, 0, sizeof(double), s);
                st = half_step(0, true);
                xr_eps_check<<<cgrid, 256, 0, s>>>(n, err, eps, done, iters_done, j - 1, log_u, lalt, 1);
                gs_count(ctx, 1);
            } else {
                st = half_step(0, false);
            }
            if (st == GS_OK) st = half_step(1, false);
        }
        if (st != GS_OK) return st;
        if (iters % 10 == 0) {
            cudaMemsetAsync(err, 0, sizeof(double), s);
            if ((st = half_step(0, true)) != GS_OK) return st;
            xr_eps_check<<<1, 32, 0, s>>>(n, err, eps, done, iters_done, iters, log_u, lalt, 0);
            gs_count(ctx, 1 + K);
        }
        xr_eps_finalize<<<1, 1, 0, s>>>(done, ctx->flags);
        gs_count(ctx, 2 + 2 * (int64_t)iters * K);
    } else if (iters == 1) {
        if ((st = iteration()) != GS_OK) return st;
    } else {  // launch-bound on small graphs: replay one captured iteration
        cudaGraphExec_t exec = nullptr;
        if ((st = capture_iteration(ctx, iteration, &exec)) != GS_OK) return st;
        cudaError_t e = cudaSuccess;
        for (int it = 0; it < iters && e == cudaSuccess; ++it) e = cudaGraphLaunch(exec, s);
        cudaGraphExecDestroy(exec);  // freed once the launches above have run
        if ((st = gs_cuda_check(ctx, e, "log-domain Sinkhorn replay")) != GS_OK) return st;
    }
    if (!use_eps) gs_count(ctx, 1 + 2 * (int64_t)iters * K);
    if (dist) {
        xr_distance<<<1, kRedThreads, 0, s>>>(n, a, b, vol, log_u, log_v, t, dist, ctx->flags);
        gs_count(ctx, 1);
    }
    return gs_cuda_check(ctx, cudaGetLastError(), "log-domain Sinkhorn");
}
