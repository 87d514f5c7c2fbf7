// Fused Chebyshev heat filter (Sec. 3.5) and the loops built on it: the Sinkhorn scaling loop
// (Algorithm 1) and the fixed-support barycenter (Sec. 3.3).
//
// p_K(L, t) x = sum_{k=0..K} c_k T_k(P) x with P = D^{-1/2} A D^{-1/2}.  One kernel launch per
// order k computes, for every row i,
//     T_k[i] = 2 (P T_{k-1})[i] - T_{k-2}[i]      (T_1 = P x, T_0 = x)
//     y[i]  += c_k T_k[i]                          (y = c_0 x + c_1 T_1 after order 1)
// reading the CSR row of P once, gathering T_{k-1} at its columns, and reading T_{k-2} and y
// at row i only.  T_k overwrites T_{k-2} in place (only row i ever reads T_{k-2}[i]), so two
// vectors plus y carry the whole recurrence.  The last order does not store T_K: it hands
// f = y + c_K T_K to an epilogue (store, Sinkhorn division, barycenter update) that also writes
// the next filter input vol * result, so the loops need no separate elementwise kernels.
//
// Two row mappings:
//   B == 1  : G lanes (a power of two) share a row and split its nonzeros; shuffle reduction.
//   B  > 1  : a group of lanes shares a row and splits its B columns (float4 when B % 4 == 0);
//             each lane walks the row's nonzeros and gathers its slice of each neighbour row.
#include <math.h>
#include <string.h>

#include "gs_internal.cuh"
#include "sell_row.cuh"
#include "async_copy.cuh"

namespace {

struct OrderArgs {
    int64_t n;
    int B;
    const int* rowptr;
    const int* col;
    const float* pval;
    const int* sptr;    // sliced ELL (B == 1 kernel), or null
    const int* scol;
    const float* sval;
    const float* cur;   // T_{k-1} (the gathered block); x for order 1
    const float* prev;  // T_{k-2}; unused for order 1
    float* next;        // destination of T_k (non-last orders), may alias prev
    float* y;           // running sum
    float ck;           // c_k
    float c0;           // c_0 (order 1)
    int first;
    int last;
    const int* done;    // loop early-exit flag (eps stop) or null
    int* flags;         // status bits
    const int* heavy = nullptr;  // B > 1 row-group kernel: rows longer than heavy_len, summed by
    int64_t nheavy = 0;          // split warps
    int heavy_len = 0;           // 0: no split, every row summed by its own lane group
    Epilogue epi;
};

__device__ __forceinline__ void flag(int* flags, int bit) { atomicOr(flags, bit); }

// Zero mass stays zero; a positive numerator over a non-positive or non-finite denominator is
// reported (the result is then inf/NaN/negative and the loop's output is invalid).
__device__ __forceinline__ float safe_div(float num, float den, int* flags)
{
    if (num == 0.f) return 0.f;
    const float r = num / den;
    if (!(r > 0.f) || isinf(r)) flag(flags, GS_FLAG_NONFINITE);
    return r;
}

__device__ __forceinline__ void block_add(double v, double* dst)
{
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (l == 0 && v != 0.0) atomicAdd(dst, v);
    }
}

// ------------------------------------------------------------------------------- B == 1
template <int G>
__global__ void __launch_bounds__(256) order_b1(const OrderArgs p)
{
    if (p.done != nullptr && *p.done) return;
    const int lane = threadIdx.x & (G - 1);
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    const bool active = row < p.n;
    float s = 0.f;
    if (active) {
        const int beg = __ldg(p.rowptr + row), end = __ldg(p.rowptr + row + 1);
        int e = beg + lane;
        for (; e + G < end; e += 2 * G) {
            const int j0 = __ldg(p.col + e), j1 = __ldg(p.col + e + G);
            const float w0 = __ldg(p.pval + e), w1 = __ldg(p.pval + e + G);
            const float x0 = __ldg(p.cur + j0), x1 = __ldg(p.cur + j1);
            s = fmaf(w0, x0, s);
            s = fmaf(w1, x1, s);
        }
        if (e < end) s = fmaf(__ldg(p.pval + e), __ldg(p.cur + __ldg(p.col + e)), s);
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);

    double err = 0.0;
    if (active && lane == 0) {
        const float tk = p.first ? s : fmaf(2.f, s, -p.prev[row]);
        const float acc = p.first ? fmaf(p.ck, tk, p.c0 * p.cur[row]) : fmaf(p.ck, tk, p.y[row]);
        if (!p.last) {
            p.next[row] = tk;
            p.y[row] = acc;
        } else {
            const Epilogue& e = p.epi;
            if (e.kind == EPI_STORE) {
                e.out[row] = acc;
            } else {  // EPI_DIVIDE
                const float num = e.num[row];
                const float r = safe_div(num, acc, p.flags);
                if (e.fsave) e.fsave[row] = acc;
                if (e.out) e.out[row] = r;
                if (e.xnext) e.xnext[row] = e.vol ? e.vol[row] * r : r;
                if (e.old) err = fabs((double)e.old[row] * (double)acc - (double)num);
            }
        }
    }
    if (p.last && p.epi.err_partials != nullptr) block_add(err, p.epi.err_partials);
}

// ------------------------------------------------------------------ B == 1, sliced ELL
// One thread per row; a warp owns one 32-row slice whose entries are stored column-major, so each
// step j reads 32 consecutive column indices and values.  Eight gathers are issued before the
// first is used, and the row-local loads (T_{k-2}, y) go out before the gathers.
// Recurrence update and epilogue of one row, given the row's sum s of P T_{k-1} and its row-local
// values (T_{k-2}, y or c_0 x).  Returns the row's share of the eps-check error.
__device__ __forceinline__ double sell_finish(const OrderArgs& p, int64_t row, float s, float pv, float yv)
{
    double err = 0.0;
    const float tk = p.first ? s : fmaf(2.f, s, -pv);
    const float acc = fmaf(p.ck, tk, yv);
    if (!p.last) {
        p.next[row] = tk;
        p.y[row] = acc;
    } else {
        const Epilogue& e = p.epi;
        if (e.kind == EPI_STORE) {
            e.out[row] = acc;
        } else {  // EPI_DIVIDE
            const float num = e.num[row];
            const float r = safe_div(num, acc, p.flags);
            if (e.fsave) e.fsave[row] = acc;
            if (e.out) e.out[row] = r;
            if (e.xnext) e.xnext[row] = e.vol ? e.vol[row] * r : r;
            if (e.old) err = fabs((double)e.old[row] * (double)acc - (double)num);
        }
    }
    return err;
}

__device__ __forceinline__ double order_sell_row(const OrderArgs& p, int64_t row, bool active)
{
    if (!active) return 0.0;
    const float pv = p.first ? 0.f : p.prev[row];
    const float yv = p.first ? p.c0 * p.cur[row] : p.y[row];
    const float s = gs_sell_row<true>(p.sptr, p.scol, p.sval, p.cur, row);
    return sell_finish(p, row, s, pv, yv);
}

// One block of 1024 threads per SM, each walking one contiguous range of rows, so that one SM's
// gathers fall in one window of the locality order.
__global__ void __launch_bounds__(1024) order_sell_sm_range(const OrderArgs p, int64_t rows_per_block)
{
    if (p.done != nullptr && *p.done) return;
    const int64_t b0 = (int64_t)blockIdx.x * rows_per_block;
    int64_t b1 = b0 + rows_per_block;
    b1 = b1 < p.n ? b1 : p.n;
    double err = 0.0;
    for (int64_t base = b0; base < b1; base += 1024) {
        const int64_t row = base + threadIdx.x;
        err += order_sell_row(p, row, row < b1);
    }
    if (p.last && p.epi.err_partials != nullptr) block_add(err, p.epi.err_partials);
}

// T threads per row (32 / T rows per warp): phase t of a row takes entries j = t, t + T, ...
template <int T>
__global__ void __launch_bounds__(256) order_sell_split(const OrderArgs p)
{
    if (p.done != nullptr && *p.done) return;
    constexpr int RPW = 32 / T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int phase = lane / RPW;
    const int64_t row = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp) * RPW + (lane % RPW);
    const bool active = row < p.n;
    float pv = 0.f, yv = 0.f;
    if (active && phase == 0) {
        pv = p.first ? 0.f : p.prev[row];
        yv = p.first ? p.c0 * p.cur[row] : p.y[row];
    }
    const float s = gs_sell_row_split<T, true>(p.sptr, p.scol, p.sval, p.cur, row, active, phase);
    double err = 0.0;
    if (active && phase == 0) err = sell_finish(p, row, s, pv, yv);
    if (p.last && p.epi.err_partials != nullptr) block_add(err, p.epi.err_partials);
}

__global__ void __launch_bounds__(256) order_sell(const OrderArgs p)
{
    if (p.done != nullptr && *p.done) return;
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double err = order_sell_row(p, row, row < p.n);
    if (p.last && p.epi.err_partials != nullptr) block_add(err, p.epi.err_partials);
}

// Each block walks one contiguous range of 32-row slices (8 slices per pass).
__global__ void __launch_bounds__(256) order_sell_ranged(const OrderArgs p, int64_t rows_per_block)
{
    if (p.done != nullptr && *p.done) return;
    const int64_t b0 = (int64_t)blockIdx.x * rows_per_block;
    int64_t b1 = b0 + rows_per_block;
    b1 = b1 < p.n ? b1 : p.n;
    double err = 0.0;
    for (int64_t base = b0; base < b1; base += 256) {
        const int64_t row = base + threadIdx.x;
        err += order_sell_row(p, row, row < b1);
    }
    if (p.last && p.epi.err_partials != nullptr) block_add(err, p.epi.err_partials);
}

// -------------------------------------------------------------------------------- B > 1
template <int VEC>
struct VecT;
template <>
struct VecT<4> {
    static __device__ __forceinline__ void load(const float* src, float (&v)[4])
    {
        const float4 q = __ldg(reinterpret_cast<const float4*>(src));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <>
struct VecT<1> {
    static __device__ __forceinline__ void load(const float* src, float (&v)[1]) { v[0] = __ldg(src); }
};

template <int VEC>
__device__ __forceinline__ void stream_load(const float* src, float (&v)[VEC])
{
    if constexpr (VEC == 4) {
        const float4 q = __ldcs(reinterpret_cast<const float4*>(src));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) v[i] = __ldcs(src + i);
    }
}

template <int VEC, bool STREAM>
__device__ __forceinline__ void store_vec(float* dst, const float (&v)[VEC])
{
    if constexpr (VEC == 4) {
        const float4 q = make_float4(v[0], v[1], v[2], v[3]);
        if (STREAM) __stcs(reinterpret_cast<float4*>(dst), q);
        else *reinterpret_cast<float4*>(dst) = q;
    } else {
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
            if (STREAM) __stcs(dst + i, v[i]);
            else dst[i] = v[i];
        }
    }
}


// One row of the row-group kernels: the row's lpr lanes each own VEC columns of every chunk of
// lpr * VEC columns.  split = false: the lane group sums the whole row and skips rows longer than
// p.heavy_len (the split warps take those).  split = true: every lane group of the warp is given
// the same row and sums one contiguous segment of its entries; the segments' partial sums are then
// added in segment order and the first group finishes the row.
template <int VEC, int MAXCH>
__device__ __forceinline__ void order_blk_row(const OrderArgs& p, int lpr_log2, int64_t row,
                                              bool active, bool split)
{
    const int lpr = 1 << lpr_log2;
    const int lane = threadIdx.x & (lpr - 1);
    const int B = p.B;
    int beg = 0, end = 0;
    if (active) {
        beg = __ldg(p.rowptr + row);
        end = __ldg(p.rowptr + row + 1);
        if (!split && p.heavy_len > 0 && end - beg > p.heavy_len) active = false;
    }
    const int groups_log2 = split ? 5 - lpr_log2 : 0;
    if (split && groups_log2 > 0) {
        const int gi = (threadIdx.x & 31) >> lpr_log2;
        const int seg = (end - beg + (1 << groups_log2) - 1) >> groups_log2;
        const int sb = min(beg + gi * seg, end);
        end = min(sb + seg, end);
        beg = sb;
    }
    float f[MAXCH][VEC];
#pragma unroll
    for (int ch = 0; ch < MAXCH; ++ch) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) f[ch][v] = 0.f;
        const int c0 = (ch * lpr + lane) * VEC;
        if (!active || c0 >= B) continue;
        float* acc = f[ch];
        int e = beg;
        for (; e + 2 <= end; e += 2) {
            int j[2];
            float w[2], x[2][VEC];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                j[u] = __ldg(p.col + e + u);
                w[u] = __ldg(p.pval + e + u);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) VecT<VEC>::load(p.cur + (int64_t)j[u] * B + c0, x[u]);
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[v] = fmaf(w[u], x[u][v], acc[v]);
        }
        for (; e < end; ++e) {
            float x[VEC];
            const float w = __ldg(p.pval + e);
            VecT<VEC>::load(p.cur + (int64_t)__ldg(p.col + e) * B + c0, x);
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[v] = fmaf(w, x[v], acc[v]);
        }
    }
    if (split && groups_log2 > 0) {
        // the segments' partial sums, added in segment order (every lane gets its column's total)
        const int li = (threadIdx.x & 31) & (lpr - 1);
#pragma unroll
        for (int ch = 0; ch < MAXCH; ++ch)
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                float t = __shfl_sync(0xffffffffu, f[ch][v], li);
                for (int gsrc = 1; gsrc < (1 << groups_log2); ++gsrc)
                    t += __shfl_sync(0xffffffffu, f[ch][v], li + (gsrc << lpr_log2));
                f[ch][v] = t;
            }
        if ((threadIdx.x & 31) >> lpr_log2) active = false;
    }
#pragma unroll
    for (int ch = 0; ch < MAXCH; ++ch) {
        const int c0 = (ch * lpr + lane) * VEC;
        if (!active || c0 >= B) break;
        const float* acc = f[ch];
        const int64_t base = row * (int64_t)B + c0;
        // row-local streams (T_{k-2} and y read, T_k and y written, once per order) are marked
        // evict-first, so they do not push the gathered neighbour rows out of L1 and L2
        float pv[VEC], yv0[VEC];
        if (p.first) {
            stream_load<VEC>(p.cur + base, yv0);
        } else {
            stream_load<VEC>(p.prev + base, pv);
            stream_load<VEC>(p.y + base, yv0);
        }
        float tk[VEC], yv[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            tk[v] = p.first ? acc[v] : fmaf(2.f, acc[v], -pv[v]);
            yv[v] = p.first ? fmaf(p.ck, tk[v], p.c0 * yv0[v]) : fmaf(p.ck, tk[v], yv0[v]);
        }
#pragma unroll
        for (int v = 0; v < VEC; ++v) f[ch][v] = yv[v];
        if (!p.last) {
            store_vec<VEC, true>(p.next + base, tk);
            store_vec<VEC, true>(p.y + base, yv);
        }
    }
    if (!p.last) return;

    const Epilogue& e = p.epi;
    const float vol = (active && e.vol) ? e.vol[row] : 1.f;
    if (e.kind == EPI_STORE || e.kind == EPI_DIVIDE) {
#pragma unroll
        for (int ch = 0; ch < MAXCH; ++ch) {
            const int c0 = (ch * lpr + lane) * VEC;
            if (!active || c0 >= B) break;
            const int64_t base = row * (int64_t)B + c0;
#pragma unroll
            for (int v = 0; v < VEC; ++v) {
                if (e.kind == EPI_STORE) {
                    e.out[base + v] = f[ch][v];
                } else {
                    const float r = safe_div(e.num[base + v], f[ch][v], p.flags);
                    if (e.fsave) e.fsave[base + v] = f[ch][v];
                    if (e.out) e.out[base + v] = r;
                    if (e.xnext) e.xnext[base + v] = vol * r;
                }
            }
        }
        return;
    }

    // EPI_BARY_V: d_i = v_i * f_i; mu = exp(sum_i alpha_i ln d_i); v_i <- v_i mu / d_i.
    double lsum = 0.0;
#pragma unroll
    for (int ch = 0; ch < MAXCH; ++ch) {
        const int c0 = (ch * lpr + lane) * VEC;
        if (!active || c0 >= B) break;
        const int64_t base = row * (int64_t)B + c0;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            if (e.fsave) e.fsave[base + v] = f[ch][v];
            const float d = e.V[base + v] * f[ch][v];
            f[ch][v] = d;
            const double al = e.alpha[c0 + v];
            if (al != 0.0) lsum += al * (double)logf(d);
        }
    }
    for (int off = lpr >> 1; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    const float mu = (float)exp(lsum);
    if (!active) return;
    if (lane == 0) {
        e.mu[row] = mu;
        if (!(mu >= 0.f) || isinf(mu)) flag(p.flags, GS_FLAG_NONFINITE);
    }
#pragma unroll
    for (int ch = 0; ch < MAXCH; ++ch) {
        const int c0 = (ch * lpr + lane) * VEC;
        if (c0 >= B) break;
        const int64_t base = row * (int64_t)B + c0;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const float vnum = e.V[base + v] * mu;
            const float d = f[ch][v];
            const float vn = (vnum == 0.f) ? 0.f : vnum / d;
            if (e.dsave) e.dsave[base + v] = d;
            e.V[base + v] = vn;
            if (e.xnext) e.xnext[base + v] = vol * vn;
        }
    }
}

// The first split_blocks blocks take the long rows (one warp each, dispatched first so that the
// longest chains start first); the rest take every other row, 256 / lpr consecutive rows a block.
template <int VEC, int MAXCH>
__global__ void __launch_bounds__(256) order_blk(const OrderArgs p, int lpr_log2, int split_blocks)
{
    if (p.done != nullptr && *p.done) return;
    if ((int)blockIdx.x < split_blocks) {
        const int64_t h = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
        const bool act = h < p.nheavy;
        const int64_t row = act ? __ldg(p.heavy + h) : 0;
        order_blk_row<VEC, MAXCH>(p, lpr_log2, row, act, true);
        return;
    }
    const int64_t row = ((int64_t)(blockIdx.x - split_blocks) * blockDim.x + threadIdx.x) >> lpr_log2;
    order_blk_row<VEC, MAXCH>(p, lpr_log2, row, row < p.n, false);
}

// Same rows, but each block walks one contiguous range of rows in passes, so that the rows an SM
// works on one after another are neighbours in the locality order and share gathered lines in L1.
template <int VEC, int MAXCH>
__global__ void __launch_bounds__(256) order_blk_ranged(const OrderArgs p, int lpr_log2,
                                                        int64_t rows_per_block)
{
    if (p.done != nullptr && *p.done) return;
    const int rpp = 256 >> lpr_log2;  // rows per pass
    const int64_t b0 = (int64_t)blockIdx.x * rows_per_block;
    int64_t b1 = b0 + rows_per_block;
    b1 = b1 < p.n ? b1 : p.n;
    for (int64_t base = b0; base < b1; base += rpp) {
        const int64_t row = base + (threadIdx.x >> lpr_log2);
        order_blk_row<VEC, MAXCH>(p, lpr_log2, row, row < b1, false);
    }
}

// B = L * V columns, L lanes per row (8, 16 or 32), V consecutive floats per lane (1, 2 or 4).
// The row's column indices and values are fetched L at a time, one entry per lane in a single
// coalesced load, and handed to the group by shuffles, so the gathers of a round never wait on
// an index load (four float4 or eight narrower gathers in flight per lane); the row-local loads
// (T_{k-2}, y) go out before the first round.  Entries are summed in CSR order (the same order as order_blk).
// The first split_blocks blocks take the long rows, one warp per row: its 32 / L groups each sum
// one contiguous segment of the entries and the segments are added in order.
template <int V>
__device__ __forceinline__ void vload(const float* src, float (&v)[V])
{
    if constexpr (V == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(src));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (V == 2) {
        const float2 q = __ldg(reinterpret_cast<const float2*>(src));
        v[0] = q.x; v[1] = q.y;
    } else {
        v[0] = __ldg(src);
    }
}
template <int V>
__device__ __forceinline__ void vload_stream(const float* src, float (&v)[V])
{
    if constexpr (V == 4) {
        const float4 q = __ldcs(reinterpret_cast<const float4*>(src));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (V == 2) {
        const float2 q = __ldcs(reinterpret_cast<const float2*>(src));
        v[0] = q.x; v[1] = q.y;
    } else {
        v[0] = __ldcs(src);
    }
}
template <int V>
__device__ __forceinline__ void vstore_stream(float* dst, const float (&v)[V])
{
    if constexpr (V == 4) __stcs(reinterpret_cast<float4*>(dst), make_float4(v[0], v[1], v[2], v[3]));
    else if constexpr (V == 2) __stcs(reinterpret_cast<float2*>(dst), make_float2(v[0], v[1]));
    else __stcs(dst, v[0]);
}

template <int L, int V>
__global__ void __launch_bounds__(256, 4) order_grp(const OrderArgs p, int split_blocks)
{
    if (p.done != nullptr && *p.done) return;
    constexpr int G = 32 / L;  // row groups per warp
    constexpr int U = V == 4 ? 4 : 8;  // gathers in flight per lane (64 or 32 bytes)
    const int wl = threadIdx.x & 31;
    const int lane = wl & (L - 1);
    const int gi = wl / L;
    const unsigned gmask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << (gi * L));
    const bool split = (int)blockIdx.x < split_blocks;
    int64_t row;
    bool active;
    if (split) {
        const int64_t h = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
        active = h < p.nheavy;
        row = active ? __ldg(p.heavy + h) : 0;
    } else {
        row = ((int64_t)(blockIdx.x - split_blocks) * blockDim.x + threadIdx.x) / L;
        active = row < p.n;
    }
    int beg = 0, end = 0;
    if (active) {
        beg = __ldg(p.rowptr + row);
        end = __ldg(p.rowptr + row + 1);
        if (!split && p.heavy_len > 0 && end - beg > p.heavy_len) active = false;
    }
    if (!active) beg = end = 0;
    if (split && G > 1) {
        const int seg = (end - beg + G - 1) / G;
        const int sb = min(beg + gi * seg, end);
        end = min(sb + seg, end);
        beg = sb;
    }
    constexpr int B = L * V;
    const int64_t base = row * (int64_t)B + lane * V;
    // row-local loads first (the finishing group's lanes only)
    const bool finisher = active && (!split || gi == 0);
    float pv[V], yv0[V];
#pragma unroll
    for (int v = 0; v < V; ++v) pv[v] = yv0[v] = 0.f;
    if (finisher) {
        if (p.first) {
            vload_stream<V>(p.cur + base, yv0);
        } else {
            vload_stream<V>(p.prev + base, pv);
            vload_stream<V>(p.y + base, yv0);
        }
    }
    float acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.f;
    for (int e0 = beg; e0 < end; e0 += L) {
        const int cnt = min(L, end - e0);
        int cj = 0;
        float wj = 0.f;
        if (lane < cnt) {
            cj = __ldg(p.col + e0 + lane);
            wj = __ldg(p.pval + e0 + lane);
        }
        for (int j = 0; j < cnt; j += U) {
            float x[U][V], w[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int jj = j + u;
                const int c = __shfl_sync(gmask, cj, jj & (L - 1), L);
                w[u] = __shfl_sync(gmask, wj, jj & (L - 1), L);
                if (jj < cnt) {
                    vload<V>(p.cur + (int64_t)c * B + lane * V, x[u]);
                } else {
                    w[u] = 0.f;
#pragma unroll
                    for (int v = 0; v < V; ++v) x[u][v] = 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j + u < cnt) {
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[v] = fmaf(w[u], x[u][v], acc[v]);
                }
            }
        }
    }
    if (split && G > 1) {
        // the segments' partial sums, added in segment order (every group gets its column's total)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            float t = __shfl_sync(0xffffffffu, acc[v], lane);
#pragma unroll
            for (int gsrc = 1; gsrc < G; ++gsrc) t += __shfl_sync(0xffffffffu, acc[v], lane + gsrc * L);
            acc[v] = t;
        }
    }
    if (split && gi != 0) return;  // the first group finishes a long row (no shuffles below cross groups)
    float tk[V], f[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        tk[v] = p.first ? acc[v] : fmaf(2.f, acc[v], -pv[v]);
        f[v] = p.first ? fmaf(p.ck, tk[v], p.c0 * yv0[v]) : fmaf(p.ck, tk[v], yv0[v]);
    }
    if (!p.last) {
        if (active) {
            vstore_stream<V>(p.next + base, tk);
            vstore_stream<V>(p.y + base, f);
        }
        return;
    }
    const Epilogue& e = p.epi;
    const float vol = (active && e.vol) ? e.vol[row] : 1.f;
    if (e.kind == EPI_STORE || e.kind == EPI_DIVIDE) {
        if (!active) return;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (e.kind == EPI_STORE) {
                e.out[base + v] = f[v];
            } else {
                const float r = safe_div(e.num[base + v], f[v], p.flags);
                if (e.fsave) e.fsave[base + v] = f[v];
                if (e.out) e.out[base + v] = r;
                if (e.xnext) e.xnext[base + v] = vol * r;
            }
        }
        return;
    }
    // EPI_BARY_V: d_i = v_i * f_i; mu = exp(sum_i alpha_i ln d_i); v_i <- v_i mu / d_i
    const unsigned fmask = split ? ((L == 32) ? 0xffffffffu : ((1u << L) - 1u)) : gmask;
    double lsum = 0.0;
    float d[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        d[v] = 0.f;
        if (!active) continue;
        if (e.fsave) e.fsave[base + v] = f[v];
        d[v] = e.V[base + v] * f[v];
        const double al = e.alpha[lane * V + v];
        if (al != 0.0) lsum += al * (double)logf(d[v]);
    }
    for (int off = L >> 1; off > 0; off >>= 1) lsum += __shfl_xor_sync(fmask, lsum, off, L);
    const float mu = (float)exp(lsum);
    if (!active) return;
    if (lane == 0) {
        e.mu[row] = mu;
        if (!(mu >= 0.f) || isinf(mu)) flag(p.flags, GS_FLAG_NONFINITE);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const float vnum = e.V[base + v] * mu;
        const float vn = (vnum == 0.f) ? 0.f : vnum / d[v];
        if (e.dsave) e.dsave[base + v] = d[v];
        e.V[base + v] = vn;
        if (e.xnext) e.xnext[base + v] = vol * vn;
    }
}

// Shared tail of the float4 row-group kernels: recurrence update and the epilogues.  Every
// thread of the block calls it (the barycenter epilogue reduces across the row's lanes).
template <int LPR>
__device__ __forceinline__ void blk4_finish(const OrderArgs& p, int64_t row, bool active, int lane,
                                            int c0, int64_t base, float (&acc)[4],
                                            const float (&pv)[4], const float (&yv)[4])
{
    float f[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float tk = p.first ? acc[v] : fmaf(2.f, acc[v], -pv[v]);
        f[v] = fmaf(p.ck, tk, yv[v]);
        acc[v] = tk;
    }
    if (!p.last) {
        if (active) {
            *reinterpret_cast<float4*>(p.next + base) = make_float4(acc[0], acc[1], acc[2], acc[3]);
            *reinterpret_cast<float4*>(p.y + base) = make_float4(f[0], f[1], f[2], f[3]);
        }
        return;
    }
    const Epilogue& e = p.epi;
    const float vol = (active && e.vol) ? e.vol[row] : 1.f;
    if (e.kind == EPI_STORE) {
        if (active) *reinterpret_cast<float4*>(e.out + base) = make_float4(f[0], f[1], f[2], f[3]);
        return;
    }
    if (e.kind == EPI_DIVIDE) {
        if (!active) return;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const float r = safe_div(e.num[base + v], f[v], p.flags);
            if (e.fsave) e.fsave[base + v] = f[v];
            if (e.out) e.out[base + v] = r;
            if (e.xnext) e.xnext[base + v] = vol * r;
        }
        return;
    }
    // EPI_BARY_V
    double lsum = 0.0;
    float d[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        d[v] = 0.f;
        if (!active) continue;
        if (e.fsave) e.fsave[base + v] = f[v];
        d[v] = e.V[base + v] * f[v];
        const double al = e.alpha[c0 + v];
        if (al != 0.0) lsum += al * (double)logf(d[v]);
    }
    for (int off = LPR >> 1; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
    const float mu = (float)exp(lsum);
    if (!active) return;
    if (lane == 0) {
        e.mu[row] = mu;
        if (!(mu >= 0.f) || isinf(mu)) flag(p.flags, GS_FLAG_NONFINITE);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const float vnum = e.V[base + v] * mu;
        const float vn = (vnum == 0.f) ? 0.f : vnum / d[v];
        if (e.dsave) e.dsave[base + v] = d[v];
        e.V[base + v] = vn;
        if (e.xnext) e.xnext[base + v] = vol * vn;
    }
}

// B = 4 * LPR columns (float4 per lane, one chunk): each row's neighbour list is staged in
// shared memory 32 entries at a time with one coalesced load per lane, then every lane issues
// eight float4 gathers before consuming them.  Row-local loads go out first.
template <int LPR>
__global__ void __launch_bounds__(256) order_blk_staged(const OrderArgs p)
{
    if (p.done != nullptr && *p.done) return;
    constexpr int RPB = 256 / LPR;
    __shared__ int s_col[RPB][33];
    __shared__ float s_val[RPB][33];
    const int lane = threadIdx.x & (LPR - 1);
    const int rloc = threadIdx.x / LPR;
    const int64_t row = (int64_t)blockIdx.x * RPB + rloc;
    const bool active = row < p.n;
    const int B = 4 * LPR;
    const int c0 = lane * 4;
    const int64_t base = row * (int64_t)B + c0;
    int beg = 0, len = 0;
    float pv[4] = {0.f, 0.f, 0.f, 0.f}, yv[4] = {0.f, 0.f, 0.f, 0.f};
    if (active) {
        beg = __ldg(p.rowptr + row);
        len = __ldg(p.rowptr + row + 1) - beg;
        if (!p.first) {
            const float4 q = *reinterpret_cast<const float4*>(p.prev + base);
            const float4 w = *reinterpret_cast<const float4*>(p.y + base);
            pv[0] = q.x; pv[1] = q.y; pv[2] = q.z; pv[3] = q.w;
            yv[0] = w.x; yv[1] = w.y; yv[2] = w.z; yv[3] = w.w;
        } else {
            const float4 q = __ldg(reinterpret_cast<const float4*>(p.cur + base));
            yv[0] = p.c0 * q.x; yv[1] = p.c0 * q.y; yv[2] = p.c0 * q.z; yv[3] = p.c0 * q.w;
        }
    }
    // warp-uniform chunk count
    int nch = (len + 31) >> 5;
    for (int off = 16; off > 0; off >>= 1) nch = max(nch, __shfl_xor_sync(0xffffffffu, nch, off));
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int ch = 0; ch < nch; ++ch) {
        const int o = ch * 32;
        for (int i = lane; i < 32; i += LPR) {
            const bool ok = o + i < len;
            s_col[rloc][i] = ok ? __ldg(p.col + beg + o + i) : 0;
            s_val[rloc][i] = ok ? __ldg(p.pval + beg + o + i) : 0.f;
        }
        __syncwarp();
        const int cnt = min(32, len - o);
        int e = 0;
        for (; e + 8 <= cnt; e += 8) {
            float4 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                x[u] = __ldg(reinterpret_cast<const float4*>(p.cur + (int64_t)s_col[rloc][e + u] * B + c0));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float w = s_val[rloc][e + u];
                acc[0] = fmaf(w, x[u].x, acc[0]);
                acc[1] = fmaf(w, x[u].y, acc[1]);
                acc[2] = fmaf(w, x[u].z, acc[2]);
                acc[3] = fmaf(w, x[u].w, acc[3]);
            }
        }
        for (; e < cnt; ++e) {
            const float4 x = __ldg(reinterpret_cast<const float4*>(p.cur + (int64_t)s_col[rloc][e] * B + c0));
            const float w = s_val[rloc][e];
            acc[0] = fmaf(w, x.x, acc[0]);
            acc[1] = fmaf(w, x.y, acc[1]);
            acc[2] = fmaf(w, x.z, acc[2]);
            acc[3] = fmaf(w, x.w, acc[3]);
        }
        __syncwarp();
    }
    blk4_finish<LPR>(p, row, active, lane, c0, base, acc, pv, yv);
}


// B = 4 * LPR columns with the gathers issued as asynchronous copies: a block owns RPB
// consecutive rows, whose nonzeros form one contiguous CSR range.  That range is processed in
// chunks of CH neighbour rows (32 KB of data): the chunk's column indices and values are loaded
// coalesced, then every thread issues cp.async copies of 16-byte slices of the neighbour rows into
// shared memory, so hundreds of independent loads per block are in flight at once without holding
// them in registers.  Chunks are double-buffered; each row group then accumulates its own entries
// from shared memory.
template <int LPR>
__global__ void __launch_bounds__(256) order_blk_async(const OrderArgs p)
{
    if (p.done != nullptr && *p.done) return;
    constexpr int B = 4 * LPR;
    constexpr int RPB = 256 / LPR;
    constexpr int CH = 8192 / B;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* sdata = reinterpret_cast<float4*>(smem_raw);           // [2][CH * LPR]
    int* scol = reinterpret_cast<int*>(sdata + 2 * CH * LPR);      // [2][CH]
    float* sval = reinterpret_cast<float*>(scol + 2 * CH);         // [2][CH]
    const int tid = threadIdx.x;
    const int lane = tid % LPR, rloc = tid / LPR;
    const int64_t r0 = (int64_t)blockIdx.x * RPB;
    const int64_t r1 = (r0 + RPB) < p.n ? (r0 + RPB) : p.n;
    const int64_t row = r0 + rloc;
    const bool active = row < r1;
    const int ebeg = __ldg(p.rowptr + r0), eend = __ldg(p.rowptr + r1);
    int myb = 0, mye = 0;
    const int c0 = lane * 4;
    const int64_t base = row * (int64_t)B + c0;
    float pv[4] = {0.f, 0.f, 0.f, 0.f}, yv[4] = {0.f, 0.f, 0.f, 0.f};
    if (active) {
        myb = __ldg(p.rowptr + row);
        mye = __ldg(p.rowptr + row + 1);
        if (!p.first) {
            const float4 q = *reinterpret_cast<const float4*>(p.prev + base);
            const float4 w = *reinterpret_cast<const float4*>(p.y + base);
            pv[0] = q.x; pv[1] = q.y; pv[2] = q.z; pv[3] = q.w;
            yv[0] = w.x; yv[1] = w.y; yv[2] = w.z; yv[3] = w.w;
        } else {
            const float4 q = __ldg(reinterpret_cast<const float4*>(p.cur + base));
            yv[0] = p.c0 * q.x; yv[1] = p.c0 * q.y; yv[2] = p.c0 * q.z; yv[3] = p.c0 * q.w;
        }
    }
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const int nch = (eend - ebeg + CH - 1) / CH;
    auto stage = [&](int c, int buf) {
        const int cb = ebeg + c * CH;
        const int cnt = (eend - cb) < CH ? (eend - cb) : CH;
        for (int i = tid; i < cnt; i += 256) {
            scol[buf * CH + i] = __ldg(p.col + cb + i);
            sval[buf * CH + i] = __ldg(p.pval + cb + i);
        }
        __syncthreads();
        for (int i = tid; i < cnt * LPR; i += 256) {
            const int e = i / LPR, q = i - e * LPR;
            gs_cp_async16(&sdata[buf * CH * LPR + i], p.cur + (int64_t)scol[buf * CH + e] * B + q * 4);
        }
        gs_cp_async_commit();
    };
    if (nch > 0) stage(0, 0);
    for (int c = 0; c < nch; ++c) {
        const int buf = c & 1;
        if (c + 1 < nch) {
            stage(c + 1, buf ^ 1);
            gs_cp_async_wait<1>();
        } else {
            gs_cp_async_wait<0>();
        }
        __syncthreads();
        const int cb = ebeg + c * CH;
        const int ce = (cb + CH) < eend ? (cb + CH) : eend;
        const int lo = myb > cb ? myb : cb, hi = mye < ce ? mye : ce;
        for (int e = lo; e < hi; ++e) {
            const float w = sval[buf * CH + e - cb];
            const float4 x = sdata[buf * CH * LPR + (e - cb) * LPR + lane];
            acc[0] = fmaf(w, x.x, acc[0]);
            acc[1] = fmaf(w, x.y, acc[1]);
            acc[2] = fmaf(w, x.z, acc[2]);
            acc[3] = fmaf(w, x.w, acc[3]);
        }
        __syncthreads();
    }
    blk4_finish<LPR>(p, row, active, lane, c0, base, acc, pv, yv);
}

template <int LPR>
constexpr int blk_async_smem() { return 2 * (8192 / (4 * LPR)) * LPR * 16 + 2 * (8192 / (4 * LPR)) * 8; }

// B = 1 with the gathers issued as 4-byte asynchronous copies: a block owns 256 consecutive rows
// (one per thread); their contiguous CSR range is processed in double-buffered chunks of 2048
// entries (indices and values loaded coalesced, x[col] copied asynchronously into shared memory),
// then each thread sums its own row's entries from shared memory.
constexpr int kB1Chunk = 2048;
__global__ void __launch_bounds__(256) order_b1_async(const OrderArgs p)
{
    if (p.done != nullptr && *p.done) return;
    __shared__ float sx[2][kB1Chunk];
    __shared__ float sval[2][kB1Chunk];
    const int tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * 256;
    const int64_t r1 = (r0 + 256) < p.n ? (r0 + 256) : p.n;
    const int64_t row = r0 + tid;
    const bool active = row < r1;
    const int ebeg = __ldg(p.rowptr + r0), eend = __ldg(p.rowptr + r1);
    int myb = 0, mye = 0;
    float pv = 0.f, yv = 0.f;
    if (active) {
        myb = __ldg(p.rowptr + row);
        mye = __ldg(p.rowptr + row + 1);
        pv = p.first ? 0.f : p.prev[row];
        yv = p.first ? p.c0 * p.cur[row] : p.y[row];
    }
    const int nch = (eend - ebeg + kB1Chunk - 1) / kB1Chunk;
    auto stage = [&](int c, int buf) {
        const int cb = ebeg + c * kB1Chunk;
        const int cnt = (eend - cb) < kB1Chunk ? (eend - cb) : kB1Chunk;
        for (int i = tid; i < cnt; i += 256) {
            const int j = __ldg(p.col + cb + i);
            sval[buf][i] = __ldg(p.pval + cb + i);
            gs_cp_async4(&sx[buf][i], p.cur + j);
        }
        gs_cp_async_commit();
    };
    float s0 = 0.f;
    if (nch > 0) stage(0, 0);
    for (int c = 0; c < nch; ++c) {
        const int buf = c & 1;
        if (c + 1 < nch) {
            stage(c + 1, buf ^ 1);
            gs_cp_async_wait<1>();
        } else {
            gs_cp_async_wait<0>();
        }
        __syncthreads();
        const int cb = ebeg + c * kB1Chunk;
        const int ce = (cb + kB1Chunk) < eend ? (cb + kB1Chunk) : eend;
        const int lo = myb > cb ? myb : cb, hi = mye < ce ? mye : ce;
        for (int e = lo; e < hi; ++e) s0 = fmaf(sval[buf][e - cb], sx[buf][e - cb], s0);
        __syncthreads();
    }
    double err = 0.0;
    if (active) {
        const float tk = p.first ? s0 : fmaf(2.f, s0, -pv);
        const float acc = fmaf(p.ck, tk, yv);
        if (!p.last) {
            p.next[row] = tk;
            p.y[row] = acc;
        } else {
            const Epilogue& e = p.epi;
            if (e.kind == EPI_STORE) {
                e.out[row] = acc;
            } else {  // EPI_DIVIDE
                const float num = e.num[row];
                const float r = safe_div(num, acc, p.flags);
                if (e.fsave) e.fsave[row] = acc;
                if (e.out) e.out[row] = r;
                if (e.xnext) e.xnext[row] = e.vol ? e.vol[row] * r : r;
                if (e.old) err = fabs((double)e.old[row] * (double)acc - (double)num);
            }
        }
    }
    if (p.last && p.epi.err_partials != nullptr) block_add(err, p.epi.err_partials);
}

// ------------------------------------------------------------------------------ helpers
__global__ void fill_kernel(int64_t count, float* __restrict__ out, const float* __restrict__ vol,
                            int B, float value)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    out[i] = vol ? vol[i / B] * value : value;
}

__global__ void sink_init(int32_t* iters_done, int iters, int* done)
{
    if (iters_done) *iters_done = iters;
    if (done) *done = 0;
}

// eps check after a checked u-half-step: stop (keep the previous u) or commit the new u.
__global__ void eps_check(int64_t n, const double* err, double eps, int* done, int32_t* iters_done,
                          int j, float* __restrict__ u, const float* __restrict__ unew, int commit)
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
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        u[i] = unew[i];
}

__global__ void sink_finalize(const int* done, int* flags)
{
    if (!*done) atomicOr(flags, GS_FLAG_NOT_CONVERGED);
}

inline unsigned nblocks(int64_t work, int per) { return (unsigned)((work + per - 1) / per); }

int ilog2(int v)
{
    int r = 0;
    while ((1 << (r + 1)) <= v) ++r;
    return r;
}

// Rows per block for the ranged kernels: one wave of resident blocks (occupancy of the kernel),
// each a contiguous run of whole passes.
template <class Kern>
int resident_blocks_per_sm(Kern kernel)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, 256, 0) != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 4;
    }
    return b;
}

int64_t ranged_rows(const gs_ctx* ctx, int64_t n, int rows_per_pass, int per_sm)
{
    const int64_t blocks = (int64_t)(ctx->num_sms > 0 ? ctx->num_sms : 148) * per_sm;
    int64_t r = (n + blocks - 1) / blocks;
    r = (r + rows_per_pass - 1) / rows_per_pass * rows_per_pass;
    return r > 0 ? r : rows_per_pass;
}

template <int LPR>
void launch_blk_async(gs_ctx* ctx, const gs_graph* g, const OrderArgs& a)
{
    constexpr int smem = blk_async_smem<LPR>();
    static bool attr_set = false;  // per instantiation; set outside any capture by the first call
    if (!attr_set) {
        cudaFuncSetAttribute(order_blk_async<LPR>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr_set = true;
    }
    const unsigned grid = nblocks(g->n, 256 / LPR);
    order_blk_async<LPR><<<grid, 256, smem, ctx->stream>>>(a);
}

// The lane-group kernels for B = L * V: one warp per row (L = 32, V = B / 32) or float4 lanes
// (V = 4, L = B / 4); long rows to split warps in front.  False when B has no such shape.
bool launch_grp(gs_ctx* ctx, const gs_graph* g, int B, bool warp_rows, const OrderArgs& a)
{
    int L = 0, V = 0;
    if (warp_rows && (B == 32 || B == 64 || B == 128)) {
        L = 32;
        V = B / 32;
    } else if (!warp_rows && (B == 32 || B == 64 || B == 128)) {
        L = B / 4;
        V = 4;
    }
    if (!L) return false;
    OrderArgs sa = a;
    int split_blocks = 0;
    if (g->heavy != nullptr && g->nheavy > 0) {
        sa.heavy = g->heavy;
        sa.nheavy = g->nheavy;
        sa.heavy_len = GS_HEAVY_ROW;
        split_blocks = (int)((g->nheavy + 7) / 8);
    }
    const unsigned grid = nblocks(g->n * L, 256) + (unsigned)split_blocks;
    cudaStream_t s = ctx->stream;
    if (L == 32 && V == 1) order_grp<32, 1><<<grid, 256, 0, s>>>(sa, split_blocks);
    else if (L == 32 && V == 2) order_grp<32, 2><<<grid, 256, 0, s>>>(sa, split_blocks);
    else if (L == 32 && V == 4) order_grp<32, 4><<<grid, 256, 0, s>>>(sa, split_blocks);
    else if (L == 8) order_grp<8, 4><<<grid, 256, 0, s>>>(sa, split_blocks);
    else if (L == 16) order_grp<16, 4><<<grid, 256, 0, s>>>(sa, split_blocks);
    else return false;
    return true;
}

void launch_order(gs_ctx* ctx, const gs_graph* g, const FilterPlan& pl, const OrderArgs& a)
{
    gs_count(ctx, 1);
    const int TB = pl.block;
    if (pl.B == 1 && a.epi.kind != EPI_BARY_V) {
        const int mode = pl.kernel;
        if (mode == GS_KERNEL_ASYNC) {
            order_b1_async<<<nblocks(g->n, 256), 256, 0, ctx->stream>>>(a);
            return;
        }
        if ((mode == GS_KERNEL_AUTO || mode == GS_KERNEL_SPLIT) && a.sptr != nullptr) {
            switch (pl.split_t) {
                case 2: order_sell_split<2><<<nblocks(g->n, 8 * 16), 256, 0, ctx->stream>>>(a); break;
                case 8: order_sell_split<8><<<nblocks(g->n, 8 * 4), 256, 0, ctx->stream>>>(a); break;
                default: order_sell_split<4><<<nblocks(g->n, 8 * 8), 256, 0, ctx->stream>>>(a); break;
            }
            return;
        }
        if (mode == GS_KERNEL_SM_RANGE && a.sptr != nullptr) {
            const int blocks = ctx->num_sms > 0 ? ctx->num_sms : 148;
            int64_t rpb = (g->n + blocks - 1) / blocks;
            rpb = (rpb + GS_SELL_C - 1) / GS_SELL_C * GS_SELL_C;
            order_sell_sm_range<<<nblocks(g->n, (int)rpb), 1024, 0, ctx->stream>>>(a, rpb);
            return;
        }
        if (mode == GS_KERNEL_RANGED && a.sptr != nullptr) {
            static const int per_sm = resident_blocks_per_sm(order_sell_ranged);
            const int64_t rpb = ranged_rows(ctx, g->n, 256, per_sm);
            order_sell_ranged<<<nblocks(g->n, (int)rpb), 256, 0, ctx->stream>>>(a, rpb);
            return;
        }
        if (mode == GS_KERNEL_SELL && a.sptr != nullptr) {
            order_sell<<<nblocks(g->n, 256), 256, 0, ctx->stream>>>(a);
            return;
        }
    }
    if (pl.B == 1 && a.epi.kind != EPI_BARY_V) {
        const unsigned grid = nblocks(g->n * pl.group, TB);
        switch (pl.group) {
            case 4: order_b1<4><<<grid, TB, 0, ctx->stream>>>(a); break;
            case 8: order_b1<8><<<grid, TB, 0, ctx->stream>>>(a); break;
            case 16: order_b1<16><<<grid, TB, 0, ctx->stream>>>(a); break;
            default: order_b1<32><<<grid, TB, 0, ctx->stream>>>(a); break;
        }
        return;
    }
    const int vec = pl.vec;
    const int lpr = pl.B == 1 ? 1 : pl.group;
    const unsigned grid = nblocks(g->n * lpr, TB);
    const int blk_mode = pl.kernel;
    if (vec == 4 && pl.B == 4 * lpr && lpr >= 2) {  // one float4 chunk per lane
        const int mode = blk_mode;
        if (mode == GS_KERNEL_ASYNC) {
            switch (lpr) {
                case 2: launch_blk_async<2>(ctx, g, a); return;
                case 4: launch_blk_async<4>(ctx, g, a); return;
                case 8: launch_blk_async<8>(ctx, g, a); return;
                case 16: launch_blk_async<16>(ctx, g, a); return;
                case 32: launch_blk_async<32>(ctx, g, a); return;
                default: break;
            }
        }
        if (mode == GS_KERNEL_STAGED) {
            switch (lpr) {
                case 2: order_blk_staged<2><<<grid, TB, 0, ctx->stream>>>(a); return;
                case 4: order_blk_staged<4><<<grid, TB, 0, ctx->stream>>>(a); return;
                case 8: order_blk_staged<8><<<grid, TB, 0, ctx->stream>>>(a); return;
                case 16: order_blk_staged<16><<<grid, TB, 0, ctx->stream>>>(a); return;
                case 32: order_blk_staged<32><<<grid, TB, 0, ctx->stream>>>(a); return;
                default: break;
            }
        }
    }
    if (pl.B > 1 && (blk_mode == GS_KERNEL_GROUP_WARP || blk_mode == GS_KERNEL_GROUP_VEC4) && vec == 4) {
        if (launch_grp(ctx, g, pl.B, blk_mode == GS_KERNEL_GROUP_WARP, a)) return;
    }
    // chunks of lpr * vec columns each lane group walks (the RHS tile width is lpr * vec)
    const int chunks = (pl.B + lpr * vec - 1) / (lpr * vec);
    const int lg = ilog2(lpr);
    if (pl.B > 1 && blk_mode == GS_KERNEL_RANGED) {
        static const int occ41 = resident_blocks_per_sm(order_blk_ranged<4, 1>);
        static const int occ42 = resident_blocks_per_sm(order_blk_ranged<4, 2>);
        static const int occ48 = resident_blocks_per_sm(order_blk_ranged<4, 8>);
        static const int occ11 = resident_blocks_per_sm(order_blk_ranged<1, 1>);
        static const int occ12 = resident_blocks_per_sm(order_blk_ranged<1, 2>);
        static const int occ18 = resident_blocks_per_sm(order_blk_ranged<1, 8>);
        const int occ = vec == 4 ? (chunks == 1 ? occ41 : (chunks == 2 ? occ42 : occ48))
                                 : (chunks == 1 ? occ11 : (chunks == 2 ? occ12 : occ18));
        const int64_t rpb = ranged_rows(ctx, g->n, TB / lpr, occ);
        const unsigned rgrid = nblocks(g->n, (int)rpb);
        if (vec == 4) {
            if (chunks == 1) order_blk_ranged<4, 1><<<rgrid, TB, 0, ctx->stream>>>(a, lg, rpb);
            else if (chunks == 2) order_blk_ranged<4, 2><<<rgrid, TB, 0, ctx->stream>>>(a, lg, rpb);
            else order_blk_ranged<4, 8><<<rgrid, TB, 0, ctx->stream>>>(a, lg, rpb);
        } else {
            if (chunks == 1) order_blk_ranged<1, 1><<<rgrid, TB, 0, ctx->stream>>>(a, lg, rpb);
            else if (chunks == 2) order_blk_ranged<1, 2><<<rgrid, TB, 0, ctx->stream>>>(a, lg, rpb);
            else order_blk_ranged<1, 8><<<rgrid, TB, 0, ctx->stream>>>(a, lg, rpb);
        }
        return;
    }
    // long rows go to split warps (8 to a block) in front of the regular blocks
    OrderArgs sa = a;
    int split_blocks = 0;
    if (g->heavy != nullptr && g->nheavy > 0) {
        sa.heavy = g->heavy;
        sa.nheavy = g->nheavy;
        sa.heavy_len = GS_HEAVY_ROW;
        split_blocks = (int)((g->nheavy + 7) / 8);
    }
    const unsigned sgrid = grid + (unsigned)split_blocks;
    if (vec == 4) {
        if (chunks == 1) order_blk<4, 1><<<sgrid, TB, 0, ctx->stream>>>(sa, lg, split_blocks);
        else if (chunks == 2) order_blk<4, 2><<<sgrid, TB, 0, ctx->stream>>>(sa, lg, split_blocks);
        else order_blk<4, 8><<<sgrid, TB, 0, ctx->stream>>>(sa, lg, split_blocks);
    } else {
        if (chunks == 1) order_blk<1, 1><<<sgrid, TB, 0, ctx->stream>>>(sa, lg, split_blocks);
        else if (chunks == 2) order_blk<1, 2><<<sgrid, TB, 0, ctx->stream>>>(sa, lg, split_blocks);
        else order_blk<1, 8><<<sgrid, TB, 0, ctx->stream>>>(sa, lg, split_blocks);
    }
}

}  // namespace

FilterPlan gs_filter_plan(const gs_ctx* ctx, const gs_graph* g, int B, bool aligned, int K)
{
    FilterPlan p;
    p.B = B;
    p.block = 256;
    p.vec = (B % 4 == 0 && aligned) ? 4 : 1;
    const TuneRecord* r = gs_tune_lookup(ctx, g, B, K);
    if (B == 1) {
        const float m = g->mean_row;
        p.group = m <= 6.f ? 4 : (m <= 14.f ? 8 : (m <= 28.f ? 16 : 32));
        // variant: the context option, else this graph's tuning, else the record for its size,
        // else the context's last one-column choice
        int split = 0;
        if (ctx->b1_kernel != GS_KERNEL_AUTO) {
            p.kernel = ctx->b1_kernel;
            split = ctx->lanes_override;
        } else if (g->tuned_b1) {
            p.kernel = g->tuned_b1;
            split = g->tuned_split;
        } else if (r) {
            p.kernel = r->kernel;
            split = r->lanes;
        } else {
            p.kernel = ctx->tuned_b1;
        }
        p.split_t = (split == 2 || split == 4 || split == 8) ? split : GS_SPLIT_T;
    } else {
        int lanes = B / p.vec;
        if (lanes > 32) lanes = 32;
        p.group = 1 << ilog2(lanes);
        int tl = 0;
        if (ctx->blk_kernel != GS_KERNEL_AUTO) {
            p.kernel = ctx->blk_kernel;
            tl = ctx->lanes_override;
        } else if (g->tuned_blk_B == B) {
            p.kernel = g->tuned_blk;
            tl = g->tuned_lanes;
        } else if (r) {
            p.kernel = r->kernel;
            tl = r->lanes;
        }
        // a tuned RHS tile width: fewer lanes per row, each walking more chunks (at most 8)
        if (tl > 0 && tl < p.group && (tl & (tl - 1)) == 0 && (B + tl * p.vec - 1) / (tl * p.vec) <= 8)
            p.group = tl;
    }
    return p;
}

// Column counts the row-group kernels cover: at most 8 chunks of (lanes x vec) columns per lane.
bool gs_filter_supports(int B, bool aligned)
{
    if (B < 1) return false;
    if (B == 1) return true;
    return (B % 4 == 0 && aligned) ? B <= 1024 : B <= 256;
}

gs_status gs_filter_enqueue(gs_ctx* ctx, const gs_graph* g, const double* c, int K, int B,
                            float* x, bool x_writable, float* bufA, float* bufB, float* y,
                            const Epilogue& epi_in, const int* done_flag, float** scratch_out)
{
    // float4 rows need every block the kernels read or write as float4 on a 16-byte boundary: the
    // gathered and recurrence blocks, the running sum and the stored output
    const bool aligned = ((uintptr_t)x % 16) == 0 && ((uintptr_t)bufA % 16) == 0 &&
                         (bufB == nullptr || ((uintptr_t)bufB % 16) == 0) && ((uintptr_t)y % 16) == 0 &&
                         (epi_in.out == nullptr || ((uintptr_t)epi_in.out % 16) == 0);
    if (!gs_filter_supports(B, aligned))
        return gs_fail(ctx, GS_ERR_UNSUPPORTED, "B > 256 needs 16-byte aligned blocks with B % 4 == 0");
    const FilterPlan pl = gs_filter_plan(ctx, g, B, aligned, K);
    OrderArgs a;
    const FilterCsr csr = gs_filter_csr(g);
    a.n = g->n;
    a.B = B;
    a.rowptr = csr.rowptr;
    a.col = csr.col;
    a.pval = csr.pval;
    a.sptr = g->sptr;  // present only together with the reordered CSR
    a.scol = g->scol;
    a.sval = g->sval;
    a.done = done_flag;
    a.flags = ctx->flags;
    a.y = y;
    a.c0 = (float)c[0];
    Epilogue epi = epi_in;

    // order 1: T_1 = P x, y = c_0 x + c_1 T_1
    a.cur = x;
    a.prev = nullptr;
    a.ck = (float)c[1];
    a.first = 1;
    if (K == 1) {
        float* scratch = bufA;
        if (epi.xnext_to_scratch) epi.xnext = scratch;
        if (scratch_out) *scratch_out = scratch;
        a.next = nullptr;
        a.last = 1;
        a.epi = epi;
        launch_order(ctx, g, pl, a);
        return gs_cuda_check(ctx, cudaGetLastError(), "Chebyshev order launch");
    }
    a.next = bufA;
    a.last = 0;
    a.epi = Epilogue();
    launch_order(ctx, g, pl, a);

    const float* cur = bufA;
    float* prev = x;
    bool prev_w = x_writable;
    float* spare = bufB;
    a.first = 0;
    for (int k = 2; k <= K; ++k) {
        a.cur = cur;
        a.prev = prev;
        a.ck = (float)c[k];
        if (k < K) {
            float* dst = prev_w ? prev : spare;
            a.next = dst;
            a.last = 0;
            a.epi = Epilogue();
            launch_order(ctx, g, pl, a);
            prev = const_cast<float*>(cur);
            cur = dst;
            prev_w = true;
        } else {
            float* scratch = prev_w ? prev : spare;
            if (epi.xnext_to_scratch) epi.xnext = scratch;
            if (scratch_out) *scratch_out = scratch;
            a.next = nullptr;
            a.last = 1;
            a.epi = epi;
            launch_order(ctx, g, pl, a);
        }
    }
    return gs_cuda_check(ctx, cudaGetLastError(), "Chebyshev order launch");
}

// ------------------------------------------------------------------------ graph capture
template <class F>
gs_status gs_capture(gs_ctx* ctx, F&& body, int reps, cudaGraphExec_t* out)
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
    gs_status st = GS_OK;
    if (e == cudaSuccess)
        for (int r = 0; r < reps && st == GS_OK; ++r) st = body();
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = (e == cudaSuccess) ? cudaStreamEndCapture(ctx->cap, &graph) : e;
    ctx->stream = user;
    ctx->capturing = false;
    if (st != GS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if ((st = gs_cuda_check(ctx, e2, "graph capture")) != GS_OK) return st;
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    return gs_cuda_check(ctx, e, "graph instantiate");
}

void gs_graph_cache_clear(gs_ctx* ctx)
{
    for (auto& en : ctx->gcache) {
        if (en.exec1) cudaGraphExecDestroy(en.exec1);
        if (en.execR) cudaGraphExecDestroy(en.execR);
    }
    ctx->gcache.clear();
    gs_batch_cache_clear(ctx);  // batched tables point into the workspace too
}

// ----------------------------------------------------------------------------- Sinkhorn
gs_status gs_sinkhorn_impl(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b,
                           const float* vol, double t, int K, double eps, int iters, float* u_user,
                           float* v_user, double* dist, int32_t* iters_done)
{
    std::vector<double> c((size_t)K + 1);
    gs_heat_coefficients(t, K, c.data());
    const int64_t n = g->n;
    const bool perm = g->perm != nullptr;       // the loop runs in the filter's node order
    const bool own_uv = perm || !u_user || !v_user;
    const size_t vec = sizeof(float) * (size_t)n;
    WsPlan plan;
    const size_t ix = plan.add(vec), iA = plan.add(vec), iy = plan.add(vec), iu = plan.add(vec),
                 ie = plan.add(sizeof(double) * 2), id = plan.add(sizeof(int) * 2),
                 ip = plan.add(sizeof(double) * gs_reduce_blocks());
    const size_t iuu = own_uv ? plan.add(vec) : 0, ivv = own_uv ? plan.add(vec) : 0;
    const size_t icf = plan.add(sizeof(float) * ((size_t)K + 1)), ibar = plan.add(sizeof(unsigned) * gs_persist_bar_words(ctx));
    const size_t iap = perm ? plan.add(vec) : 0, ibp = perm ? plan.add(vec) : 0,
                 ivp = (perm && vol) ? plan.add(vec) : 0;
    // exchange buffer of the tagged-value persistent kernel (only sizes it can run at)
    const bool want_tag = gs_persist_sync_choice(ctx, g) == 2 &&
                          n <= (int64_t)4 * 1024 * std::max(ctx->num_sms, 1);
    const size_t itg = want_tag ? plan.add(sizeof(unsigned long long) * 3 * (size_t)n) : 0;
    gs_status st = gs_ws_ensure(ctx, plan.total);
    if (st != GS_OK) return st;
    float* x = ws_at<float>(ctx, plan, ix);
    float* A = ws_at<float>(ctx, plan, iA);
    float* y = ws_at<float>(ctx, plan, iy);
    float* ualt = ws_at<float>(ctx, plan, iu);
    double* err = ws_at<double>(ctx, plan, ie);
    int* done = ws_at<int>(ctx, plan, id);
    double* partials = ws_at<double>(ctx, plan, ip);
    float* u = own_uv ? ws_at<float>(ctx, plan, iuu) : u_user;
    float* v = own_uv ? ws_at<float>(ctx, plan, ivv) : v_user;
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
    const bool use_eps = eps > 0.0;
    const int* dflag = use_eps ? done : nullptr;

    sink_init<<<1, 1, 0, ctx->stream>>>(iters_done, iters, done);
    fill_kernel<<<nblocks(n, 256), 256, 0, ctx->stream>>>(n, x, vol, 1, 1.f);  // vol * (v = 1)
    gs_count(ctx, 2);

    auto half = [&](const float* num, float* out, const float* old, double* errp) -> gs_status {
        Epilogue e;
        e.kind = EPI_DIVIDE;
        e.num = num;
        e.vol = vol;
        e.out = out;
        e.old = old;
        e.err_partials = errp;
        e.xnext_to_scratch = true;
        float* scratch = nullptr;
        gs_status s = gs_filter_enqueue(ctx, g, c.data(), K, 1, x, true, A, nullptr, y, e, dflag,
                                        &scratch);
        if (scratch != x) std::swap(x, A);
        return s;
    };
    auto iteration = [&]() -> gs_status {
        gs_status s = half(a, u, nullptr, nullptr);
        if (s == GS_OK) s = half(b, v, nullptr, nullptr);
        return s;
    };

    bool looped = false;
    const TuneRecord* rec = g->tuned_loop ? nullptr : gs_tune_lookup(ctx, g, 1, K);
    const int tl = g->tuned_loop ? g->tuned_loop : (rec && rec->loop ? rec->loop : ctx->tuned_loop);
    const int loop = ctx->loop_mode != 2 ? ctx->loop_mode : (tl == 2 ? 1 : 0);
    if (!use_eps && loop == 0) {
        // Fixed iteration count, persistent mode: the whole loop as one cooperative launch.
        std::vector<float> cf((size_t)K + 1);
        for (int k = 0; k <= K; ++k) cf[k] = (float)c[k];
        float* cdev = ws_at<float>(ctx, plan, icf);
        cudaMemcpyAsync(cdev, cf.data(), sizeof(float) * cf.size(), cudaMemcpyHostToDevice, ctx->stream);
        st = gs_sinkhorn_persistent(ctx, g, a, b, vol, cdev, K, iters, x, A, y, u, v,
                                    ws_at<unsigned>(ctx, plan, ibar),
                                    want_tag ? ws_at<unsigned long long>(ctx, plan, itg) : nullptr);
        if (st == GS_OK) looped = true;
        else if (st != GS_ERR_UNSUPPORTED) return st;
        st = GS_OK;
    }
    if (looped) {
        // done
    } else if (!use_eps) {
        // Fixed iteration count: replay captured CUDA graphs of R and 1 iterations.  Both halves
        // swap the (x, A) roles the same number of times, so every iteration starts from the
        // same buffers and one captured iteration is valid for all of them.
        const int R = iters >= 50 ? 25 : (iters >= 10 ? 10 : 1);
        std::vector<uintptr_t> key = {(uintptr_t)g->rowptr, (uintptr_t)g->col, (uintptr_t)g->pval,
                                      (uintptr_t)n,         (uintptr_t)K,      (uintptr_t)a,
                                      (uintptr_t)b,         (uintptr_t)vol,    (uintptr_t)u,
                                      (uintptr_t)v,         (uintptr_t)ctx->ws, (uintptr_t)R,
                                      (uintptr_t)gs_filter_plan(ctx, g, 1, true, K).kernel,
                                      (uintptr_t)gs_filter_plan(ctx, g, 1, true, K).split_t};
        uint64_t tb;
        memcpy(&tb, &t, sizeof(tb));
        key.push_back((uintptr_t)tb);
        GraphCacheEntry* ent = nullptr;
        for (auto& en : ctx->gcache)
            if (en.key == key) ent = &en;
        if (!ent) {
            GraphCacheEntry en;
            en.key = key;
            en.R = R;
            float* x0 = x;
            float* A0 = A;
            if ((st = gs_capture(ctx, iteration, 1, &en.exec1)) != GS_OK) return st;
            if (R > 1 && (st = gs_capture(ctx, iteration, R, &en.execR)) != GS_OK) {
                cudaGraphExecDestroy(en.exec1);
                return st;
            }
            x = x0;
            A = A0;
            if (ctx->gcache.size() >= 8) {
                cudaGraphExecDestroy(ctx->gcache.front().exec1);
                if (ctx->gcache.front().execR) cudaGraphExecDestroy(ctx->gcache.front().execR);
                ctx->gcache.erase(ctx->gcache.begin());
            }
            ctx->gcache.push_back(en);
            ent = &ctx->gcache.back();
        }
        int left = iters;
        cudaError_t e = cudaSuccess;
        while (R > 1 && left >= R && e == cudaSuccess) {
            e = cudaGraphLaunch(ent->execR, ctx->stream);
            left -= R;
        }
        while (left > 0 && e == cudaSuccess) {
            e = cudaGraphLaunch(ent->exec1, ctx->stream);
            --left;
        }
        gs_count(ctx, (int64_t)iters * 2 * K);
        if ((st = gs_cuda_check(ctx, e, "Sinkhorn graph launch")) != GS_OK) return st;
    } else {
        const unsigned cgrid = (unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
        for (int j = 1; j <= iters && st == GS_OK; ++j) {
            const bool check = j > 1 && ((j - 1) % 10 == 0);
            if (check) {
                cudaMemsetAsync(err, 0, sizeof(double), ctx->stream);
                st = half(a, ualt, u, err);
                eps_check<<<cgrid, 256, 0, ctx->stream>>>(n, err, eps, done, iters_done, j - 1, u,
                                                          ualt, 1);
                gs_count(ctx, 1);
            } else {
                st = half(a, u, nullptr, nullptr);
            }
            if (st == GS_OK) st = half(b, v, nullptr, nullptr);
        }
        if (st != GS_OK) return st;
        if (iters % 10 == 0) {
            cudaMemsetAsync(err, 0, sizeof(double), ctx->stream);
            if ((st = half(a, ualt, u, err)) != GS_OK) return st;
            eps_check<<<1, 32, 0, ctx->stream>>>(n, err, eps, done, iters_done, iters, u, ualt, 0);
            gs_count(ctx, 1);
        }
        sink_finalize<<<1, 1, 0, ctx->stream>>>(done, ctx->flags);
        gs_count(ctx, 1);
    }
    if (dist) {
        if ((st = gs_distance_enqueue(ctx, n, a, b, vol, u, v, t, partials, dist)) != GS_OK)
            return st;
    }
    if (own_uv && u_user && v_user) {
        if (perm) {
            gs_permute_rows(ctx, n, 1, g->perm, u, u_user, false);
            gs_permute_rows(ctx, n, 1, g->perm, v, v_user, false);
        } else {
            cudaMemcpyAsync(u_user, u, vec, cudaMemcpyDeviceToDevice, ctx->stream);
            cudaMemcpyAsync(v_user, v, vec, cudaMemcpyDeviceToDevice, ctx->stream);
        }
    }
    return gs_cuda_check(ctx, cudaGetLastError(), "Sinkhorn loop");
}

// --------------------------------------------------------------------------- barycenter
gs_status gs_barycenter_impl(gs_ctx* ctx, const gs_graph* g, const float* M, int m,
                             const double* alpha, const float* vol, double t, int K, int iters,
                             float* mu_user, float* v_state)
{
    std::vector<double> c((size_t)K + 1);
    gs_heat_coefficients(t, K, c.data());
    const int64_t n = g->n;
    const bool perm = g->perm != nullptr;
    const size_t blk = sizeof(float) * (size_t)n * (size_t)m;
    const size_t vec = sizeof(float) * (size_t)n;
    WsPlan plan;
    const size_t ix = plan.add(blk), iA = plan.add(blk), iy = plan.add(blk), iV = plan.add(blk);
    const size_t iM = perm ? plan.add(blk) : 0, imu = perm ? plan.add(vec) : 0,
                 ivp = (perm && vol) ? plan.add(vec) : 0;
    gs_status st = gs_ws_ensure(ctx, plan.total);
    if (st != GS_OK) return st;
    float* x = ws_at<float>(ctx, plan, ix);
    float* A = ws_at<float>(ctx, plan, iA);
    float* y = ws_at<float>(ctx, plan, iy);
    float* V = ws_at<float>(ctx, plan, iV);
    float* mu = mu_user;
    if (perm) {
        float* Mp = ws_at<float>(ctx, plan, iM);
        gs_permute_rows(ctx, n, m, g->perm, M, Mp, true);
        M = Mp;
        mu = ws_at<float>(ctx, plan, imu);
        if (vol) {
            float* vp = ws_at<float>(ctx, plan, ivp);
            gs_permute_rows(ctx, n, 1, g->perm, vol, vp, true);
            vol = vp;
        }
    }
    const int64_t nm = n * (int64_t)m;
    fill_kernel<<<nblocks(nm, 256), 256, 0, ctx->stream>>>(nm, V, nullptr, m, 1.f);
    fill_kernel<<<nblocks(nm, 256), 256, 0, ctx->stream>>>(nm, x, vol, m, 1.f);
    gs_count(ctx, 2);

    for (int j = 0; j < iters && st == GS_OK; ++j) {
        // w_i = mu_i / H(vol v_i); next input vol * w_i
        Epilogue e1;
        e1.kind = EPI_DIVIDE;
        e1.num = M;
        e1.vol = vol;
        e1.xnext_to_scratch = true;
        float* scratch = nullptr;
        st = gs_filter_enqueue(ctx, g, c.data(), K, m, x, true, A, nullptr, y, e1, nullptr, &scratch);
        if (scratch != x) std::swap(x, A);
        if (st != GS_OK) break;
        // d_i = v_i H(vol w_i); mu = prod d_i^alpha_i; v_i <- v_i mu / d_i; next input vol * v_i
        Epilogue e2;
        e2.kind = EPI_BARY_V;
        e2.vol = vol;
        e2.V = V;
        e2.alpha = alpha;
        e2.mu = mu;
        e2.xnext_to_scratch = true;
        st = gs_filter_enqueue(ctx, g, c.data(), K, m, x, true, A, nullptr, y, e2, nullptr, &scratch);
        if (scratch != x) std::swap(x, A);
    }
    if (st != GS_OK) return st;
    if (perm) {
        gs_permute_rows(ctx, n, 1, g->perm, mu, mu_user, false);
        if (v_state) gs_permute_rows(ctx, n, m, g->perm, V, v_state, false);
    } else if (v_state) {
        cudaMemcpyAsync(v_state, V, blk, cudaMemcpyDeviceToDevice, ctx->stream);
    }
    return gs_cuda_check(ctx, cudaGetLastError(), "barycenter loop");
}
