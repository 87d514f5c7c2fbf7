// One row of P times a block column in the sliced-ELL layout (GS_SELL_C-row slices stored
// column-major, padding entries have value 0), shared by the launch-per-order, persistent and
// batched kernels so that they sum in exactly the same order.  READONLY: the gathered vector is
// constant for the kernel's lifetime and may use the read-only cache; otherwise ordinary
// coherent loads are used.
#pragma once
#include <stdint.h>

template <bool READONLY>
__device__ __forceinline__ float gs_ld(const float* p)
{
    if (READONLY) return __ldg(p);
    return *p;
}

// Dot product of one sliced-ELL row: cp / vp point at the row's first column index / value,
// successive entries GS_SELL_C words apart.  GLOBAL_GRAPH: cp / vp are in global memory (read-only
// path); otherwise they are in shared memory.
template <bool READONLY, bool GLOBAL_GRAPH>
__device__ __forceinline__ float gs_sell_dot(const int* cp, const float* vp, int width, const float* cur)
{
    float s0 = 0.f, s1 = 0.f;
    int j = 0;
    for (; j + 8 <= width; j += 8) {
        int c[8];
        float w[8], x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            c[u] = GLOBAL_GRAPH ? __ldg(cp + (j + u) * GS_SELL_C) : cp[(j + u) * GS_SELL_C];
            w[u] = GLOBAL_GRAPH ? __ldg(vp + (j + u) * GS_SELL_C) : vp[(j + u) * GS_SELL_C];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = gs_ld<READONLY>(cur + c[u]);
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            s0 = fmaf(w[u], x[u], s0);
            s1 = fmaf(w[u + 1], x[u + 1], s1);
        }
    }
    for (; j < width; ++j) {
        const int c = GLOBAL_GRAPH ? __ldg(cp + j * GS_SELL_C) : cp[j * GS_SELL_C];
        const float w = GLOBAL_GRAPH ? __ldg(vp + j * GS_SELL_C) : vp[j * GS_SELL_C];
        s0 = fmaf(w, gs_ld<READONLY>(cur + c), s0);
    }
    return s0 + s1;
}

// Local column indices of the gather cache (16-bit positions in a block's distinct-column list),
// stored per slice with two steps of a row in one 32-bit word: steps 2q and 2q + 1 of row r are
// the low and high halves of word q * GS_SELL_C + r of the slice, so one warp-wide load brings two
// steps' indices; an odd last step keeps the plain layout, entry (W - 1) * GS_SELL_C + r.
// slice_lidx must be 4-byte aligned (slices are whole multiples of GS_SELL_C entries).

// Calls f(j, index) for the steps j = 0 .. width - 1 of row r in order, one 32-bit load per pair.
template <class F>
__device__ __forceinline__ void gs_cached_lidx_each(const uint16_t* slice_lidx, int r, int width, F&& f)
{
    const uint32_t* lp2 = reinterpret_cast<const uint32_t*>(slice_lidx) + r;
    int j = 0;
    for (; j + 2 <= width; j += 2) {
        const unsigned pr = lp2[(j >> 1) * GS_SELL_C];
        f(j, pr & 0xffffu);
        f(j + 1, pr >> 16);
    }
    if (j < width) f(j, (unsigned)slice_lidx[j * GS_SELL_C + r]);
}

// Same loop with the neighbour values taken from a shared-memory cache through the paired 16-bit
// local indices above (the per-block gather cache of the persistent loop); identical summation
// order.  vp points at row r's first value.
__device__ __forceinline__ float gs_sell_dot_cached(const uint16_t* slice_lidx, int r, const float* vp, int width,
                                                    const float* xc)
{
    const uint32_t* lp2 = reinterpret_cast<const uint32_t*>(slice_lidx) + r;
    float s0 = 0.f, s1 = 0.f;
    int j = 0;
    for (; j + 8 <= width; j += 8) {
        float w[8], x[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const unsigned pr = lp2[((j >> 1) + q) * GS_SELL_C];
            w[2 * q] = vp[(j + 2 * q) * GS_SELL_C];
            w[2 * q + 1] = vp[(j + 2 * q + 1) * GS_SELL_C];
            x[2 * q] = xc[pr & 0xffffu];
            x[2 * q + 1] = xc[pr >> 16];
        }
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            s0 = fmaf(w[u], x[u], s0);
            s1 = fmaf(w[u + 1], x[u + 1], s1);
        }
    }
    for (; j + 2 <= width; j += 2) {
        const unsigned pr = lp2[(j >> 1) * GS_SELL_C];
        s0 = fmaf(vp[j * GS_SELL_C], xc[pr & 0xffffu], s0);
        s0 = fmaf(vp[(j + 1) * GS_SELL_C], xc[pr >> 16], s0);
    }
    if (j < width) s0 = fmaf(vp[j * GS_SELL_C], xc[slice_lidx[j * GS_SELL_C + r]], s0);
    return s0 + s1;
}

// Whole row by one thread, graph read from global memory.
template <bool READONLY>
__device__ __forceinline__ float gs_sell_row(const int* __restrict__ sptr, const int* __restrict__ scol,
                                             const float* __restrict__ sval, const float* cur,
                                             int64_t row)
{
    const int64_t sl = row / GS_SELL_C;
    const int beg = __ldg(sptr + sl);
    const int width = (__ldg(sptr + sl + 1) - beg) / GS_SELL_C;
    return gs_sell_dot<READONLY, true>(scol + beg + (row % GS_SELL_C), sval + beg + (row % GS_SELL_C),
                                       width, cur);
}

// Row split across T threads of a warp: lane = phase * (32 / T) + row-in-warp, phase t takes the
// entries j = t, t + T, ...; the partial sums are combined with xor shuffles over the phases, so
// every lane returns the full row sum.  All 32 lanes must call it (inactive rows pass width 0).
template <int T, bool READONLY>
__device__ __forceinline__ float gs_sell_row_split(const int* __restrict__ sptr,
                                                   const int* __restrict__ scol,
                                                   const float* __restrict__ sval, const float* cur,
                                                   int64_t row, bool active, int phase)
{
    float s0 = 0.f, s1 = 0.f;
    if (active) {
        const int64_t sl = row / GS_SELL_C;
        const int beg = __ldg(sptr + sl);
        const int width = (__ldg(sptr + sl + 1) - beg) / GS_SELL_C;
        const int* cp = scol + beg + (row % GS_SELL_C);
        const float* vp = sval + beg + (row % GS_SELL_C);
        int j = phase;
        for (; j + 3 * T < width; j += 4 * T) {
            int c[4];
            float w[4], x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                c[u] = __ldg(cp + (j + u * T) * GS_SELL_C);
                w[u] = __ldg(vp + (j + u * T) * GS_SELL_C);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) x[u] = gs_ld<READONLY>(cur + c[u]);
            s0 = fmaf(w[0], x[0], s0);
            s1 = fmaf(w[1], x[1], s1);
            s0 = fmaf(w[2], x[2], s0);
            s1 = fmaf(w[3], x[3], s1);
        }
        for (; j < width; j += T)
            s0 = fmaf(__ldg(vp + j * GS_SELL_C), gs_ld<READONLY>(cur + __ldg(cp + j * GS_SELL_C)), s0);
    }
    float s = s0 + s1;
#pragma unroll
    for (int off = 32 / T; off < 32; off <<= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return s;
}
