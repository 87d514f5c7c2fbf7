// Shared-memory residency of one partition block's operator slice for the persistent loops: the
// block's sliced-ELL values, their 16-bit indices into the block's list of distinct columns, and
// that list, copied from global memory by bulk (TMA) copies completing on one mbarrier.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Bulk (TMA) copy of `bytes` from global to this CTA's shared memory, completing on `mbar`.
__device__ __forceinline__ void gs_bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* mbar)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const unsigned m = (unsigned)__cvta_generic_to_shared(mbar);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(d),
        "l"(src), "r"(bytes), "r"(m)
        : "memory");
}

// Rows [r0, r1) of block `blk` (whole 32-row slices): values sval[e0, e1) into sval_s, local
// indices xc_lidx[e0, e1) into lidx_s, and the block's xc_ucnt[blk] distinct columns (stored from
// xc_ucol + e0) into ucol_s.  Every thread must call it.  The wait is bounded by `budget` clock
// cycles; false = it ran out (GS_FLAG_TIMEOUT is then set in *flags by the caller's convention).
__device__ __forceinline__ bool gs_load_cache_tables(const int* sptr, const float* sval, const uint16_t* xc_lidx,
                                                     const int* xc_ucol, const int* xc_ucnt, int blk, int r0, int r1,
                                                     long long budget, float* sval_s, uint16_t* lidx_s,
                                                     int* ucol_s, int* e0_out, int* ucnt_out,
                                                     unsigned long long* mbar, bool* timed_out)
{
    const int s0 = r0 / 32;
    const int s1 = (r1 + 31) / 32;
    const int e0 = __ldg(sptr + s0);
    const int e1 = (r1 > r0) ? __ldg(sptr + s1) : e0;
    const int uc = (r1 > r0) ? __ldg(xc_ucnt + blk) : 0;
    *e0_out = e0;
    *ucnt_out = uc;
    *timed_out = false;
    const unsigned E = (unsigned)(e1 - e0);
    if (E == 0) return true;
    const unsigned bv = E * 4u, bl = E * 2u;               // E is a multiple of 32: both multiples of 16
    const unsigned bu = ((unsigned)uc * 4u + 15u) & ~15u;  // <= E * 4 (the list lives in [e0, e1))
    const unsigned m = (unsigned)__cvta_generic_to_shared(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(m) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(m), "r"(bv + bl + bu)
                     : "memory");
        gs_bulk_g2s(sval_s, sval + e0, bv, mbar);
        gs_bulk_g2s(lidx_s, xc_lidx + e0, bl, mbar);
        if (bu) gs_bulk_g2s(ucol_s, xc_ucol + e0, bu, mbar);
    }
    const long long t0 = clock64();
    unsigned done = 0;
    while (!done) {
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], 0;\n"
            " selp.u32 %0, 1, 0, P;\n}\n"
            : "=r"(done)
            : "r"(m)
            : "memory");
        if (!done && clock64() - t0 > budget) {
            *timed_out = true;
            return false;
        }
    }
    return true;
}
