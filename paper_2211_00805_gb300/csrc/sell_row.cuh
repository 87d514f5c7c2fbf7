// One row of P times a block column in the sliced-ELL layout (32-row slices stored column-major,
// padding entries have value 0), shared by the launch-per-order and the persistent kernels so both
// sum in exactly the same order.  READONLY: the gathered vector is constant for the kernel's
// lifetime and may use the read-only cache; otherwise ordinary coherent loads are used.
#pragma once

template <bool READONLY>
__device__ __forceinline__ float gs_ld(const float* p)
{
    if (READONLY) return __ldg(p);
    return *p;
}

template <bool READONLY>
__device__ __forceinline__ float gs_sell_row(const int* __restrict__ sptr, const int* __restrict__ scol,
                                             const float* __restrict__ sval, const float* cur,
                                             int64_t row)
{
    const int64_t sl = row >> 5;
    const int beg = __ldg(sptr + sl);
    const int width = (__ldg(sptr + sl + 1) - beg) >> 5;
    const int* cp = scol + beg + (row & 31);
    const float* vp = sval + beg + (row & 31);
    float s0 = 0.f, s1 = 0.f;
    int j = 0;
    for (; j + 8 <= width; j += 8) {
        int c[8];
        float w[8], x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            c[u] = __ldg(cp + (j + u) * 32);
            w[u] = __ldg(vp + (j + u) * 32);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = gs_ld<READONLY>(cur + c[u]);
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            s0 = fmaf(w[u], x[u], s0);
            s1 = fmaf(w[u + 1], x[u + 1], s1);
        }
    }
    for (; j < width; ++j) s0 = fmaf(__ldg(vp + j * 32), gs_ld<READONLY>(cur + __ldg(cp + j * 32)), s0);
    return s0 + s1;
}
