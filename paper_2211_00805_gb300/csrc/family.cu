// Families of distributions (Sec. 4): the barycentric distance of Definition 4.3, the Geodesic
// Sinkhorn distance between the barycenters of two families, and the expected barycenter effect
// of Definition 4.4, the difference of the features' expectations under the two barycenters.
// Both are compositions of the barycenter (cheb.cu) and the Sinkhorn loop; the kernels here are
// the two small reductions that join them: a barycenter divided by its mass (Algorithm 1 needs
// marginals of equal mass, and the definition compares distributions), and the weighted feature
// means.  All sums are FP64 in a fixed order, so the results repeat bit for bit.
#include "gs_internal.cuh"

namespace {

constexpr int kNormThreads = 1024;
constexpr int kEffectThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();  // red may still be read by the previous call
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];  // every thread, same order
    return t;
}

// Block 0 divides a by its mass, block 1 divides b by its mass.  A mass that is not positive and
// finite is reported (GS_FLAG_NONFINITE) and leaves the vector as it is.
__global__ void __launch_bounds__(kNormThreads) normalise_two(float* __restrict__ a, float* __restrict__ b,
                                                              int64_t n, int* __restrict__ flags)
{
    __shared__ double red[kNormThreads / 32];
    float* x = blockIdx.x == 0 ? a : b;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)x[i];
    const double m = block_sum(s, red);
    if (!(m > 0.0) || isinf(m)) {
        if (threadIdx.x == 0) atomicOr(flags, GS_FLAG_NONFINITE);
        return;
    }
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] = (float)((double)x[i] / m);
}

// out[j] = sum_i muT_i Y_ij / sum_i muT_i - sum_i muC_i Y_ij / sum_i muC_i, one block per feature.
__global__ void __launch_bounds__(kEffectThreads) barycenter_effect_kernel(const float* __restrict__ Y, int64_t n, int d,
                                                                           const float* __restrict__ muT,
                                                                           const float* __restrict__ muC,
                                                                           double* __restrict__ out, int* __restrict__ flags)
{
    __shared__ double red[kEffectThreads / 32];
    const int j = blockIdx.x;
    double sT = 0.0, mT = 0.0, sC = 0.0, mC = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double y = (double)Y[i * d + j], wt = (double)muT[i], wc = (double)muC[i];
        sT += wt * y;
        mT += wt;
        sC += wc * y;
        mC += wc;
    }
    sT = block_sum(sT, red);
    mT = block_sum(mT, red);
    sC = block_sum(sC, red);
    mC = block_sum(mC, red);
    if (threadIdx.x == 0) {
        if (!(mT > 0.0) || !(mC > 0.0) || isinf(mT) || isinf(mC)) atomicOr(flags, GS_FLAG_NONFINITE);
        out[j] = sT / mT - sC / mC;
    }
}

}  // namespace

gs_status gs_barycentric_distance_impl(gs_ctx* ctx, const gs_graph* g, const float* MT, int mT,
                                       const double* alphaT, const float* MC, int mC, const double* alphaC,
                                       const float* vol, double t, int K, int bary_iters, int sink_iters,
                                       float* muT, float* muC, double* dist)
{
    gs_status st = gs_barycenter_impl(ctx, g, MT, mT, alphaT, vol, t, K, bary_iters, muT, nullptr);
    if (st != GS_OK) return st;
    if ((st = gs_barycenter_impl(ctx, g, MC, mC, alphaC, vol, t, K, bary_iters, muC, nullptr)) != GS_OK) return st;
    normalise_two<<<2, kNormThreads, 0, ctx->stream>>>(muT, muC, g->n, ctx->flags);
    gs_count(ctx, 1);
    return gs_sinkhorn_impl(ctx, g, muT, muC, vol, t, K, 0.0, sink_iters, nullptr, nullptr, dist, nullptr);
}

gs_status gs_barycenter_effect_impl(gs_ctx* ctx, const float* Y, int64_t n, int d, const float* muT,
                                    const float* muC, double* out)
{
    barycenter_effect_kernel<<<d, kEffectThreads, 0, ctx->stream>>>(Y, n, d, muT, muC, out, ctx->flags);
    gs_count(ctx, 1);
    return gs_cuda_check(ctx, cudaGetLastError(), "barycenter effect");
}
