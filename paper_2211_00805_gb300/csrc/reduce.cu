// Distance reduction of Algorithm 1's return statement and Definition 4.1:
//     W^2 = 4t sum_i vol_i (a_i ln u_i + b_i ln v_i),   W = sqrt(W^2),
// accumulated in FP64 with a fixed two-pass tree (deterministic), 0 ln 0 := 0.
#include <math.h>

#include "gs_internal.cuh"

namespace {

constexpr int kReduceBlocks = 1024;
constexpr int kThreads = 256;

__device__ __forceinline__ double term(float mass, float s, int* flags)
{
    if (mass == 0.f) return 0.0;
    if (!(s > 0.f) || isinf(s)) {
        atomicOr(flags, GS_FLAG_NONFINITE);
        return 0.0;
    }
    return (double)mass * log((double)s);
}

__global__ void __launch_bounds__(kThreads) dist_partial(int64_t n, const float* __restrict__ a,
                                                         const float* __restrict__ b,
                                                         const float* __restrict__ vol,
                                                         const float* __restrict__ u,
                                                         const float* __restrict__ v,
                                                         double* __restrict__ partials, int* flags)
{
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double w = vol ? (double)vol[i] : 1.0;
        s += w * (term(a[i], u[i], flags) + term(b[i], v[i], flags));
    }
    __shared__ double red[kThreads];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = kThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kReduceBlocks) dist_final(int nparts, const double* __restrict__ partials,
                                                            double scale, double* __restrict__ dist,
                                                            int* flags)
{
    __shared__ double red[kReduceBlocks];
    red[threadIdx.x] = threadIdx.x < nparts ? partials[threadIdx.x] : 0.0;
    __syncthreads();
    for (int h = kReduceBlocks / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double w2 = scale * red[0];
        dist[0] = w2;
        dist[1] = w2 >= 0.0 ? sqrt(w2) : nan("");
        if (!isfinite(w2)) atomicOr(flags, GS_FLAG_NONFINITE);
    }
}

}  // namespace

int gs_reduce_blocks() { return kReduceBlocks; }

gs_status gs_distance_enqueue(gs_ctx* ctx, int64_t n, const float* a, const float* b,
                              const float* vol, const float* u, const float* v, double t,
                              double* partials, double* dist)
{
    int64_t nb = (n + kThreads - 1) / kThreads;
    if (nb > kReduceBlocks) nb = kReduceBlocks;
    dist_partial<<<(unsigned)nb, kThreads, 0, ctx->stream>>>(n, a, b, vol, u, v, partials, ctx->flags);
    dist_final<<<1, kReduceBlocks, 0, ctx->stream>>>((int)nb, partials, 4.0 * t, dist, ctx->flags);
    gs_count(ctx, 2);
    return gs_cuda_check(ctx, cudaGetLastError(), "distance reduction");
}
