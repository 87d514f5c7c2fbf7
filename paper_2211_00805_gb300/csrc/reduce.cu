// Distance reduction of Algorithm 1's return statement and Definition 4.1:
//     W^2 = 4t sum_i vol_i (a_i ln u_i + b_i ln v_i),   W = sqrt(W^2),
// accumulated in FP64 with a fixed two-pass tree (deterministic), 0 ln 0 := 0; and the device-side
// argument checks of the marginals and barycenter weights.
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

// ---------------------------------------------------------------------- argument checks
// Algorithm 1 transports a onto b: a plan with marginals vol * a and vol * b exists only when both
// are non-negative and carry the same mass, sum_i vol_i a_i = sum_i vol_i b_i (the vertex weights
// multiply both marginals of the plan).  The masses are summed in FP64 (one problem over many
// blocks, or many problems at one block each) and a negative or non-finite entry, or masses further
// apart than rtol times the larger one, raise GS_FLAG_ARG.
namespace {

constexpr int kCheckThreads = 1024;

__device__ void check_one(const gs_marginals& p, double rtol, int* flags)
{
    double ma = 0.0, mb = 0.0;
    int bad = 0;
    for (int64_t i = threadIdx.x; i < p.n; i += blockDim.x) {
        const float ai = p.a[i], bi = p.b[i];
        if (!(ai >= 0.f) || !(bi >= 0.f) || isinf(ai) || isinf(bi)) bad = 1;
        const double w = p.vol ? (double)p.vol[i] : 1.0;
        ma += w * (double)ai;
        mb += w * (double)bi;
    }
    __shared__ double ra[kCheckThreads / 32], rb[kCheckThreads / 32];
    for (int off = 16; off > 0; off >>= 1) {
        ma += __shfl_xor_sync(0xffffffffu, ma, off);
        mb += __shfl_xor_sync(0xffffffffu, mb, off);
    }
    bad = __syncthreads_or(bad);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        ra[w] = ma;
        rb[w] = mb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ma = mb = 0.0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) {
            ma += ra[j];
            mb += rb[j];
        }
        const double top = fmax(fabs(ma), fabs(mb));
        if (bad || !(fabs(ma - mb) <= rtol * top)) atomicOr(flags, GS_FLAG_ARG);
    }
}

// One problem over many blocks: each block sums a fixed stride of the entries, the last block to
// finish adds the blocks' partial masses in block order (so the sums do not depend on timing)
// and resets the arrival counter for the next call.
constexpr int kPartThreads = 256;
__global__ void __launch_bounds__(kPartThreads) check_marginals_part(const gs_marginals p, double rtol,
                                                                     double* __restrict__ part,
                                                                     unsigned* __restrict__ counter, int* flags)
{
    double ma = 0.0, mb = 0.0;
    int bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n; i += (int64_t)gridDim.x * blockDim.x) {
        const float ai = p.a[i], bi = p.b[i];
        if (!(ai >= 0.f) || !(bi >= 0.f) || isinf(ai) || isinf(bi)) bad = 1;
        const double w = p.vol ? (double)p.vol[i] : 1.0;
        ma += w * (double)ai;
        mb += w * (double)bi;
    }
    for (int off = 16; off > 0; off >>= 1) {
        ma += __shfl_xor_sync(0xffffffffu, ma, off);
        mb += __shfl_xor_sync(0xffffffffu, mb, off);
    }
    __shared__ double ra[kPartThreads / 32], rb[kPartThreads / 32];
    __shared__ bool s_last;
    bad = __syncthreads_or(bad);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        ra[w] = ma;
        rb[w] = mb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ma = mb = 0.0;
        for (int j = 0; j < kPartThreads / 32; ++j) {
            ma += ra[j];
            mb += rb[j];
        }
        part[2 * blockIdx.x] = ma;
        part[2 * blockIdx.x + 1] = mb;
        if (bad) atomicOr(flags, GS_FLAG_ARG);
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        double ta = 0.0, tb = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            ta += __ldcg(part + 2 * b);
            tb += __ldcg(part + 2 * b + 1);
        }
        const double top = fmax(fabs(ta), fabs(tb));
        if (!(fabs(ta - tb) <= rtol * top)) atomicOr(flags, GS_FLAG_ARG);
        *counter = 0u;
    }
}

__global__ void __launch_bounds__(kCheckThreads) check_marginals_many(const gs_marginals* __restrict__ ps,
                                                                      double rtol, int* flags)
{
    check_one(ps[blockIdx.x], rtol, flags);
}

// Barycenter weights (Sec. 3.3): alpha_i >= 0 and sum_i alpha_i = 1 within tol.
__global__ void __launch_bounds__(32) check_weights(const double* __restrict__ alpha, int m, double tol, int* flags)
{
    double s = 0.0;
    int bad = 0;
    for (int i = threadIdx.x; i < m; i += 32) {
        const double ai = alpha[i];
        if (!(ai >= 0.0) || isinf(ai)) bad = 1;
        s += ai;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    bad = __any_sync(0xffffffffu, bad);
    if (threadIdx.x == 0 && (bad || !(fabs(s - 1.0) <= tol))) atomicOr(flags, GS_FLAG_ARG);
}

}  // namespace

gs_status gs_check_marginals(gs_ctx* ctx, const gs_marginals& m)
{
    if (!ctx->check_args) return GS_OK;
    int64_t blocks = (m.n + kPartThreads - 1) / kPartThreads;
    if (blocks > GS_CHECK_BLOCKS) blocks = GS_CHECK_BLOCKS;
    if (blocks < 1) blocks = 1;
    check_marginals_part<<<(unsigned)blocks, kPartThreads, 0, ctx->stream>>>(
        m, GS_MASS_RTOL, ctx->check_part, reinterpret_cast<unsigned*>(ctx->flags + 2), ctx->flags);
    gs_count(ctx, 1);
    return gs_cuda_check(ctx, cudaGetLastError(), "marginal check");
}

gs_status gs_check_marginals_dev(gs_ctx* ctx, const gs_marginals* probs_dev, int count)
{
    if (!ctx->check_args || count < 1) return GS_OK;
    check_marginals_many<<<(unsigned)count, kCheckThreads, 0, ctx->stream>>>(probs_dev, GS_MASS_RTOL, ctx->flags);
    gs_count(ctx, 1);
    return gs_cuda_check(ctx, cudaGetLastError(), "marginal check");
}

gs_status gs_check_weights(gs_ctx* ctx, const double* alpha, int m)
{
    if (!ctx->check_args) return GS_OK;
    check_weights<<<1, 32, 0, ctx->stream>>>(alpha, m, GS_WEIGHT_TOL, ctx->flags);
    gs_count(ctx, 1);
    return gs_cuda_check(ctx, cudaGetLastError(), "weight check");
}
