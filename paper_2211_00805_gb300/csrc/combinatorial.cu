// The combinatorial Laplacian L = D - A of Sec. 3.4 under the Chebyshev heat filter of Sec. 3.5.
//
// Sec. 3.5 expands exp(-tL) in Chebyshev polynomials of L - Id, which assumes the spectrum of L
// lies in [0, 2].  The spectrum of D - A lies in [0, lam] with lam = 2 max_i D_ii (Gershgorin:
// the disc of row i is centred at D_ii with radius D_ii), so L' = (2 / lam) L has its spectrum in
// [0, 2] and exp(-t L) = exp(-s L') with s = t lam / 2.  In the variable
//     M = Id - L' = Id - (2 / lam)(D - A),   M_ii = 1 - D_ii / max_j D_jj,   M_ij = A_ij / max_j D_jj,
// the expansion is sum_k c_k(s) T_k(M) with the same positive coefficients c_k as the normalised
// filter uses for P (T_k(L' - Id) = (-1)^k T_k(M)).  So the fused order kernels run unchanged on
// M; the only difference from P is the stored diagonal, which every kernel sums as one more entry.
//
// M is built once per graph, in the filter's locality order, on the first combinatorial apply.
#include <math.h>

#include "gs_internal.cuh"

namespace {

inline unsigned nblk(int64_t work, int per) { return (unsigned)((work + per - 1) / per); }

// largest degree (one block, FP64)
__global__ void __launch_bounds__(1024) degree_max(int64_t n, const double* __restrict__ deg, double* __restrict__ out)
{
    double m = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, deg[i]);
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
        *out = fmax(m, red[0]);
    }
}

// entries of row r of M (new order): the old row's entries plus the diagonal
__global__ void comb_count(int64_t n, const int* __restrict__ perm, const int* __restrict__ rowptr,
                           int* __restrict__ cnt)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int o = perm ? perm[r] : (int)r;
    cnt[r] = rowptr[o + 1] - rowptr[o] + 1;
}

// Row r of M in the new order, columns ascending: M_rj = A_oj / dmax at the renamed columns and
// M_rr = 1 - D_oo / dmax, inserted in order (rows are short; insertion sort).
__global__ void comb_fill(int64_t n, const int* __restrict__ perm, const int* __restrict__ iperm,
                          const int* __restrict__ rowptr, const int* __restrict__ col,
                          const float* __restrict__ aval, const double* __restrict__ deg,
                          const double* __restrict__ dmax_dev, const int64_t* __restrict__ off64,
                          int* __restrict__ mrowptr, int* __restrict__ mcol, float* __restrict__ mval)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n) return;
    mrowptr[r] = (int)off64[r];
    if (r == n) return;
    const double dmax = *dmax_dev;
    const int o = perm ? perm[r] : (int)r;
    const int b = (int)off64[r];
    const int len = rowptr[o + 1] - rowptr[o];
    mcol[b] = (int)r;
    mval[b] = (float)(1.0 - deg[o] / dmax);
    for (int i = 0; i < len; ++i) {
        const int e = rowptr[o] + i;
        const int c = iperm ? iperm[col[e]] : col[e];
        const float v = (float)((double)aval[e] / dmax);
        int j = b + i;  // entries b .. b + i hold the diagonal and the first i entries, sorted
        while (j >= b && mcol[j] > c) {
            mcol[j + 1] = mcol[j];
            mval[j + 1] = mval[j];
            --j;
        }
        mcol[j + 1] = c;
        mval[j + 1] = v;
    }
}

}  // namespace

gs_status gs_graph_build_combinatorial(gs_ctx* ctx, gs_graph* g)
{
    if (g->mrowptr) return GS_OK;
    const int64_t n = g->n, mnnz = g->nnz + g->n;
    if (mnnz >= ((int64_t)1 << 31)) return gs_fail(ctx, GS_ERR_UNSUPPORTED, "graph too large for int32 offsets");
    WsPlan plan;
    const size_t i_cnt = plan.add(sizeof(int) * n), i_off = plan.add(sizeof(int64_t) * (n + 1)),
                 i_sums = plan.add(sizeof(int64_t) * (n / 4096 + 2)), i_max = plan.add(sizeof(double));
    gs_status st = gs_ws_ensure(ctx, plan.total);
    if (st != GS_OK) return st;
    int* cnt = ws_at<int>(ctx, plan, i_cnt);
    int64_t* off = ws_at<int64_t>(ctx, plan, i_off);
    int64_t* sums = ws_at<int64_t>(ctx, plan, i_sums);
    double* dmax = ws_at<double>(ctx, plan, i_max);
    int *mrowptr = nullptr, *mcol = nullptr;
    float* mval = nullptr;
    cudaError_t e = cudaMalloc(&mrowptr, sizeof(int) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&mcol, sizeof(int) * mnnz);
    if (e == cudaSuccess) e = cudaMalloc(&mval, sizeof(float) * mnnz);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(mrowptr);
        cudaFree(mcol);
        cudaFree(mval);
        return gs_fail(ctx, GS_ERR_OOM, "combinatorial operator allocation failed");
    }
    cudaStream_t s = ctx->stream;
    degree_max<<<1, 1024, 0, s>>>(n, g->deg, dmax);
    comb_count<<<nblk(n, 256), 256, 0, s>>>(n, g->perm, g->rowptr, cnt);
    gs_exclusive_scan(s, cnt, n, off, sums);
    comb_fill<<<nblk(n + 1, 128), 128, 0, s>>>(n, g->perm, g->iperm, g->rowptr, g->col, g->aval, g->deg, dmax,
                                                off, mrowptr, mcol, mval);
    gs_count(ctx, 6);
    double hmax = 0.0;
    cudaMemcpyAsync(&hmax, dmax, sizeof(double), cudaMemcpyDeviceToHost, s);
    if ((st = gs_cuda_check(ctx, cudaStreamSynchronize(s), "combinatorial operator")) != GS_OK) {
        cudaFree(mrowptr);
        cudaFree(mcol);
        cudaFree(mval);
        return st;
    }
    if (!(hmax > 0.0) || !isfinite(hmax)) {
        cudaFree(mrowptr);
        cudaFree(mcol);
        cudaFree(mval);
        return gs_fail(ctx, GS_ERR_NONFINITE, "largest degree is not positive and finite");
    }
    g->mrowptr = mrowptr;
    g->mcol = mcol;
    g->mval = mval;
    g->comb_lam = 2.0 * hmax;
    return GS_OK;
}

// The same graph with M in place of P: CSR kernels only (no sliced ELL, no long-row list, no tuned
// choices), in the graph's locality order.
void gs_combinatorial_view(const gs_graph* g, gs_graph* v)
{
    v->device = g->device;
    v->n = g->n;
    v->nnz = g->nnz + g->n;
    v->mean_row = (float)((double)v->nnz / (double)g->n);
    v->rowptr = g->mrowptr;
    v->col = g->mcol;
    v->pval = g->mval;
    v->prowptr = g->mrowptr;
    v->pcol = g->mcol;
    v->ppval = g->mval;
    v->perm = g->perm;
    v->iperm = g->iperm;
}
