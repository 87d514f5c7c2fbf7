// Graph operator assembly (Sec. 3.4): degrees D_ii = sum_j A_ij and the normalised weights
// P_ij = A_ij / sqrt(D_ii D_jj) on a CSR pattern; import/export of caller CSR arrays.
#include <stdio.h>

#include "gs_internal.cuh"

namespace {

// One warp per row: FP64 degree of the row; flags rows with no positive weight.
__global__ void degree_kernel(int64_t n, const int* __restrict__ rowptr,
                              const float* __restrict__ aval, double* __restrict__ deg,
                              int* __restrict__ bad)
{
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32) s += (double)aval[e];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
        deg[row] = s;
        if (!(s > 0.0)) atomicOr(bad, 1);
    }
}

// One warp per row: P_ij = A_ij / sqrt(deg_i deg_j) computed in FP64, stored FP32.
__global__ void normalise_kernel(int64_t n, const int* __restrict__ rowptr,
                                 const int* __restrict__ col, const float* __restrict__ aval,
                                 const double* __restrict__ deg, float* __restrict__ pval)
{
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const double di = deg[row];
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32)
        pval[e] = (float)((double)aval[e] / sqrt(di * deg[col[e]]));
}

__global__ void rowptr64_to32(int64_t n1, const int64_t* __restrict__ in, int* __restrict__ out,
                              int64_t nnz, int* __restrict__ bad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n1) return;
    const int64_t v = in[i];
    if (v < 0 || v > nnz || (i > 0 && in[i - 1] > v)) atomicOr(bad, 1);
    out[i] = (int)v;
}

__global__ void check_cols(int64_t nnz, int64_t n, const int32_t* __restrict__ col,
                           int* __restrict__ bad)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nnz && (col[e] < 0 || col[e] >= n)) atomicOr(bad, 1);
}

__global__ void rowptr32_to64(int64_t n1, const int* __restrict__ in, int64_t* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) out[i] = in[i];
}

inline unsigned blocks_for(int64_t work, int per_block)
{
    return (unsigned)((work + per_block - 1) / per_block);
}

}  // namespace

gs_status gs_graph_alloc(gs_ctx* ctx, int64_t n, int64_t nnz, gs_graph** out)
{
    gs_graph* g = new gs_graph();
    g->device = ctx->device;
    g->n = n;
    g->nnz = nnz;
    g->mean_row = n > 0 ? (float)((double)nnz / (double)n) : 0.f;
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&g->rowptr, sizeof(int) * (size_t)(n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->col, sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->pval, sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->aval, sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->deg, sizeof(double) * (size_t)n);
    if (e != cudaSuccess) {
        gs_graph_destroy(g);
        cudaGetLastError();
        return gs_fail(ctx, GS_ERR_OOM, "graph allocation failed");
    }
    *out = g;
    return GS_OK;
}

gs_status gs_graph_finish(gs_ctx* ctx, gs_graph* g)
{
    int* bad = ctx->flags + 1;  // scratch word next to the status bits
    cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream);
    degree_kernel<<<blocks_for(g->n * 32, 256), 256, 0, ctx->stream>>>(g->n, g->rowptr, g->aval,
                                                                        g->deg, bad);
    normalise_kernel<<<blocks_for(g->n * 32, 256), 256, 0, ctx->stream>>>(
        g->n, g->rowptr, g->col, g->aval, g->deg, g->pval);
    gs_count(ctx, 2);
    int hbad = 0;
    cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    gs_status st = gs_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "graph normalisation");
    if (st != GS_OK) return st;
    if (hbad) return gs_fail(ctx, GS_ERR_ARG, "graph has a node without positive edge weight");
    return GS_OK;
}

gs_status gs_graph_import_csr(gs_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* col,
                              const float* w, gs_graph** out)
{
    int64_t nnz = 0;
    gs_status st = gs_cuda_check(
        ctx, cudaMemcpyAsync(&nnz, rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream),
        "reading rowptr[n]");
    if (st != GS_OK) return st;
    if ((st = gs_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "reading rowptr[n]")) != GS_OK)
        return st;
    if (nnz < n || nnz >= (int64_t)1 << 31)
        return gs_fail(ctx, GS_ERR_ARG, "rowptr[n] must be in [n, 2^31)");
    gs_graph* g = nullptr;
    if ((st = gs_graph_alloc(ctx, n, nnz, &g)) != GS_OK) return st;
    int* bad = ctx->flags + 1;
    cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream);
    rowptr64_to32<<<blocks_for(n + 1, 256), 256, 0, ctx->stream>>>(n + 1, rowptr, g->rowptr, nnz, bad);
    check_cols<<<blocks_for(nnz, 256), 256, 0, ctx->stream>>>(nnz, n, col, bad);
    gs_count(ctx, 2);
    cudaMemcpyAsync(g->col, col, sizeof(int) * (size_t)nnz, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(g->aval, w, sizeof(float) * (size_t)nnz, cudaMemcpyDeviceToDevice, ctx->stream);
    int hbad = 0;
    cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if ((st = gs_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "CSR import")) != GS_OK) {
        gs_graph_destroy(g);
        return st;
    }
    if (hbad) {
        gs_graph_destroy(g);
        return gs_fail(ctx, GS_ERR_ARG, "rowptr not monotone or column index out of range");
    }
    if ((st = gs_graph_finish(ctx, g)) != GS_OK || (st = gs_graph_reorder(ctx, g, nullptr, 0, nullptr)) != GS_OK) {
        gs_graph_destroy(g);
        return st;
    }
    *out = g;
    return GS_OK;
}

gs_status gs_graph_export(gs_ctx* ctx, const gs_graph* g, int64_t* rowptr, int32_t* col, float* A,
                          float* P)
{
    if (rowptr) {
        rowptr32_to64<<<blocks_for(g->n + 1, 256), 256, 0, ctx->stream>>>(g->n + 1, g->rowptr, rowptr);
        gs_count(ctx, 1);
    }
    if (col)
        cudaMemcpyAsync(col, g->col, sizeof(int) * (size_t)g->nnz, cudaMemcpyDeviceToDevice, ctx->stream);
    if (A)
        cudaMemcpyAsync(A, g->aval, sizeof(float) * (size_t)g->nnz, cudaMemcpyDeviceToDevice, ctx->stream);
    if (P)
        cudaMemcpyAsync(P, g->pval, sizeof(float) * (size_t)g->nnz, cudaMemcpyDeviceToDevice, ctx->stream);
    return gs_cuda_check(ctx, cudaGetLastError(), "graph export");
}
