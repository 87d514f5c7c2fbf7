// Locality-preserving node order for the sparse products (a Cuthill-McKee sweep without the
// degree sort), computed on the GPU level by level, and the graph permuted into that order.
//
// The filter gathers neighbour rows of the previous block for every edge.  With nodes in the
// order the points arrived (random), every gather is a fresh cache line; after a breadth-first
// renumbering a node's neighbours sit in the previous, current or next level, and nodes placed
// next to each other share most of their neighbours, so consecutive rows processed by one thread
// block hit the same lines in L1.
//
// Deterministic parallel level construction: every unvisited neighbour w of the current level is
// owned by the lowest-positioned parent that reaches it (atomicMin); each parent counts the
// children it owns, an exclusive scan over the level turns counts into slots, and each parent
// writes its children in ascending node id.  A second sweep starts from the last node of a first
// sweep from node 0 (a pseudo-peripheral start).  Disconnected parts restart from the lowest
// unvisited node.
#include <vector>

#include "gs_internal.cuh"

namespace {

inline unsigned nblk(int64_t work, int per) { return (unsigned)((work + per - 1) / per); }

__global__ void order_init(int64_t n, int* __restrict__ iperm, int* __restrict__ owner)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        iperm[i] = -1;
        owner[i] = 0x7fffffff;
    }
}

__global__ void order_root(int* __restrict__ perm, int* __restrict__ iperm, int pos,
                           const int* __restrict__ root, int64_t n)
{
    const int r = *root;
    if (r < 0 || r >= n) return;  // cannot happen while unvisited nodes remain; never index past n
    perm[pos] = r;
    iperm[r] = pos;
}

__global__ void order_first_unvisited(int64_t n, const int* __restrict__ iperm, int* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && iperm[i] < 0) atomicMin(out, (int)i);
}

__global__ void order_claim(int lo, int hi, const int* __restrict__ perm,
                            const int* __restrict__ rowptr, const int* __restrict__ col,
                            const int* __restrict__ iperm, int* __restrict__ owner)
{
    const int p = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= hi) return;
    const int u = perm[p];
    for (int e = rowptr[u]; e < rowptr[u + 1]; ++e) {
        const int w = col[e];
        if (iperm[w] < 0) atomicMin(&owner[w], p);
    }
}

__global__ void order_count(int lo, int hi, const int* __restrict__ perm,
                            const int* __restrict__ rowptr, const int* __restrict__ col,
                            const int* __restrict__ iperm, const int* __restrict__ owner,
                            int* __restrict__ cnt)
{
    const int p = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= hi) return;
    const int u = perm[p];
    int c = 0;
    for (int e = rowptr[u]; e < rowptr[u + 1]; ++e) {
        const int w = col[e];
        c += (iperm[w] < 0 && owner[w] == p);
    }
    cnt[p - lo] = c;
}

__global__ void order_place(int lo, int hi, const int* perm_in, int* perm,
                            const int* __restrict__ rowptr, const int* __restrict__ col,
                            int* __restrict__ iperm, const int* __restrict__ owner,
                            const int64_t* __restrict__ offs)
{
    const int p = lo + blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= hi) return;
    const int u = perm_in[p];
    int j = hi + (int)offs[p - lo];
    for (int e = rowptr[u]; e < rowptr[u + 1]; ++e) {
        const int w = col[e];
        if (owner[w] == p && iperm[w] < 0) {
            perm[j] = w;
            iperm[w] = j;
            ++j;
        }
    }
}

// Permuted CSR: new row r holds old row perm[r] with columns renamed by iperm, sorted ascending.
__global__ void permute_count(int64_t n, const int* __restrict__ perm, const int* __restrict__ rowptr,
                              int* __restrict__ cnt)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int o = perm[r];
    cnt[r] = rowptr[o + 1] - rowptr[o];
}

__global__ void permute_fill(int64_t n, const int* __restrict__ perm, const int* __restrict__ iperm,
                             const int* __restrict__ rowptr, const int* __restrict__ col,
                             const float* __restrict__ pval, const int64_t* __restrict__ prow64,
                             int* __restrict__ pcol, float* __restrict__ ppval)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int o = perm[r];
    const int b = (int)prow64[r];
    const int len = rowptr[o + 1] - rowptr[o];
    for (int i = 0; i < len; ++i) {  // insertion sort by new column id (rows are short)
        const int c = iperm[col[rowptr[o] + i]];
        const float v = pval[rowptr[o] + i];
        int j = b + i - 1;
        while (j >= b && pcol[j] > c) {
            pcol[j + 1] = pcol[j];
            ppval[j + 1] = ppval[j];
            --j;
        }
        pcol[j + 1] = c;
        ppval[j + 1] = v;
    }
}

// Within each window of W consecutive positions, reorder nodes by decreasing degree (stable), so
// that sliced-ELL slices hold rows of similar length and their padding stays small.
__global__ void window_degree_sort(int64_t n, int W, const int* __restrict__ perm_in,
                                   const int* __restrict__ rowptr, int* __restrict__ perm_out)
{
    extern __shared__ int sdeg[];  // [W]
    const int64_t w0 = (int64_t)blockIdx.x * W;
    const int len = (int)((n - w0) < W ? (n - w0) : W);
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        if (i < len) {
            const int node = perm_in[w0 + i];
            sdeg[i] = rowptr[node + 1] - rowptr[node];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const int di = sdeg[i];
        int rank = 0;
        for (int j = 0; j < len; ++j) {
            const int dj = sdeg[j];
            rank += (dj > di) || (dj == di && j < i);
        }
        perm_out[w0 + rank] = perm_in[w0 + i];
    }
}

__global__ void invert_perm(int64_t n, const int* __restrict__ perm, int* __restrict__ iperm)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) iperm[perm[r]] = (int)r;
}

// Sliced ELL: slice width = longest row of the slice (in entries), stored width * GS_SELL_C.
__global__ void sell_width(int64_t n, int64_t nslices, const int* __restrict__ prowptr,
                           int* __restrict__ cnt)
{
    const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= nslices) return;
    int w = 0;
    for (int64_t r = sl * GS_SELL_C; r < (sl + 1) * GS_SELL_C && r < n; ++r) {
        const int len = prowptr[r + 1] - prowptr[r];
        w = len > w ? len : w;
    }
    cnt[sl] = w * GS_SELL_C;
}

// One thread per row of the padded slice range [0, 32 * nslices): rows past n (the tail of the last
// slice) get only padding entries, pointing at row n - 1 (in the same slice) with value 0, so that
// every stored column is a valid row index.
__global__ void sell_fill(int64_t n, int64_t nslices, const int* __restrict__ prowptr,
                          const int* __restrict__ pcol, const float* __restrict__ ppval,
                          const int64_t* __restrict__ sptr64, int* __restrict__ scol,
                          float* __restrict__ sval)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nslices * GS_SELL_C) return;
    const int64_t sl = r / GS_SELL_C, lane = r % GS_SELL_C;
    const int64_t base = sptr64[sl];
    const int width = (int)((sptr64[sl + 1] - base) / GS_SELL_C);
    const bool real = r < n;
    const int b = real ? prowptr[r] : 0, len = real ? prowptr[r + 1] - b : 0;
    for (int j = 0; j < width; ++j) {
        const int64_t o = base + (int64_t)j * GS_SELL_C + lane;
        if (j < len) {
            scol[o] = pcol[b + j];
            sval[o] = ppval[b + j];
        } else {
            scol[o] = (int)(real ? r : n - 1);
            sval[o] = 0.f;
        }
    }
}

__global__ void permute_rows_kernel(int64_t count, int B, const int* __restrict__ perm,
                                    const float* __restrict__ src, float* __restrict__ dst, int to)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t r = i / B, c = i - r * B;
    const int64_t o = (int64_t)perm[r] * B + c;
    if (to) dst[i] = src[o];
    else dst[o] = src[i];
}

__global__ void heavy_flag(int64_t n, const int* __restrict__ prowptr, int len, int* __restrict__ flag)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (prowptr[i + 1] - prowptr[i]) > len ? 1 : 0;
}

__global__ void heavy_place(int64_t n, const int* __restrict__ flag, const int64_t* __restrict__ pos,
                            int* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = (int)i;
}

__global__ void rowptr_narrow(int64_t n1, const int64_t* __restrict__ in, int* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) out[i] = (int)in[i];
}

}  // namespace

void gs_permute_rows(gs_ctx* ctx, int64_t n, int B, const int* perm, const float* src, float* dst,
                     bool to_filter_order)
{
    const int64_t count = n * (int64_t)B;
    permute_rows_kernel<<<nblk(count, 256), 256, 0, ctx->stream>>>(count, B, perm, src, dst,
                                                                    to_filter_order ? 1 : 0);
    gs_count(ctx, 1);
}

// One breadth-first sweep from `root` (device int), producing perm/iperm over all components.
static gs_status bfs_sweep(gs_ctx* ctx, const gs_graph* g, const int* root, int* perm, int* iperm,
                           int* owner, int* cnt, int64_t* offs, int64_t* sums, int* scratch_int,
                           int* levels_out)
{
    cudaStream_t s = ctx->stream;
    const int64_t n = g->n;
    order_init<<<nblk(n, 256), 256, 0, s>>>(n, iperm, owner);
    order_root<<<1, 1, 0, s>>>(perm, iperm, 0, root, n);
    gs_count(ctx, 2);
    int lo = 0, hi = 1, levels = 0;
    while (hi < n) {
        const int m = hi - lo;
        order_claim<<<nblk(m, 128), 128, 0, s>>>(lo, hi, perm, g->rowptr, g->col, iperm, owner);
        order_count<<<nblk(m, 128), 128, 0, s>>>(lo, hi, perm, g->rowptr, g->col, iperm, owner, cnt);
        gs_exclusive_scan(s, cnt, m, offs, sums);
        order_place<<<nblk(m, 128), 128, 0, s>>>(lo, hi, perm, perm, g->rowptr, g->col, iperm, owner, offs);
        gs_count(ctx, 6);
        int64_t total = 0;
        cudaMemcpyAsync(&total, offs + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        gs_status st = gs_cuda_check(ctx, cudaStreamSynchronize(s), "node ordering");
        if (st != GS_OK) return st;
        ++levels;
        if (total > 0) {
            lo = hi;
            hi += (int)total;
            continue;
        }
        // this component is exhausted: restart from the lowest unvisited node
        int init = 0x7fffffff;
        cudaMemcpyAsync(scratch_int, &init, sizeof(int), cudaMemcpyHostToDevice, s);
        order_first_unvisited<<<nblk(n, 256), 256, 0, s>>>(n, iperm, scratch_int);
        order_root<<<1, 1, 0, s>>>(perm, iperm, hi, scratch_int, n);
        gs_count(ctx, 2);
        lo = hi;
        hi += 1;
    }
    if (levels_out) *levels_out = levels;
    return gs_cuda_check(ctx, cudaGetLastError(), "node ordering");
}

gs_status gs_graph_reorder(gs_ctx* ctx, gs_graph* g)
{
    const int64_t n = g->n, nnz = g->nnz;
    WsPlan plan;
    const size_t i_owner = plan.add(sizeof(int) * n), i_cnt = plan.add(sizeof(int) * n),
                 i_offs = plan.add(sizeof(int64_t) * (n + 1)),
                 i_sums = plan.add(sizeof(int64_t) * (n / 4096 + 2)), i_int = plan.add(sizeof(int) * 4),
                 i_p64 = plan.add(sizeof(int64_t) * (n + 1)), i_hflag = plan.add(sizeof(int) * n),
                 i_h64 = plan.add(sizeof(int64_t) * (n + 1));
    gs_status st = gs_ws_ensure(ctx, plan.total);
    if (st != GS_OK) return st;
    int* owner = ws_at<int>(ctx, plan, i_owner);
    int* cnt = ws_at<int>(ctx, plan, i_cnt);
    int64_t* offs = ws_at<int64_t>(ctx, plan, i_offs);
    int64_t* sums = ws_at<int64_t>(ctx, plan, i_sums);
    int* sint = ws_at<int>(ctx, plan, i_int);
    int64_t* p64 = ws_at<int64_t>(ctx, plan, i_p64);
    int* hflag = ws_at<int>(ctx, plan, i_hflag);
    int64_t* h64 = ws_at<int64_t>(ctx, plan, i_h64);

    cudaError_t e = cudaMalloc(&g->perm, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&g->iperm, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&g->prowptr, sizeof(int) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->pcol, sizeof(int) * (nnz > 0 ? nnz : 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->ppval, sizeof(float) * (nnz > 0 ? nnz : 1));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return gs_fail(ctx, GS_ERR_OOM, "graph ordering allocation failed");
    }
    cudaStream_t s = ctx->stream;
    // sweep 1 from node 0; sweep 2 from the node it placed last
    const int zero = 0;
    cudaMemcpyAsync(sint + 1, &zero, sizeof(int), cudaMemcpyHostToDevice, s);
    int levels = 0;
    if ((st = bfs_sweep(ctx, g, sint + 1, g->perm, g->iperm, owner, cnt, offs, sums, sint, &levels)) != GS_OK)
        return st;
    cudaMemcpyAsync(sint + 2, g->perm + (n - 1), sizeof(int), cudaMemcpyDeviceToDevice, s);
    if ((st = bfs_sweep(ctx, g, sint + 2, g->perm, g->iperm, owner, cnt, offs, sums, sint, &levels)) != GS_OK)
        return st;
    g->levels = levels;
    // degree sort inside windows of 256 positions, then the inverse permutation
    {
        const int W = 256;
        cudaMemcpyAsync(owner, g->perm, sizeof(int) * n, cudaMemcpyDeviceToDevice, s);
        window_degree_sort<<<nblk(n, W), 256, sizeof(int) * W, s>>>(n, W, owner, g->rowptr, g->perm);
        invert_perm<<<nblk(n, 256), 256, 0, s>>>(n, g->perm, g->iperm);
        gs_count(ctx, 2);
    }
    // permuted CSR
    permute_count<<<nblk(n, 256), 256, 0, s>>>(n, g->perm, g->rowptr, cnt);
    gs_exclusive_scan(s, cnt, n, p64, sums);
    rowptr_narrow<<<nblk(n + 1, 256), 256, 0, s>>>(n + 1, p64, g->prowptr);
    permute_fill<<<nblk(n, 128), 128, 0, s>>>(n, g->perm, g->iperm, g->rowptr, g->col, g->pval, p64,
                                              g->pcol, g->ppval);
    gs_count(ctx, 6);
    // the long rows, ascending
    heavy_flag<<<nblk(n, 256), 256, 0, s>>>(n, g->prowptr, GS_HEAVY_ROW, hflag);
    gs_exclusive_scan(s, hflag, n, h64, sums);
    gs_count(ctx, 4);
    int64_t nheavy = 0;
    cudaMemcpyAsync(&nheavy, h64 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    // sliced ELL of the permuted operator
    const int64_t ns = (n + GS_SELL_C - 1) / GS_SELL_C;
    sell_width<<<nblk(ns, 256), 256, 0, s>>>(n, ns, g->prowptr, cnt);
    gs_exclusive_scan(s, cnt, ns, p64, sums);
    int64_t tot = 0;
    cudaMemcpyAsync(&tot, p64 + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if ((st = gs_cuda_check(ctx, cudaStreamSynchronize(s), "sliced ELL size")) != GS_OK) return st;
    if (nheavy > 0) {
        if (cudaMalloc(&g->heavy, sizeof(int) * nheavy) != cudaSuccess) {
            cudaGetLastError();
            return gs_fail(ctx, GS_ERR_OOM, "long-row list allocation failed");
        }
        heavy_place<<<nblk(n, 256), 256, 0, s>>>(n, hflag, h64, g->heavy);
        gs_count(ctx, 1);
        g->nheavy = nheavy;
    }
    if (tot >= ((int64_t)1 << 31)) return GS_OK;  // too large for int32 offsets: CSR kernels only
    e = cudaMalloc(&g->sptr, sizeof(int) * (ns + 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->scol, sizeof(int) * (tot > 0 ? tot : 1));
    if (e == cudaSuccess) e = cudaMalloc(&g->sval, sizeof(float) * (tot > 0 ? tot : 1));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return gs_fail(ctx, GS_ERR_OOM, "sliced ELL allocation failed");
    }
    g->nslices = ns;
    g->sell_nnz = tot;
    rowptr_narrow<<<nblk(ns + 1, 256), 256, 0, s>>>(ns + 1, p64, g->sptr);
    sell_fill<<<nblk(ns * GS_SELL_C, 256), 256, 0, s>>>(n, ns, g->prowptr, g->pcol, g->ppval, p64,
                                                          g->scol, g->sval);
    gs_count(ctx, 6);
    g->sptr_host.resize((size_t)ns + 1);
    cudaMemcpyAsync(g->sptr_host.data(), g->sptr, sizeof(int) * (ns + 1), cudaMemcpyDeviceToHost, s);
    if ((st = gs_cuda_check(ctx, cudaStreamSynchronize(s), "graph permutation")) != GS_OK) return st;
    const int blocks = gs_persist_cache_blocks(ctx);
    return gs_graph_build_xcache(ctx, g, blocks);
}
