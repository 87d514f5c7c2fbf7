// C-ABI entry points of libgeosink (declared in include/geosink.h): argument checks, context
// and workspace management, and dispatch to the kernel drivers.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "gs_internal.cuh"

// ------------------------------------------------------------------------------ helpers
gs_status gs_fail(gs_ctx* ctx, gs_status st, const std::string& msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

gs_status gs_cuda_check(gs_ctx* ctx, cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return GS_OK;
    const gs_status st = (e == cudaErrorMemoryAllocation) ? GS_ERR_OOM : GS_ERR_CUDA;
    return gs_fail(ctx, st, std::string(what) + ": " + cudaGetErrorString(e));
}

gs_status gs_ws_ensure(gs_ctx* ctx, size_t bytes)
{
    if (bytes <= ctx->ws_bytes) return GS_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(ctx->stream, &cap);
    if (cap != cudaStreamCaptureStatusNone)
        return gs_fail(ctx, GS_ERR_UNSUPPORTED,
                       "workspace must grow while the stream is being captured; run the call once "
                       "before capture or call gs_reserve");
    gs_status st = gs_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "workspace grow (sync)");
    if (st != GS_OK) return st;
    gs_graph_cache_clear(ctx);  // captured graphs point into the old workspace
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    const size_t want = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = cudaMalloc(&ctx->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return gs_fail(ctx, GS_ERR_OOM, "workspace allocation failed");
    }
    ctx->ws_bytes = want;
    return GS_OK;
}

namespace {

bool bad_ptr(const void* p) { return p == nullptr; }

gs_status check_graph(gs_ctx* ctx, const gs_graph* g)
{
    if (!g) return gs_fail(ctx, GS_ERR_ARG, "null graph");
    if (g->device != ctx->device) return gs_fail(ctx, GS_ERR_ARG, "graph lives on another device");
    return GS_OK;
}

gs_status check_filter(gs_ctx* ctx, double t, int K)
{
    if (!(t > 0.0) || !isfinite(t)) return gs_fail(ctx, GS_ERR_ARG, "t must be finite and > 0");
    if (K < 1 || K > 10000) return gs_fail(ctx, GS_ERR_ARG, "K must be in [1, 10000]");
    return GS_OK;
}

gs_status enter(gs_ctx* ctx)
{
    if (!ctx) return GS_ERR_ARG;
    ctx->err.clear();
    return gs_cuda_check(ctx, cudaSetDevice(ctx->device), "cudaSetDevice");
}


}  // namespace

// ------------------------------------------------------------------------------ context
extern "C" gs_status gs_create(gs_ctx** out, int device, void* stream)
{
    if (!out) return GS_ERR_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return GS_ERR_ARG;
    }
    gs_ctx* ctx = new gs_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    gs_status st = gs_cuda_check(ctx, cudaSetDevice(device), "cudaSetDevice");
    if (st == GS_OK) st = gs_cuda_check(ctx, cudaMalloc(&ctx->flags, 4 * sizeof(int)), "flags");
    if (st == GS_OK) st = gs_cuda_check(ctx, cudaMemset(ctx->flags, 0, 4 * sizeof(int)), "flags");
    if (st == GS_OK)
        st = gs_cuda_check(ctx, cudaMalloc(&ctx->check_part, 2 * sizeof(double) * GS_CHECK_BLOCKS), "check scratch");
    if (st == GS_OK)
        st = gs_cuda_check(ctx, cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device),
                           "SM count");
    if (st != GS_OK) {
        gs_destroy(ctx);
        return st;
    }
    *out = ctx;
    return GS_OK;
}

extern "C" gs_status gs_destroy(gs_ctx* ctx)
{
    if (!ctx) return GS_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    gs_graph_cache_clear(ctx);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->flags) cudaFree(ctx->flags);
    if (ctx->check_part) cudaFree(ctx->check_part);
    delete ctx;
    return GS_OK;
}

extern "C" gs_status gs_set_stream(gs_ctx* ctx, void* stream)
{
    if (!ctx) return GS_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return GS_OK;
}

extern "C" const char* gs_last_error(const gs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" gs_status gs_sync(gs_ctx* ctx)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = gs_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronize")) != GS_OK)
        return st;
    int f = 0;
    if ((st = gs_cuda_check(ctx, cudaMemcpy(&f, ctx->flags, sizeof(int), cudaMemcpyDeviceToHost),
                            "reading status")) != GS_OK)
        return st;
    cudaMemset(ctx->flags, 0, sizeof(int));
    if (f & GS_FLAG_TIMEOUT) return gs_fail(ctx, GS_ERR_TIMEOUT, "a bounded in-kernel wait gave up");
    if (f & GS_FLAG_ARG)
        return gs_fail(ctx, GS_ERR_ARG,
                       "device argument check: a marginal with a negative or non-finite entry, marginals whose "
                       "masses sum(vol a), sum(vol b) differ by more than 1e-6 relative, or barycenter weights "
                       "that are negative or do not sum to 1 (GS_OPT_CHECK_ARGS 0 skips these checks)");
    if (f & GS_FLAG_NONFINITE)
        return gs_fail(ctx, GS_ERR_NONFINITE, "non-finite or non-positive value in a scaling or filter output");
    if (f & GS_FLAG_NOT_CONVERGED)
        return gs_fail(ctx, GS_ERR_NOT_CONVERGED, "marginal error never fell below eps");
    return GS_OK;
}

extern "C" gs_status gs_reserve(gs_ctx* ctx, int64_t bytes)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if (bytes < 0) return gs_fail(ctx, GS_ERR_ARG, "negative size");
    return gs_ws_ensure(ctx, (size_t)bytes);
}

extern "C" gs_status gs_set_option(gs_ctx* ctx, int option, int value)
{
    if (!ctx) return GS_ERR_ARG;
    if (option == GS_OPT_LOOP && (value >= 0 && value <= 2)) {
        ctx->loop_mode = value;
        return GS_OK;
    }
    if (option == GS_OPT_TILE_LANES && (value == 0 || value == 1 || value == 2 || value == 4 || value == 8 ||
                                        value == 16 || value == 32)) {
        ctx->lanes_override = value;
        return GS_OK;
    }
    if (option == GS_OPT_CHECK_ARGS && (value == 0 || value == 1)) {
        ctx->check_args = value;
        return GS_OK;
    }
    if (option == GS_OPT_BARRIER_SELFTEST && (value == 0 || value == 1)) {
        ctx->barrier_selftest = value;
        return GS_OK;
    }
    if (option == GS_OPT_PERSIST_SMEM_GRAPH && (value >= 0 && value <= 2)) {
        ctx->persist_smem_graph = value;
        return GS_OK;
    }
    if (option == GS_OPT_TAG_WORD && (value == 4 || value == 8)) {
        ctx->tag_word = value;
        return GS_OK;
    }
    if (option == GS_OPT_PERSIST_BLOCKS && (value == 1 || value == 2)) {
        ctx->persist_bps = value;
        return GS_OK;
    }
    if (option == GS_OPT_PERSIST_SYNC && (value >= 0 && value <= 4)) {
        ctx->persist_sync = value;
        return GS_OK;
    }
    if (option == GS_OPT_KNN_TENSOR && (value >= 0 && value <= 2)) {
        ctx->knn_tensor_cores = value;
        return GS_OK;
    }
    if (option == GS_OPT_B1_KERNEL && (value >= 0 && value <= 3 || (value >= 5 && value <= 7))) {
        ctx->b1_kernel = value;
        return GS_OK;
    }
    if (option == GS_OPT_NODE_ORDER && (value == 0 || value == 1)) {
        ctx->node_order = value;
        return GS_OK;
    }
    if (option == GS_OPT_LOOP_REGS && (value == 0 || value == 1)) {
        ctx->loop_regs = value;
        return GS_OK;
    }
    if (option == GS_OPT_BLK_KERNEL && (value == 0 || (value >= 2 && value <= 5) || value == 8 || value == 9)) {
        ctx->blk_kernel = value;
        return GS_OK;
    }
    return gs_fail(ctx, GS_ERR_ARG, "unknown option or value");
}

extern "C" gs_status gs_get_option(const gs_ctx* ctx, int option, int* value)
{
    if (!ctx || !value) return GS_ERR_ARG;
    switch (option) {
        case GS_OPT_LOOP:
            *value = ctx->loop_mode != 2 ? ctx->loop_mode : (ctx->tuned_loop == 2 ? 1 : 0);
            return GS_OK;
        case GS_OPT_BARRIER_SELFTEST: *value = ctx->barrier_selftest; return GS_OK;
        case GS_OPT_B1_KERNEL:
            *value = ctx->b1_kernel != GS_KERNEL_AUTO ? ctx->b1_kernel
                     : (ctx->tuned_b1 ? ctx->tuned_b1 : GS_KERNEL_SPLIT);
            return GS_OK;
        case GS_OPT_BLK_KERNEL: *value = ctx->blk_kernel; return GS_OK;
        case GS_OPT_KNN_TENSOR: *value = ctx->knn_tensor_cores; return GS_OK;
        case GS_OPT_PERSIST_SMEM_GRAPH: *value = ctx->persist_smem_graph; return GS_OK;
        case GS_OPT_PERSIST_SYNC: *value = gs_persist_sync_setting(ctx, nullptr); return GS_OK;
        case GS_OPT_PERSIST_BLOCKS: *value = ctx->persist_bps; return GS_OK;
        case GS_OPT_TAG_WORD: *value = ctx->tag_word; return GS_OK;
        case GS_OPT_CHECK_ARGS: *value = ctx->check_args; return GS_OK;
        case GS_OPT_TILE_LANES: *value = ctx->lanes_override; return GS_OK;
        case GS_OPT_NODE_ORDER: *value = ctx->node_order; return GS_OK;
        case GS_OPT_LOOP_REGS: *value = ctx->loop_regs; return GS_OK;
        default: return GS_ERR_ARG;
    }
}

extern "C" gs_status gs_launch_count(const gs_ctx* ctx, int64_t* count)
{
    if (!ctx || !count) return GS_ERR_ARG;
    *count = ctx->launches;
    return GS_OK;
}

// ------------------------------------------------------------------------ coefficients
extern "C" gs_status gs_cheb_coeffs(double t, int K, double* c)
{
    if (!c || !(t > 0.0) || !isfinite(t) || K < 0) return GS_ERR_ARG;
    gs_heat_coefficients(t, K, c);
    return GS_OK;
}

// ------------------------------------------------------------------------------ graphs
extern "C" gs_status gs_knn(gs_ctx* ctx, const float* X, int64_t n, int d, int k, int32_t* idx,
                            float* dist)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if (bad_ptr(X) || bad_ptr(idx)) return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    if (n < 2 || n >= ((int64_t)1 << 31) || d < 1 || d > 1024 || k < 1 || k > 24 || k >= n)
        return gs_fail(ctx, GS_ERR_ARG, "need 2 <= n < 2^31, 1 <= d <= 1024, 1 <= k <= 24, k < n");
    return gs_knn_launch(ctx, X, n, d, k, idx, dist, nullptr, nullptr);
}

extern "C" gs_status gs_build_graph(gs_ctx* ctx, const float* X, int64_t n, int d, int k,
                                    float sigma, gs_graph** out)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if (bad_ptr(X) || bad_ptr(out)) return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    *out = nullptr;
    if (n < 2 || n >= ((int64_t)1 << 31) || d < 1 || d > 1024 || k < 1 || k > 24 || k >= n)
        return gs_fail(ctx, GS_ERR_ARG, "need 2 <= n < 2^31, 1 <= d <= 1024, 1 <= k <= 24, k < n");
    if (!isfinite(sigma)) return gs_fail(ctx, GS_ERR_ARG, "sigma must be finite");
    return gs_build_graph_impl(ctx, X, n, d, k, sigma, out);
}

extern "C" gs_status gs_graph_from_csr(gs_ctx* ctx, int64_t n, const int64_t* rowptr,
                                       const int32_t* col, const float* w, gs_graph** out)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if (bad_ptr(rowptr) || bad_ptr(col) || bad_ptr(w) || bad_ptr(out))
        return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    *out = nullptr;
    if (n < 2 || n >= ((int64_t)1 << 31)) return gs_fail(ctx, GS_ERR_ARG, "need 2 <= n < 2^31");
    return gs_graph_import_csr(ctx, n, rowptr, col, w, out);
}

extern "C" gs_status gs_graph_info(const gs_graph* g, int64_t* n, int64_t* nnz, double* sigma)
{
    if (!g) return GS_ERR_ARG;
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (sigma) *sigma = g->sigma;
    return GS_OK;
}

extern "C" gs_status gs_graph_layout(const gs_graph* g, int64_t* out, int count)
{
    if (!g || !out || count < 0) return GS_ERR_ARG;
    int64_t sum_u = 0;
    for (int v : g->xc_ucnt_host) sum_u += v > 0 ? v : 0;
    const int64_t v[9] = {g->nslices, g->sell_nnz, g->xc_ok ? 1 : 0, g->xc_blocks, g->xc_rpb,
                          g->xc_max_e, g->xc_max_u, sum_u, g->xc_max_deps};
    for (int i = 0; i < count && i < 9; ++i) out[i] = v[i];
    return GS_OK;
}

extern "C" gs_status gs_graph_export_csr(gs_ctx* ctx, const gs_graph* g, int64_t* rowptr,
                                         int32_t* col, float* A, float* P)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = check_graph(ctx, g)) != GS_OK) return st;
    return gs_graph_export(ctx, g, rowptr, col, A, P);
}

extern "C" gs_status gs_autotune(gs_ctx* ctx, gs_graph* g, int B, int K, int* choice)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = check_graph(ctx, g)) != GS_OK) return st;
    if (K < 1 || K > 10000) return gs_fail(ctx, GS_ERR_ARG, "K must be in [1, 10000]");
    if (!gs_filter_supports(B, true))
        return gs_fail(ctx, GS_ERR_UNSUPPORTED, "B must be 1..256, or a multiple of 4 up to 1024");
    return gs_autotune_impl(ctx, g, B, K, choice);
}

extern "C" gs_status gs_autotune_choices(const gs_ctx* ctx, const gs_graph* g, int B, int K, int* out, int count)
{
    if (!ctx || !g || !out || count < 1 || B < 1) return GS_ERR_ARG;
    int v[6] = {0, 0, 0, 0, -1, 0};
    const TuneRecord* r = gs_tune_lookup(ctx, g, B, K);
    if (r) {
        v[0] = r->kernel;
        v[1] = r->lanes;
        v[3] = r->loop;
        v[4] = r->sync;
    }
    // what a call would run: lanes per row and columns per pass of the chosen mapping
    const FilterPlan pl = gs_filter_plan(ctx, g, B, true, K);
    if (B == 1) {
        v[1] = pl.kernel == GS_KERNEL_SPLIT || pl.kernel == GS_KERNEL_AUTO ? pl.split_t : v[1];
        v[2] = 1;
    } else {
        v[1] = pl.group;
        v[2] = pl.group * pl.vec;
    }
    v[5] = r ? 1 : 0;
    for (int i = 0; i < count && i < 6; ++i) out[i] = v[i];
    return GS_OK;
}

extern "C" gs_status gs_graph_destroy(gs_graph* g)
{
    if (!g) return GS_OK;
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    cudaFree(g->rowptr);
    cudaFree(g->col);
    cudaFree(g->pval);
    cudaFree(g->aval);
    cudaFree(g->deg);
    cudaFree(g->perm);
    cudaFree(g->heavy);
    cudaFree(g->iperm);
    cudaFree(g->prowptr);
    cudaFree(g->pcol);
    cudaFree(g->ppval);
    cudaFree(g->sptr);
    cudaFree(g->scol);
    cudaFree(g->sval);
    cudaFree(g->xc_ucol);
    cudaFree(g->xc_ucnt);
    cudaFree(g->xc_lidx);
    cudaFree(g->xc_deps);
    cudaFree(g->xc_ndeps);
    cudaFree(g->xc_rows);
    cudaFree(g->mrowptr);
    cudaFree(g->mcol);
    cudaFree(g->mval);
    delete g;
    return GS_OK;
}

// ------------------------------------------------------------------------- heat filter
// Y = sum_k c_k T_k(op) V on the operator of graph g (P, or a view with M in its place): V into the
// filter's node order, the fused orders, Y back.
static gs_status heat_apply_coeffs(gs_ctx* ctx, const gs_graph* g, const double* c, int K, const float* V,
                                   int B, float* Y)
{
    gs_status st;
    const size_t blk = sizeof(float) * (size_t)g->n * (size_t)B;
    Epilogue e;
    e.kind = EPI_STORE;
    if (!g->perm) {
        WsPlan plan;
        const size_t iA = plan.add(blk), iB = plan.add(blk);
        if ((st = gs_ws_ensure(ctx, plan.total)) != GS_OK) return st;
        e.out = Y;
        return gs_filter_enqueue(ctx, g, c, K, B, const_cast<float*>(V), false, ws_at<float>(ctx, plan, iA),
                                 ws_at<float>(ctx, plan, iB), Y, e, nullptr, nullptr);
    }
    // reordered graph: V into the filter's node order, apply, Y back
    WsPlan plan;
    const size_t iA = plan.add(blk), iV = plan.add(blk), iY = plan.add(blk);
    if ((st = gs_ws_ensure(ctx, plan.total)) != GS_OK) return st;
    float* Vp = ws_at<float>(ctx, plan, iV);
    float* Yp = ws_at<float>(ctx, plan, iY);
    gs_permute_rows(ctx, g->n, B, g->perm, V, Vp, true);
    e.out = Yp;
    if ((st = gs_filter_enqueue(ctx, g, c, K, B, Vp, true, ws_at<float>(ctx, plan, iA), nullptr, Yp, e, nullptr,
                                nullptr)) != GS_OK)
        return st;
    gs_permute_rows(ctx, g->n, B, g->perm, Yp, Y, false);
    return gs_cuda_check(ctx, cudaGetLastError(), "heat apply");
}

extern "C" gs_status gs_heat_apply(gs_ctx* ctx, const gs_graph* g, double t, int K, const float* V,
                                   int B, float* Y)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = check_graph(ctx, g)) != GS_OK || (st = check_filter(ctx, t, K)) != GS_OK) return st;
    if (bad_ptr(V) || bad_ptr(Y)) return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    if (V == Y) return gs_fail(ctx, GS_ERR_ARG, "V and Y must not alias");
    if (!gs_filter_supports(B, ((uintptr_t)V % 16) == 0))
        return gs_fail(ctx, GS_ERR_UNSUPPORTED,
                       "B must be 1..256, or a multiple of 4 up to 1024 with V 16-byte aligned");
    std::vector<double> c((size_t)K + 1);
    gs_heat_coefficients(t, K, c.data());
    return heat_apply_coeffs(ctx, g, c.data(), K, V, B, Y);
}

extern "C" gs_status gs_heat_apply_combinatorial(gs_ctx* ctx, gs_graph* g, double t, int K, const float* V,
                                                 int B, float* Y, double* lam)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = check_graph(ctx, g)) != GS_OK || (st = check_filter(ctx, t, K)) != GS_OK) return st;
    if (bad_ptr(V) || bad_ptr(Y)) return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    if (V == Y) return gs_fail(ctx, GS_ERR_ARG, "V and Y must not alias");
    if (!gs_filter_supports(B, ((uintptr_t)V % 16) == 0))
        return gs_fail(ctx, GS_ERR_UNSUPPORTED,
                       "B must be 1..256, or a multiple of 4 up to 1024 with V 16-byte aligned");
    if ((st = gs_graph_build_combinatorial(ctx, g)) != GS_OK) return st;
    if (lam) *lam = g->comb_lam;
    // exp(-t (D - A)) = exp(-s L') with L' = (2 / lam)(D - A) and s = t lam / 2
    const double s = t * g->comb_lam / 2.0;
    if (!(s > 0.0) || !isfinite(s)) return gs_fail(ctx, GS_ERR_ARG, "t * lam / 2 must be positive and finite");
    std::vector<double> c((size_t)K + 1);
    gs_heat_coefficients(s, K, c.data());
    gs_graph view;
    gs_combinatorial_view(g, &view);
    return heat_apply_coeffs(ctx, &view, c.data(), K, V, B, Y);
}

// ----------------------------------------------------------------------------- Sinkhorn
extern "C" gs_status gs_sinkhorn(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b,
                                 const float* vol, double t, int K, double eps, int iters,
                                 float* u, float* v, double* dist, int32_t* iters_done)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = check_graph(ctx, g)) != GS_OK || (st = check_filter(ctx, t, K)) != GS_OK) return st;
    if (bad_ptr(a) || bad_ptr(b) || bad_ptr(u) || bad_ptr(v))
        return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    if (iters < 1) return gs_fail(ctx, GS_ERR_ARG, "iters must be >= 1");
    if (!(eps == eps)) return gs_fail(ctx, GS_ERR_ARG, "eps is NaN");
    const gs_marginals mg{a, b, vol, g->n};
    if ((st = gs_check_marginals(ctx, mg)) != GS_OK) return st;
    return gs_sinkhorn_impl(ctx, g, a, b, vol, t, K, eps, iters, u, v, dist, iters_done);
}

extern "C" gs_status gs_distance(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b,
                                 const float* vol, double t, int K, double eps, int iters,
                                 double* dist)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = check_graph(ctx, g)) != GS_OK || (st = check_filter(ctx, t, K)) != GS_OK) return st;
    if (bad_ptr(a) || bad_ptr(b) || bad_ptr(dist)) return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    if (iters < 1) return gs_fail(ctx, GS_ERR_ARG, "iters must be >= 1");
    const gs_marginals mg{a, b, vol, g->n};
    if ((st = gs_check_marginals(ctx, mg)) != GS_OK) return st;
    // the scalings stay in the workspace
    return gs_sinkhorn_impl(ctx, g, a, b, vol, t, K, eps, iters, nullptr, nullptr, dist, nullptr);
}

// --------------------------------------------------------------------------- barycenter
extern "C" gs_status gs_barycenter(gs_ctx* ctx, const gs_graph* g, const float* M, int m,
                                   const double* alpha, const float* vol, double t, int K,
                                   int iters, float* mu, float* v_state)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = check_graph(ctx, g)) != GS_OK || (st = check_filter(ctx, t, K)) != GS_OK) return st;
    if (bad_ptr(M) || bad_ptr(alpha) || bad_ptr(mu)) return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    if (m < 1 || m > 1024) return gs_fail(ctx, GS_ERR_ARG, "m must be in [1, 1024]");
    if (!gs_filter_supports(m, true))
        return gs_fail(ctx, GS_ERR_UNSUPPORTED, "m must be 1..256, or a multiple of 4 up to 1024");
    if (iters < 1) return gs_fail(ctx, GS_ERR_ARG, "iters must be >= 1");
    if ((st = gs_check_weights(ctx, alpha, m)) != GS_OK) return st;
    return gs_barycenter_impl(ctx, g, M, m, alpha, vol, t, K, iters, mu, v_state);
}

extern "C" gs_status gs_heat_apply_implicit(gs_ctx* ctx, const gs_graph* g, double t, int K, const float* V,
                                            int B, float* Y, double tol, int iters)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = check_graph(ctx, g)) != GS_OK || (st = check_filter(ctx, t, K)) != GS_OK) return st;
    if (bad_ptr(V) || bad_ptr(Y)) return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    if (B < 1 || B > 256) return gs_fail(ctx, GS_ERR_ARG, "B must be in [1, 256]");
    if (K < 1 || iters < 1 || !(tol >= 0.0)) return gs_fail(ctx, GS_ERR_ARG, "need K >= 1, iters >= 1, tol >= 0");
    return gs_heat_apply_implicit_impl(ctx, g, t, K, V, B, Y, tol, iters);
}

extern "C" gs_status gs_sinkhorn_log(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b,
                                     const float* vol, double t, int K, double eps, int iters, double* log_u,
                                     double* log_v, double* dist, int32_t* iters_done)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = check_graph(ctx, g)) != GS_OK || (st = check_filter(ctx, t, K)) != GS_OK) return st;
    if (bad_ptr(a) || bad_ptr(b) || bad_ptr(log_u) || bad_ptr(log_v))
        return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    if (log_u == log_v) return gs_fail(ctx, GS_ERR_ARG, "log_u and log_v must be distinct buffers");
    if (iters < 1) return gs_fail(ctx, GS_ERR_ARG, "iters must be >= 1");
    if (!(eps == eps)) return gs_fail(ctx, GS_ERR_ARG, "eps is NaN");
    const gs_marginals mg{a, b, vol, g->n};
    if ((st = gs_check_marginals(ctx, mg)) != GS_OK) return st;
    return gs_sinkhorn_log_impl(ctx, g, a, b, vol, t, K, eps, iters, log_u, log_v, dist, iters_done);
}

// ---------------------------------------------------------------------- families of distributions
extern "C" gs_status gs_barycentric_distance(gs_ctx* ctx, const gs_graph* g, const float* MT, int mT,
                                             const double* alphaT, const float* MC, int mC,
                                             const double* alphaC, const float* vol, double t, int K,
                                             int bary_iters, int sink_iters, float* muT, float* muC,
                                             double* dist)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = check_graph(ctx, g)) != GS_OK || (st = check_filter(ctx, t, K)) != GS_OK) return st;
    if (bad_ptr(MT) || bad_ptr(alphaT) || bad_ptr(MC) || bad_ptr(alphaC) || bad_ptr(muT) || bad_ptr(muC) ||
        bad_ptr(dist))
        return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    if (muT == muC) return gs_fail(ctx, GS_ERR_ARG, "muT and muC must be distinct buffers");
    for (int m : {mT, mC}) {
        if (m < 1 || m > 1024) return gs_fail(ctx, GS_ERR_ARG, "family sizes must be in [1, 1024]");
        if (!gs_filter_supports(m, true))
            return gs_fail(ctx, GS_ERR_UNSUPPORTED, "family sizes must be 1..256, or multiples of 4 up to 1024");
    }
    if (bary_iters < 1 || sink_iters < 1) return gs_fail(ctx, GS_ERR_ARG, "iterations must be >= 1");
    if ((st = gs_check_weights(ctx, alphaT, mT)) != GS_OK || (st = gs_check_weights(ctx, alphaC, mC)) != GS_OK)
        return st;
    return gs_barycentric_distance_impl(ctx, g, MT, mT, alphaT, MC, mC, alphaC, vol, t, K, bary_iters, sink_iters,
                                        muT, muC, dist);
}

extern "C" gs_status gs_barycenter_effect(gs_ctx* ctx, const float* Y, int64_t n, int d, const float* muT,
                                          const float* muC, double* out)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if (bad_ptr(Y) || bad_ptr(muT) || bad_ptr(muC) || bad_ptr(out)) return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    if (n < 1 || d < 1 || d > 65535) return gs_fail(ctx, GS_ERR_ARG, "need n >= 1 and 1 <= d <= 65535");
    return gs_barycenter_effect_impl(ctx, Y, n, d, muT, muC, out);
}

// ------------------------------------------------------------------------------ adjoint
extern "C" gs_status gs_sinkhorn_grad(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b,
                                      const float* vol, double t, int K, int iters, int checkpoint,
                                      double* dist, float* grad_a, float* grad_b)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = check_graph(ctx, g)) != GS_OK || (st = check_filter(ctx, t, K)) != GS_OK) return st;
    if (bad_ptr(a) || bad_ptr(b) || bad_ptr(dist) || bad_ptr(grad_a) || bad_ptr(grad_b))
        return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    if (iters < 1 || checkpoint < 1) return gs_fail(ctx, GS_ERR_ARG, "iters and checkpoint must be >= 1");
    const gs_marginals mg{a, b, vol, g->n};
    if ((st = gs_check_marginals(ctx, mg)) != GS_OK) return st;
    return gs_sinkhorn_grad_impl(ctx, g, a, b, vol, t, K, iters, checkpoint, dist, grad_a, grad_b);
}

extern "C" gs_status gs_barycenter_grad(gs_ctx* ctx, const gs_graph* g, const float* M, int m,
                                        const double* alpha, const float* vol, double t, int K,
                                        int iters, int checkpoint, const float* mubar, float* mu,
                                        double* grad_alpha)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if ((st = check_graph(ctx, g)) != GS_OK || (st = check_filter(ctx, t, K)) != GS_OK) return st;
    if (bad_ptr(M) || bad_ptr(alpha) || bad_ptr(mubar) || bad_ptr(grad_alpha))
        return gs_fail(ctx, GS_ERR_ARG, "null pointer");
    if (m < 1 || m > 1024) return gs_fail(ctx, GS_ERR_ARG, "m must be in [1, 1024]");
    if (!gs_filter_supports(m, true))
        return gs_fail(ctx, GS_ERR_UNSUPPORTED, "m must be 1..256, or a multiple of 4 up to 1024");
    if (iters < 1 || checkpoint < 1) return gs_fail(ctx, GS_ERR_ARG, "iters and checkpoint must be >= 1");
    if ((st = gs_check_weights(ctx, alpha, m)) != GS_OK) return st;
    return gs_barycenter_grad_impl(ctx, g, M, m, alpha, vol, t, K, iters, checkpoint, mubar, mu, grad_alpha);
}

// ------------------------------------------------------------------------------ batched
extern "C" gs_status gs_sinkhorn_batched(gs_ctx* ctx, int nprob, const gs_graph* const* graphs,
                                         const float* const* a, const float* const* b,
                                         const double* t, const int* K, int iters, float* const* u,
                                         float* const* v, double* dist)
{
    gs_status st = enter(ctx);
    if (st != GS_OK) return st;
    if (nprob < 1 || !graphs || !a || !b || !t || !K || !u || !v)
        return gs_fail(ctx, GS_ERR_ARG, "null pointer or nprob < 1");
    if (iters < 1) return gs_fail(ctx, GS_ERR_ARG, "iters must be >= 1");
    for (int i = 0; i < nprob; ++i) {
        if ((st = check_graph(ctx, graphs[i])) != GS_OK) return st;
        if ((st = check_filter(ctx, t[i], K[i])) != GS_OK) return st;
        if (!a[i] || !b[i] || !u[i] || !v[i]) return gs_fail(ctx, GS_ERR_ARG, "null problem pointer");
    }
    return gs_sinkhorn_batched_impl(ctx, nprob, graphs, a, b, t, K, iters, u, v, dist);
}
