// Internal declarations of libgeosink: context and graph structures, status helpers, and the
// launch wrappers each .cu file provides to the C-ABI layer (api.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/geosink.h"

// Rows per sliced-ELL slice (a slice's entries for one column index j are GS_SELL_C consecutive
// words, one 32-byte sector).
constexpr int GS_SELL_C = 32;

// Rows with more than this many entries are summed by a whole warp (its lane groups splitting the
// entry list) in the B > 1 filter, so that hub rows of high-dimensional kNN graphs do not set the
// critical path of a launch.
constexpr int GS_HEAVY_ROW = 32;

// Kernel variants of the Chebyshev order (selected per context; the autotuner picks them).
enum : int {
    GS_KERNEL_AUTO = 0,
    GS_KERNEL_SELL = 1,     // B == 1: sliced ELL, thread per row
    GS_KERNEL_VECTOR = 2,   // B == 1: CSR, lanes split the row | B > 1: lane group, direct gathers
    GS_KERNEL_ASYNC = 3,    // chunked CSR ranges with cp.async gathers into shared memory
    GS_KERNEL_STAGED = 4,   // B > 1: neighbour list staged in shared memory, 8-deep gathers
    GS_KERNEL_RANGED = 5,   // each block walks a contiguous row range (sliced ELL / lane groups)
    GS_KERNEL_SPLIT = 6,    // B == 1: sliced ELL with each row split across GS_SPLIT_T threads
    GS_KERNEL_SM_RANGE = 7, // B == 1: one 1024-thread block per SM, one contiguous row range each
    GS_KERNEL_GROUP_WARP = 8,  // B in {32, 64, 128}: one warp per row, indices loaded by the lanes
    GS_KERNEL_GROUP_VEC4 = 9,  // B in {32, 64, 128}: B / 4 float4 lanes per row, indices loaded by the lanes
};
constexpr int GS_SPLIT_T = 4;

// Bits the kernels OR into the context's device status word; gs_sync turns them into a status.
enum : int {
    GS_FLAG_NONFINITE = 1,
    GS_FLAG_NOT_CONVERGED = 2,
    GS_FLAG_TIMEOUT = 4,
    GS_FLAG_ARG = 8,        // an input failed a device-side argument check (raised as GS_ERR_ARG)
};

// A captured CUDA graph of one or more Sinkhorn iterations, replayed instead of re-launching
// the 2K kernels of every iteration from the host.
struct GraphCacheEntry {
    std::vector<uintptr_t> key;
    cudaGraphExec_t exec1 = nullptr;   // one iteration
    cudaGraphExec_t execR = nullptr;   // R iterations
    int R = 0;
};

// One gs_autotune decision, kept by the context for every graph of the same size (rebuilt graphs
// of a workload find it too).
struct TuneRecord {
    int64_t n = 0, nnz = 0;
    int B = 0, K = 0;
    int kernel = 0;    // GS_KERNEL_* order variant
    int lanes = 0;     // B > 1: lanes per row (columns per pass = lanes x floats per lane);
                       // B == 1: threads per row of the row-split kernel; 0 = the kernel's default
    int loop = 0;      // B == 1: 1 persistent loop, 2 CUDA-graph replay (0 not timed)
    int sync = -1;     // B == 1: the persistent loop's block synchronisation (-1 not timed)
};

// A batched Sinkhorn call's device tables and the CUDA graph of its launches (batched.cu).
struct BatchCacheEntry {
    std::vector<uintptr_t> key;
    void* tables = nullptr;          // device: descriptors, coefficients, check descriptors, order
    size_t off_probs = 0, off_checks = 0, off_order = 0;
    int clusters = 1;
    cudaGraphExec_t exec = nullptr;
    int nodes = 0;                   // kernels in the graph (for the launch counter)
};

struct gs_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;    // private stream used only to capture graphs
    int* flags = nullptr;          // device: [0] status bits (GS_FLAG_*), [1] scratch word, [2] the
                                   // argument check's arrival counter (zero between calls)
    double* check_part = nullptr;  // device: the argument check's partial masses [2 x GS_CHECK_BLOCKS]
    void* ws = nullptr;            // device workspace
    size_t ws_bytes = 0;
    int num_sms = 0;
    bool capturing = false;        // inside an internal capture: launches are not counted
    int loop_mode = 2;             // fixed-count Sinkhorn: 0 persistent, 1 CUDA-graph replay, 2 auto
    int barrier_selftest = 0;      // next persistent launch waits for an arrival that never comes
    int b1_kernel = 0;             // GS_KERNEL_* for one column
    int blk_kernel = 0;            // GS_KERNEL_* for several columns
    int knn_tensor_cores = 2;      // kNN screen: 2 tcgen05 (d <= 62), 1 warp-level MMA (d >= 16),
                                   // 0 CUDA cores; each falls back to the next one it can use
    int tuned_b1 = 0;              // last gs_autotune result for one column (used by untuned graphs)
    int tuned_loop = 0;            // last gs_autotune loop choice (1 persistent, 2 graph replay)
    int persist_smem_graph = 2;    // persistent loop: 0 graph from global memory, 1 graph slices in
                                   // shared memory, 2 slices plus the per-block gather cache
    int persist_sync = 3;          // persistent loop with the gather cache: 2 tagged values re-read
                                   // in groups, 4 one at a time, 1 neighbour flags, 0 grid barrier,
                                   // 3 the autotuned choice
    int tuned_sync = -1;           // last gs_autotune choice of the above (0, 1, 2, 4), -1 none
    int tag_word = 4;              // tagged-value exchange word: 4 (value with a parity bit) or 8 (exact)
    int persist_bps = 1;           // gather-cache partition of graphs built from now on: blocks per
                                   // SM (1: 1024 threads each, 2: 512 threads each)
    int check_args = 1;            // device-side checks of marginals and barycenter weights (1 on)
    int node_order = 1;            // inside each bisection part: 1 degree classes + reader, 0 degree
    int loop_regs = 1;             // persistent tagged loop: rows' first steps in registers where blocks fit
    int lanes_override = 0;        // autotuner trials: lanes per row (B > 1) / threads per row (B == 1)
    std::vector<TuneRecord> tune_log;  // gs_autotune decisions by (n, nnz, B, K)
    int64_t launches = 0;          // kernels enqueued (graph replays count their nodes)
    std::vector<GraphCacheEntry> gcache;
    std::vector<BatchCacheEntry> bcache;
    std::string err;
};

static inline void gs_count(gs_ctx* ctx, int64_t k)
{
    if (!ctx->capturing) ctx->launches += k;
}
void gs_graph_cache_clear(gs_ctx* ctx);
void gs_batch_cache_clear(gs_ctx* ctx);

struct gs_graph {
    int device = 0;
    int64_t n = 0;
    int64_t nnz = 0;
    double sigma = 0.0;
    int* rowptr = nullptr;         // [n+1] int32 offsets into col / pval / aval
    int* col = nullptr;            // [nnz] neighbour index, ascending per row
    float* pval = nullptr;         // [nnz] P_ij = A_ij / sqrt(deg_i deg_j)
    float* aval = nullptr;         // [nnz] A_ij
    double* deg = nullptr;         // [n] degrees
    float mean_row = 0.f;          // nnz / n, steers the row-split width of the B = 1 kernel
    // locality order used by the filter (breadth-first renumbering, order.cu); null = none
    int* perm = nullptr;           // [n] new position -> node id
    int* iperm = nullptr;          // [n] node id -> new position
    int* prowptr = nullptr;        // [n+1] CSR of P in the new order
    int* pcol = nullptr;
    float* ppval = nullptr;
    int levels = 0;                // breadth-first levels of the ordering sweep
    int* heavy = nullptr;          // [nheavy] rows (new order) with more than GS_HEAVY_ROW entries,
    int64_t nheavy = 0;            // ascending; the B > 1 filter splits each across a warp
    // sliced ELL copy of the reordered P for the one-column kernels: GS_SELL_C-row slices, each
    // stored column-major and padded to its longest row (padding: column = the row itself, value 0)
    int* sptr = nullptr;           // [nslices + 1] offsets into scol / sval
    int* scol = nullptr;
    float* sval = nullptr;
    int64_t nslices = 0;
    int64_t sell_nnz = 0;          // stored entries including padding
    // autotuner choices (GS_KERNEL_*, 0 = none): one column, and several columns for B = tuned_blk_B
    int tuned_b1 = 0;
    int tuned_blk = 0;
    int tuned_blk_B = 0;
    int tuned_loop = 0;            // Sinkhorn loop: 0 not tuned, 1 persistent, 2 CUDA-graph replay
    int tuned_sync = -1;           // persistent loop's block synchronisation (0, 1, 2, 4), -1 not tuned
    int tuned_lanes = 0;           // lanes per row of tuned_blk (0: the kernel's default)
    int tuned_split = 0;           // threads per row of the one-column row-split kernel (0: default)
    std::vector<int> sptr_host;    // host copy of the slice offsets (sizes the persistent kernel's
                                   // shared-memory graph slices)
    // per-block gather cache of the persistent loop (xcache.cu): for the partition into xc_blocks
    // blocks of xc_rpb rows, block b's distinct columns (sorted) at xc_ucol[entry offset of b],
    // their count xc_ucnt[b], and every entry's 16-bit index into that list
    bool xc_ok = false;
    int xc_blocks = 0, xc_rpb = 0, xc_max_e = 0, xc_max_u = 0;  // xc_rpb: rows of the largest block
    int* xc_rows = nullptr;              // [xc_blocks + 1] block b owns rows [xc_rows[b], xc_rows[b+1])
    std::vector<int> xc_rows_host;
    int* xc_ucol = nullptr;
    int* xc_ucnt = nullptr;
    uint16_t* xc_lidx = nullptr;
    int* xc_deps = nullptr;   // [xc_blocks][xc_blocks]: block b's first xc_ndeps[b] entries are the
    int* xc_ndeps = nullptr;  // other blocks owning one of its distinct columns
    int xc_max_deps = 0;
    std::vector<int> xc_ucnt_host;
    // the combinatorial operator M = I - (2 / lam)(D - A), lam = 2 max_i D_ii, in the locality order
    // with its diagonal (combinatorial.cu); built on the first combinatorial apply
    int* mrowptr = nullptr;
    int* mcol = nullptr;
    float* mval = nullptr;
    double comb_lam = 0.0;
};

// The CSR the filter kernels read: the reordered one when present.
struct FilterCsr {
    const int* rowptr;
    const int* col;
    const float* pval;
};
static inline FilterCsr gs_filter_csr(const gs_graph* g)
{
    if (g->prowptr) return FilterCsr{g->prowptr, g->pcol, g->ppval};
    return FilterCsr{g->rowptr, g->col, g->pval};
}

// ------------------------------------------------------------------------------ helpers
gs_status gs_fail(gs_ctx* ctx, gs_status st, const std::string& msg);
gs_status gs_cuda_check(gs_ctx* ctx, cudaError_t e, const char* what);

// Carves aligned sub-buffers out of the context workspace, growing it if needed.
struct WsPlan {
    std::vector<size_t> offs;
    size_t total = 0;
    size_t add(size_t bytes) {
        total = (total + 255) & ~size_t(255);
        offs.push_back(total);
        total += bytes;
        return offs.size() - 1;
    }
};
gs_status gs_ws_ensure(gs_ctx* ctx, size_t bytes);
template <class T>
static inline T* ws_at(gs_ctx* ctx, const WsPlan& p, size_t i) {
    return reinterpret_cast<T*>(static_cast<char*>(ctx->ws) + p.offs[i]);
}

// Host FP64 Chebyshev coefficients c[0..K] of exp(-tL) in the variable P (coeffs.cu).
void gs_heat_coefficients(double t, int K, double* c);

// ------------------------------------------------------------------- graph.cu
gs_status gs_graph_alloc(gs_ctx* ctx, int64_t n, int64_t nnz, gs_graph** out);
// Given rowptr/col/aval filled on the device, compute degrees and P (stream-ordered).
gs_status gs_graph_finish(gs_ctx* ctx, gs_graph* g);
gs_status gs_graph_import_csr(gs_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* col,
                              const float* w, gs_graph** out);
gs_status gs_graph_export(gs_ctx* ctx, const gs_graph* g, int64_t* rowptr, int32_t* col, float* A,
                          float* P);

// --------------------------------------------------------------------- order.cu
// Node order of the filter: recursive coordinate bisection of the points X [n, d] (device FP32,
// or null) into the persistent loop's partition, else breadth-first; then the sliced ELL and the
// gather-cache tables.
gs_status gs_graph_reorder(gs_ctx* ctx, gs_graph* g, const float* X, int d, const int* points_order);
// Coordinate bisection of the points into the persistent loop's partition (order.cu): *ord
// (inside buf) receives position -> point, or stays null when the points cannot be bisected
// (dimension, part sizes); buf holds gs_points_order_bytes(ctx, n, d) bytes (0: not possible).
size_t gs_points_order_bytes(const gs_ctx* ctx, int64_t n, int d);
gs_status gs_points_order(gs_ctx* ctx, const float* X, int64_t n, int d, void* buf, size_t bytes, int** ord);
// Gather-cache tables for `blocks` partition blocks: on the given row ranges (parts, blocks + 1
// boundaries), else on cost-balanced ranges.
gs_status gs_graph_build_xcache(gs_ctx* ctx, gs_graph* g, int blocks, const std::vector<int>* parts);
// Boundaries of `blocks` ranges of whole 32-row slices with equal slice counts (+-1).
std::vector<int> gs_equal_slice_rows(int64_t n, int blocks);
// rows per block of the persistent loop's partition (one block per SM, whole slices)
// Block synchronisation of the persistent loop: the option if set, else the autotuned choice for
// the graph, else the context's last one, else tagged values (the fastest on the graphs measured).
// The context's autotuner record for a graph of g's size and B columns (degree K preferred).
static inline const TuneRecord* gs_tune_lookup(const gs_ctx* ctx, const gs_graph* g, int B, int K)
{
    const TuneRecord* any = nullptr;
    for (auto it = ctx->tune_log.rbegin(); it != ctx->tune_log.rend(); ++it) {
        if (it->n != g->n || it->nnz != g->nnz || it->B != B) continue;
        if (it->K == K) return &*it;
        if (!any) any = &*it;
    }
    return any;
}
// Tagged-word staging for a graph without its own autotune record: grouped re-reads pay where a
// block's sums are long enough that most words are ready when its staging starts (672 rows per
// block: 2.29 against 2.36 us per order on the 100k manifold), one-at-a-time re-reads where the
// exchange dominates (480 rows: 1.87 against 1.92 us; 160 rows: 1.36 against 1.58 us).
constexpr int kGroupedStagingRows = 576;
static inline int gs_tagged_form(const gs_graph* g)
{
    return (g && g->xc_rpb > 0 && g->xc_rpb < kGroupedStagingRows) ? 4 : 2;
}
// The block synchronisation as chosen (option, else the graph's autotune record, else the
// context's last choice if it was not a tagged form, else the tagged form above): 0 grid
// barrier, 1 neighbour flags, 2 tagged words re-read in groups, 4 tagged words re-read one at a time.
static inline int gs_persist_sync_setting(const gs_ctx* ctx, const gs_graph* g)
{
    if (ctx->persist_sync != 3) return ctx->persist_sync;
    if (g && g->tuned_sync >= 0) return g->tuned_sync;
    if (g) {
        const TuneRecord* r = gs_tune_lookup(ctx, g, 1, 0);
        if (r && r->sync >= 0) return r->sync;
    }
    if (ctx->tuned_sync == 0 || ctx->tuned_sync == 1) return ctx->tuned_sync;
    if (!g && ctx->tuned_sync >= 0) return ctx->tuned_sync;
    return gs_tagged_form(g);
}
// The synchronisation family: both tagged-word forms report 2 (they need the same exchange buffer).
static inline int gs_persist_sync_choice(const gs_ctx* ctx, const gs_graph* g)
{
    const int s = gs_persist_sync_setting(ctx, g);
    return s == 4 ? 2 : s;
}
// Words of the persistent loop's synchronisation buffer: barrier counter and generation, then one
// 128-byte line per block (up to two blocks per SM) for its ready counter.
static inline size_t gs_persist_bar_words(const gs_ctx* ctx)
{
    return 32 * (1 + 2 * (size_t)(ctx->num_sms > 0 ? ctx->num_sms : 148));
}
// Blocks of the gather-cache partition (one or two per SM) and rows per block (whole slices) when
// n rows are split over `blocks` blocks.
static inline int gs_persist_cache_blocks(const gs_ctx* ctx)
{
    return (ctx->num_sms > 0 ? ctx->num_sms : 148) * ctx->persist_bps;
}
static inline int gs_persist_rows_per_block(const gs_ctx*, int64_t n, int blocks)
{
    return (int)(((n + blocks - 1) / blocks + GS_SELL_C - 1) / GS_SELL_C * GS_SELL_C);
}
// dst[r, :] = src[perm[r], :] (to the filter's order) or dst[perm[r], :] = src[r, :] (back)
void gs_permute_rows(gs_ctx* ctx, int64_t n, int B, const int* perm, const float* src, float* dst,
                     bool to_filter_order);

// --------------------------------------------------------------------- knn.cu
void gs_exclusive_scan(cudaStream_t s, const int* cnt, int64_t n, int64_t* out, int64_t* sums);
// ord: the points' bisection order (position -> point) for the tensor-memory screen, or null (it
// is then computed in the workspace when the screen runs and the points can be bisected).
gs_status gs_knn_launch(gs_ctx* ctx, const float* X, int64_t n, int d, int k, int32_t* idx,
                        float* dist, double* dist64, const int* ord);
size_t gs_knn_ws_bytes(const gs_ctx* ctx, int64_t n, int d);
// --------------------------------------------------------------------- knn_umma.cu
size_t gs_knn_umma_bytes(int64_t n, int d);
bool gs_knn_umma_available();
gs_status gs_knn_screen_umma(gs_ctx* ctx, const float* X, const float* norms, int64_t n, int d,
                             unsigned char* ws, const int* ord, int* cand);
gs_status gs_build_graph_impl(gs_ctx* ctx, const float* X, int64_t n, int d, int k, float sigma,
                              gs_graph** out);

// ------------------------------------------------------------- cheb.cu (filter + loops)
// What the last Chebyshev order does with f = p_K(x) for a block with B columns.
enum EpiKind : int {
    EPI_STORE = 0,    // out = f
    EPI_DIVIDE = 1,   // out = num / f (0 where num == 0); xnext = vol * out
    EPI_BARY_V = 2,   // d = V * f; mu = exp(sum alpha ln d); V <- V mu / d; xnext = vol * V
};

struct Epilogue {
    int kind = EPI_STORE;
    float* out = nullptr;          // [n, B] output (STORE/DIVIDE/BARY_W)
    const float* num = nullptr;    // [n, B] numerator (DIVIDE: a or b; BARY_W: M)
    const float* vol = nullptr;    // [n] vertex weights or null
    float* xnext = nullptr;        // [n, B] vol * result, the next filter input (may be null)
    bool xnext_to_scratch = false; // let the filter put xnext in its free scratch buffer
    // eps check (DIVIDE, B == 1): err += |old[i] * f[i] - num[i]|
    const float* old = nullptr;
    double* err_partials = nullptr;
    // barycenter
    float* V = nullptr;            // [n, m] scalings v_i (BARY_V, updated in place)
    const double* alpha = nullptr; // [m]
    float* mu = nullptr;           // [n] barycenter output (BARY_V)
    float* dsave = nullptr;        // [n, m] optional copy of d (tape for the adjoint)
    float* fsave = nullptr;        // [n, B] optional copy of the filter value f (adjoint tape)
};

struct FilterPlan {
    int B = 1;
    int vec = 1;                   // floats per lane access (4 needs B % 4 == 0 and 16 B alignment)
    int group = 8;                 // lanes per row (B == 1: split nonzeros; B > 1: split columns)
    int block = 256;
    int kernel = 0;                // GS_KERNEL_* variant: the context option, else the autotuned one
    int split_t = 4;               // B == 1 row-split kernel: threads per row (2, 4 or 8)
};

// aligned: every block the kernels gather from starts on a 16-byte boundary
FilterPlan gs_filter_plan(const gs_ctx* ctx, const gs_graph* g, int B, bool aligned, int K);
int gs_err_partials_count();

// Enqueue the K fused Chebyshev orders of p_K applied to x ([n, B]).
//   x_writable: x may be overwritten by intermediate orders (the loop's own buffers)
//   bufA/bufB : scratch [n, B] (bufB only needed when !x_writable or K == 1)
//   y         : accumulator [n, B] (may be the output itself for EPI_STORE)
//   scratch_out: receives the buffer the epilogue's xnext went to (when xnext_to_scratch)
gs_status gs_filter_enqueue(gs_ctx* ctx, const gs_graph* g, const double* c, int K, int B,
                            float* x, bool x_writable, float* bufA, float* bufB, float* y,
                            const Epilogue& epi, const int* done_flag, float** scratch_out);
bool gs_filter_supports(int B, bool aligned);

gs_status gs_sinkhorn_impl(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b,
                           const float* vol, double t, int K, double eps, int iters, float* u,
                           float* v, double* dist, int32_t* iters_done);
gs_status gs_sinkhorn_grad_impl(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b,
                                const float* vol, double t, int K, int iters, int ck,
                                double* dist, float* grad_a, float* grad_b);
gs_status gs_barycenter_grad_impl(gs_ctx* ctx, const gs_graph* g, const float* M, int m,
                                  const double* alpha, const float* vol, double t, int K, int iters,
                                  int ck, const float* mubar, float* mu_out, double* grad_alpha);
gs_status gs_sinkhorn_batched_impl(gs_ctx* ctx, int nprob, const gs_graph* const* graphs,
                                   const float* const* a, const float* const* b, const double* t,
                                   const int* K, int iters, float* const* u, float* const* v,
                                   double* dist);
gs_status gs_sinkhorn_persistent(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b,
                                 const float* vol, const float* coef_dev, int K, int iters,
                                 float* x, float* A, float* y, float* u, float* v, unsigned* bar,
                                 unsigned long long* tagged);
gs_status gs_autotune_impl(gs_ctx* ctx, gs_graph* g, int B, int K, int* choice_out);
gs_status gs_barycenter_impl(gs_ctx* ctx, const gs_graph* g, const float* M, int m,
                             const double* alpha, const float* vol, double t, int K, int iters,
                             float* mu, float* v_state);
// Definition 4.3 (muT, muC: [n] caller buffers, normalised barycenters) and Definition 4.4.
gs_status gs_barycentric_distance_impl(gs_ctx* ctx, const gs_graph* g, const float* MT, int mT,
                                       const double* alphaT, const float* MC, int mC, const double* alphaC,
                                       const float* vol, double t, int K, int bary_iters, int sink_iters,
                                       float* muT, float* muC, double* dist);
gs_status gs_barycenter_effect_impl(gs_ctx* ctx, const float* Y, int64_t n, int d, const float* muT,
                                    const float* muC, double* out);
// Algorithm 1 with FP64 potentials ln u, ln v and an extended-range Chebyshev recurrence
// (logdomain.cu); caller node order; eps > 0 stops as gs_sinkhorn does.
gs_status gs_sinkhorn_log_impl(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b, const float* vol,
                               double t, int K, double eps, int iters, double* log_u, double* log_v, double* dist,
                               int32_t* iters_done);
// Euler implicit heat kernel Y = (I + (t/K) L)^{-K} V by K conjugate-gradient solves (implicit.cu).
gs_status gs_heat_apply_implicit_impl(gs_ctx* ctx, const gs_graph* g, double t, int K, const float* V, int B,
                                      float* Y, double tol, int iters);

// ------------------------------------------------------------------ combinatorial.cu
// Build g's combinatorial operator (once; waits for the stream) and view g with it in place of P.
gs_status gs_graph_build_combinatorial(gs_ctx* ctx, gs_graph* g);
void gs_combinatorial_view(const gs_graph* g, gs_graph* view);

// ------------------------------------------------------------------------ reduce.cu
// dist[0] = 4t sum vol (a ln u + b ln v), dist[1] = sqrt; flags NONFINITE on bad scalings.
gs_status gs_distance_enqueue(gs_ctx* ctx, int64_t n, const float* a, const float* b,
                              const float* vol, const float* u, const float* v, double t,
                              double* partials, double* dist);
int gs_reduce_blocks();

// Device-side argument checks (raised as GS_ERR_ARG at the next gs_sync; skipped while the
// context's check option is off).  Marginals: every entry finite and >= 0, and the masses
// sum vol a and sum vol b equal within GS_MASS_RTOL of the larger.  Barycenter weights: alpha >= 0
// and |sum alpha - 1| <= GS_WEIGHT_TOL.
constexpr double GS_MASS_RTOL = 1e-6;
constexpr int GS_CHECK_BLOCKS = 128;  // blocks of the single-problem mass check
constexpr double GS_WEIGHT_TOL = 1e-6;
struct gs_marginals {
    const float* a;
    const float* b;
    const float* vol;   // null = unit weights
    int64_t n;
};
// one problem (blocks over its entries, fixed-order final sum)
gs_status gs_check_marginals(gs_ctx* ctx, const gs_marginals& m);
gs_status gs_check_weights(gs_ctx* ctx, const double* alpha, int m);
// the same checks over `count` descriptors already on the device (one block each)
gs_status gs_check_marginals_dev(gs_ctx* ctx, const gs_marginals* probs_dev, int count);
