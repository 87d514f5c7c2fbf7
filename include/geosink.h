/*
 * geosink.h -- C ABI of the GB300 Geodesic Sinkhorn library (libgeosink.so).
 *
 * Geodesic Sinkhorn (arXiv 2211.00805) computes entropic optimal transport on a data graph by
 * replacing the Gibbs kernel with the heat kernel H_t = exp(-t L) of the graph Laplacian
 * (Sec. 3.2-3.4), applied through a degree-K Chebyshev polynomial p_K(L, t) (Sec. 3.5) inside
 * the Sinkhorn scaling loop (Algorithm 1) and the fixed-support barycenter (Sec. 3.3).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Array arguments are DEVICE pointers owned by the caller (e.g. torch.empty(..., "cuda")),
 *    unless the parameter says "host".  Blocks are row-major: V[n, B] has V[i * B + c].
 *    Inputs and outputs must not alias unless stated.  Floating-point arrays are FP32 unless
 *    the type says double.
 *  - Every call is enqueued on the context's stream and returns without waiting for the GPU,
 *    except gs_sync, gs_graph_info and the graph constructors (which wait for sizes they must
 *    know on the host).  Scalar results are written to device memory.
 *  - The return value reports argument errors (GS_ERR_ARG), CUDA launch/allocation errors
 *    (GS_ERR_CUDA / GS_ERR_OOM) and unsupported shapes (GS_ERR_UNSUPPORTED) immediately.
 *    Conditions found by the kernels themselves (non-finite scalings, a loop that did not reach
 *    its tolerance, a bounded wait that ran out) are recorded in the context and returned by the
 *    next gs_sync.  gs_last_error gives a message for the last non-OK status.
 *  - Graph handles (gs_graph) and contexts (gs_ctx) are owned by the library; free them with
 *    gs_graph_destroy / gs_destroy.  A graph may be used with any context on the same device.
 *  - Nothing is thread-safe per context: one host thread at a time per gs_ctx.
 *  - Working memory: the context keeps one device workspace that grows on demand (cudaMalloc).
 *    A call that needs a larger workspace while its stream is being captured into a CUDA graph
 *    fails with GS_ERR_UNSUPPORTED; run the same call once before capturing.
 *
 * Notation (mapping to the paper)
 * -------------------------------
 *  P = D^{-1/2} A D^{-1/2}, L = I - P (symmetric-normalised Laplacian, spectrum in [0, 2]),
 *  Ls = L - Id = -P (the Chebyshev argument of Sec. 3.5).  Source/target marginals a, b are the
 *  paper's mu, nu; scalings u, v are the paper's v, w; vertex weights vol are the paper's a
 *  (Algorithm 1).  Diffusion time t relates to the regularisation by lambda = 4t (Sec. 3.2).
 */
#ifndef GEOSINK_H
#define GEOSINK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_ARG = 1,            /* invalid argument (null pointer, size, range)                  */
    GS_ERR_CUDA = 2,           /* a CUDA runtime call or kernel launch failed                   */
    GS_ERR_OOM = 3,            /* device allocation failed                                      */
    GS_ERR_NONFINITE = 4,      /* a scaling, filter output or distance became inf/NaN/negative  */
    GS_ERR_NOT_CONVERGED = 5,  /* eps > 0 and the marginal error never fell below eps           */
    GS_ERR_TIMEOUT = 6,        /* a bounded in-kernel wait gave up                              */
    GS_ERR_UNSUPPORTED = 7     /* shape or state this library does not handle                   */
} gs_status;

typedef struct gs_ctx gs_ctx;
typedef struct gs_graph gs_graph;

/* ------------------------------------------------------------------------------ context --- */

/* Create a context on CUDA device `device` that enqueues on `stream` (a cudaStream_t passed as
 * void*, NULL = the legacy default stream).  *ctx receives the handle.  Errors: GS_ERR_ARG for
 * a null ctx or bad device, GS_ERR_CUDA / GS_ERR_OOM. */
gs_status gs_create(gs_ctx **ctx, int device, void *stream);

/* Free the context and its workspace (waits for its stream first). NULL is accepted. */
gs_status gs_destroy(gs_ctx *ctx);

/* Switch the stream later calls enqueue on (cudaStream_t as void*). */
gs_status gs_set_stream(gs_ctx *ctx, void *stream);

/* Message of the last non-OK status returned on this context ("" if none).  The string is
 * owned by the context and valid until the next call on it. */
const char *gs_last_error(const gs_ctx *ctx);

/* Wait for the context's stream, then return and clear the status recorded by kernels since
 * the last gs_sync: GS_ERR_NONFINITE, GS_ERR_NOT_CONVERGED, GS_ERR_TIMEOUT, or GS_OK. */
gs_status gs_sync(gs_ctx *ctx);

/* Grow the workspace to at least `bytes` now (for use before CUDA-graph capture). */
gs_status gs_reserve(gs_ctx *ctx, int64_t bytes);

/* Context options (host call).  GS_OPT_LOOP selects how gs_sinkhorn runs a fixed iteration count
 * (eps <= 0): 0 one persistent cooperative launch with bounded grid barriers between the Chebyshev
 * orders (falls back to 1 when the device cannot co-schedule the grid); 1 CUDA-graph replay of
 * per-order launches; 2 (default) the mode gs_autotune measured faster on the graph, else 0.
 * All compute the same thing.  Errors: GS_ERR_ARG. */
/* GS_OPT_BARRIER_SELFTEST = 1 makes the next persistent launch wait at its first grid barrier for
 * one block more than the grid has (with neighbour-flag sync, tagged values, or the persistent
 * log-domain loop of gs_sinkhorn_log: for a stage no block will publish, including its own):
 * every block's bounded wait runs out (~10 ms), the launch ends and gs_sync reports
 * GS_ERR_TIMEOUT, leaving the context usable.  It exercises failure handling without faulting the
 * GPU; the option resets itself after that launch. */
/* GS_OPT_B1_KERNEL / GS_OPT_BLK_KERNEL pick the Chebyshev order kernel for one column / several
 * columns: 0 automatic, 1 sliced ELL (one column), 2 lane-split CSR, 3 chunked CSR with
 * asynchronous gathers into shared memory, 4 staged neighbour lists (several columns), 5 the
 * sliced-ELL / lane-group kernels with each block walking one contiguous row range, 6 sliced ELL
 * with every row split across 4 threads (one column: the automatic choice), 7 sliced ELL with one
 * 1024-thread block per SM over one contiguous row range.  All variants compute the same
 * recurrence; they differ in summation order only. */
/* GS_OPT_KNN_TENSOR: how kNN distances are screened before the exact FP64 rerank.  2 (default):
 * squared distances as one augmented 3xTF32 contraction on the fifth-generation tensor cores
 * (tcgen05, operands staged by TMA in each CTA's shared memory, accumulators in tensor memory) when
 * d <= 62; 1: warp-level TF32 MMA (3xTF32) when d >= 16; 0: FP32 CUDA-core dot products.  A
 * choice the shape or device does not allow falls back to the next lower one; the rerank makes
 * every choice exact. */
/* GS_OPT_PERSIST_SMEM_GRAPH: how the persistent loop reads the operator.  2 (default): each
 * block's slices (values and 16-bit local column indices) are copied into shared memory once, and
 * every order first copies the block's distinct neighbour values into a shared-memory cache;
 * 1: slices in shared memory, neighbour values gathered from global memory; 0: everything from
 * global memory.  Each mode falls back to the next lower one when its tables do not fit in 200 KB
 * of shared memory.  Same arithmetic in every mode. */
/* GS_OPT_PERSIST_SYNC: how the blocks of the persistent loop wait for one another between
 * Chebyshev orders when the gather-cache tables are in use (mode 2 above).  1: each block waits
 * only for the blocks owning rows it reads (per-block ready counters) and keeps its own rows'
 * recurrence values in registers; 2: the same, with the readiness carried by the exchanged values
 * themselves (value + stage words in three rotating slots, see GS_OPT_TAG_WORD; no counters or
 * fences), a thread's words that are not ready yet re-read together; 4: as 2, those words re-read
 * one at a time (fewer loads in flight: faster where the exchange dominates, e.g. small graphs);
 * 0: a barrier over the whole grid; 3 (default): the one gs_autotune measured fastest on the graph
 * (else on the context's last tuned graph, else 2).  Same arithmetic in all of them.  All honour
 * GS_OPT_BARRIER_SELFTEST. */
/* GS_OPT_PERSIST_BLOCKS: blocks per SM of the gather-cache partition (1 = one 1024-thread block,
 * default; 2 = two 512-thread blocks, so one block's exchange overlaps the other's sums), for the
 * tagged-value and neighbour-flag forms.  Applies to graphs built after the call. */
/* GS_OPT_TAG_WORD: the word of the tagged-value exchange (GS_OPT_PERSIST_SYNC 2).  4 (default):
 * the FP32 value with its last mantissa bit carrying the stage parity, so the values one block
 * reads from another may differ from the exact FP32 ones by one unit in the last place (results
 * agree with the exact form to ~1e-8 relative, not bitwise); 8: exact FP32 value plus a 32-bit
 * stage tag (results bitwise equal to the other loop forms), with twice the exchanged bytes. */
/* GS_OPT_CHECK_ARGS: device-side argument checks (1, default) or none (0).  gs_sinkhorn, gs_distance,
 * gs_sinkhorn_log, gs_sinkhorn_grad and gs_sinkhorn_batched check that both marginals are finite
 * and non-negative and that their masses sum_i vol_i a_i and sum_i vol_i b_i (the two marginals of
 * Algorithm 1's plan, so they must agree for a plan to exist) differ by at most 1e-6 of the larger;
 * gs_barycenter, gs_barycenter_grad and gs_barycentric_distance check that the weights alpha are
 * non-negative and sum to 1 within 1e-6 (Sec. 3.3).  The checks run on the device in the call's
 * stream (one small launch each) and a failure is raised as GS_ERR_ARG by the next gs_sync; the
 * computation itself still runs.  Turn them off to evaluate the unrolled iteration at unbalanced
 * marginals on purpose (e.g. a distance to a barycenter that is not normalised). */
/* GS_OPT_TILE_LANES: with GS_OPT_BLK_KERNEL set to a row-group variant (2 or 5), the lanes that
 * share a row (1, 2, 4, 8, 16 or 32; fewer lanes walk the row's columns in more passes, at most 8),
 * i.e. the RHS tile width; with GS_OPT_B1_KERNEL = 6, the threads per row (2, 4 or 8).  0 (default):
 * the kernel's own mapping.  gs_autotune times these widths itself; this option fixes one. */
/* GS_OPT_NODE_ORDER: the order inside each part of the coordinate bisection for graphs built from
 * points after the call.  1 (default): eight degree classes, inside a class the rows by the
 * smallest neighbouring part that reads them (fastest for the one-column filter and the Sinkhorn
 * loop, whose exchanged values a neighbouring block then stages from fewer memory sectors);
 * 0: decreasing degree only (fastest for the several-column filter and the barycenter, whose row
 * groups then hold rows of equal length).  Same results either way up to summation order. */
/* GS_OPT_LOOP_REGS: the persistent loop with tagged 4-byte exchange words, where every block of its
 * partition has at most 672 rows, runs one row per thread and keeps each row's first 16 operator
 * entries (values and cache indices) in registers for the whole loop, so that only the neighbour
 * values are read from shared memory there.  1 (default): on; 0: off (all entries read from shared
 * memory every order, 1024 threads per block).  Bitwise the same results either way. */
enum { GS_OPT_LOOP = 1, GS_OPT_BARRIER_SELFTEST = 2, GS_OPT_B1_KERNEL = 3, GS_OPT_BLK_KERNEL = 4,
       GS_OPT_KNN_TENSOR = 5, GS_OPT_PERSIST_SMEM_GRAPH = 6, GS_OPT_PERSIST_SYNC = 7,
       GS_OPT_PERSIST_BLOCKS = 8, GS_OPT_TAG_WORD = 9, GS_OPT_CHECK_ARGS = 10, GS_OPT_TILE_LANES = 11,
       GS_OPT_NODE_ORDER = 12, GS_OPT_LOOP_REGS = 13 };
gs_status gs_set_option(gs_ctx *ctx, int option, int value);

/* Host query of an option.  For GS_OPT_LOOP, GS_OPT_B1_KERNEL and GS_OPT_PERSIST_SYNC left on
 * automatic it reports what
 * a call on a graph without its own autotune record would use (the context's last autotune
 * result, else the built-in default: persistent loop, row-split kernel).  Errors: GS_ERR_ARG. */
gs_status gs_get_option(const gs_ctx *ctx, int option, int *value);

/* Host query: number of GPU kernels this context has enqueued so far (a replayed CUDA graph
 * counts each of its kernel nodes).  Used to report launch counts; *count must not be NULL. */
gs_status gs_launch_count(const gs_ctx *ctx, int64_t *count);

/* ------------------------------------------------------------------------ coefficients --- */


/* Chebyshev coefficients of the heat kernel (Sec. 3.5: "evaluated with the Bessel function").
 * HOST call.  Writes c[0..K] (host array of K+1 doubles) such that
 *     exp(-t L) ~ sum_{k=0}^{K} c[k] T_k(P),   c[0] = e^{-t} I_0(t),  c[k] = 2 e^{-t} I_k(t),
 * the expansion of Sec. 3.5 in the polynomial variable P = Id - L (T_k(L - Id) = (-1)^k T_k(P)).
 * I_k is the modified Bessel function of the first kind.  Requires t > 0, K >= 0.
 * Errors: GS_ERR_ARG. */
gs_status gs_cheb_coeffs(double t, int K, double *c);

/* Step order of one 32-row slice of the sliced-ELL operator (the graph builder's bank-aware
 * entry order for the one-column Sinkhorn loop, exposed for inspection).  HOST call.
 * idx: W * 32 local cache indices of the slice, entry j of row l at idx[j * 32 + l] (the index's
 * shared-memory bank is idx mod 32).  steps (out, same layout): the step at which each entry is
 * summed.  Every row gets each step 0..W-1 exactly once; where no bank holds more than W of the
 * slice's entries, no step has two entries in one bank (a bipartite edge colouring of
 * rows x banks), and entries beyond a full bank are grouped into shared steps.  Requires
 * 1 <= W <= 64.  Errors: GS_ERR_ARG. */
gs_status gs_sell_step_order(const uint16_t *idx, int W, unsigned char *steps);

/* ----------------------------------------------------------------------------- graphs --- */

/* k nearest neighbours of every point (the common graph of Sec. 4 is built from them).
 * X: [n, d] points.  idx: [n, k] int32 neighbour indices, dist: [n, k] Euclidean distances, both
 * ordered by increasing distance, the point itself excluded, ties broken by lower index.
 * Distances are screened in FP32 and the candidates re-ranked with FP64 direct differences.
 * Requires 2 <= n < 2^31, 1 <= d <= 1024, 1 <= k <= 24, k < n.  Errors: GS_ERR_ARG. */
gs_status gs_knn(gs_ctx *ctx, const float *X, int64_t n, int d, int k, int32_t *idx, float *dist);

/* Build the graph of Sec. 4 from a point cloud: symmetric kNN graph (union of the directed kNN
 * edges), Gaussian affinities A_ij = exp(-d_ij^2 / sigma^2) (sigma <= 0 selects sigma = median of
 * the n*k kNN distances), degrees D_ii = sum_j A_ij and P = D^{-1/2} A D^{-1/2} (Sec. 3.4).
 * Same limits as gs_knn.  Waits for the stream (the edge count sizes the graph).
 * *out receives a library-owned handle.  Errors: GS_ERR_ARG, GS_ERR_OOM, GS_ERR_CUDA. */
gs_status gs_build_graph(gs_ctx *ctx, const float *X, int64_t n, int d, int k, float sigma,
                         gs_graph **out);

/* Build the operator from a caller-supplied symmetric weighted adjacency in CSR form
 * (device rowptr [n+1] int64, col [nnz] int32 ascending per row, w [nnz] FP32 >= 0, no self-
 * loops, every row non-empty).  Degrees and P are formed as in gs_build_graph (Sec. 3.4).
 * Symmetry is the caller's promise and is not checked.  Errors: GS_ERR_ARG (n < 2,
 * nnz >= 2^31), GS_ERR_OOM. */
gs_status gs_graph_from_csr(gs_ctx *ctx, int64_t n, const int64_t *rowptr, const int32_t *col,
                            const float *w, gs_graph **out);

/* Host query of a graph's size: n nodes, nnz stored off-diagonal entries, sigma used (0 for
 * graphs from gs_graph_from_csr).  Any output pointer may be NULL. */
gs_status gs_graph_info(const gs_graph *g, int64_t *n, int64_t *nnz, double *sigma);

/* Host query of the graph's execution layout (diagnostics; not in the paper).  Writes up to
 * `count` values into `out`, in this order: 0 sliced-ELL slices, 1 sliced-ELL entries (with
 * padding), 2 gather-cache tables built (0/1), 3 partition blocks, 4 rows of the largest block,
 * 5 largest entry count of a block, 6 largest distinct-column count of a block, 7 sum of the blocks'
 * distinct-column counts, 8 largest dependency-list length.  Errors: GS_ERR_ARG. */
gs_status gs_graph_layout(const gs_graph *g, int64_t *out, int count);

/* Copy the graph out in CSR form, rows in node order and columns ascending (device arrays:
 * rowptr [n+1] int64, col [nnz] int32, A [nnz] FP32 affinities, P [nnz] FP32 normalised
 * weights D^{-1/2} A D^{-1/2}, both of Sec. 3.4).  Any of the output pointers may be NULL.  Used
 * to check edge sets against a reference. */
gs_status gs_graph_export_csr(gs_ctx *ctx, const gs_graph *g, int64_t *rowptr, int32_t *col,
                              float *A, float *P);

/* Autotuner (not in the paper; it serves throughput): times every Chebyshev-order kernel variant
 * for B columns and degree K on this graph (heat-filter applies on a synthetic block, CUDA events,
 * waits for the device) and records the fastest in the graph handle; for B = 1 it also times a
 * short fixed-count Sinkhorn loop as graph replay and as the persistent launch with each
 * GS_OPT_PERSIST_SYNC form, and records the fastest loop mode and synchronisation.
 * *choice (may be NULL) receives the chosen variant (the GS_OPT_*_KERNEL value).
 * For B > 1 it also times each row-group variant at two RHS tile widths (all of a row's columns
 * per lane-group pass, or half of them in two passes); for B == 1 the row-split kernel with 2, 4
 * and 8 threads per row.  The decision is also kept by the context per (n, nnz, B, K)
 * (gs_autotune_choices).  Errors: GS_ERR_ARG, GS_ERR_UNSUPPORTED. */
/* Later calls on the graph use the recorded choices while the context's options are automatic
 * (GS_OPT_B1_KERNEL / GS_OPT_BLK_KERNEL 0, GS_OPT_LOOP 2, GS_OPT_PERSIST_SYNC 3); the context also
 * keeps the last one-
 * column choices for graphs that were never tuned (e.g. rebuilt graphs of the same workload). */
gs_status gs_autotune(gs_ctx *ctx, gs_graph *g, int B, int K, int *choice);

/* Host query of the autotuner's decision for graphs of g's size (n, nnz) and B columns, degree K
 * preferred (the context keeps one record per (n, nnz, B, K) that gs_autotune timed, so graphs
 * rebuilt for the same workload use it too).  Writes up to `count` ints into `out`:
 *   0 order-kernel variant (a GS_OPT_*_KERNEL value; 0 none recorded),
 *   1 lanes per row the calls will use (B > 1: the RHS tile is this many lanes x 4 or 1 floats;
 *     B == 1: threads per row of the row-split kernel),
 *   2 columns per pass of a lane group (B > 1), 1 for B == 1,
 *   3 Sinkhorn loop mode recorded for B == 1 (1 persistent, 2 CUDA-graph replay, 0 not timed),
 *   4 the persistent loop's block synchronisation recorded for B == 1 (-1 not timed),
 *   5 1 if a record exists, else 0 (the other entries then describe the defaults).
 * Not in the paper (it serves throughput).  Errors: GS_ERR_ARG. */
gs_status gs_autotune_choices(const gs_ctx *ctx, const gs_graph *g, int B, int K, int *out, int count);

/* Free a graph (waits for the device). NULL is accepted. */
gs_status gs_graph_destroy(gs_graph *g);

/* ------------------------------------------------------------------------ heat filter --- */

/* Y = p_K(L, t) V (Sec. 3.5): the degree-K Chebyshev approximation of exp(-tL) applied to the
 * B columns of V[n, B], through the recurrence T_{k+1} = 2 P T_k - T_{k-1} with the running sum
 * y += c_k T_k fused into each of the K sparse products.  V and Y: [n, B] FP32, must not alias.
 * Requires t > 0, 1 <= K <= 10000, and 1 <= B <= 256, or B a multiple of 4 up to 1024 with V on
 * a 16-byte boundary (such blocks are read as float4).  Errors: GS_ERR_ARG, GS_ERR_UNSUPPORTED. */
gs_status gs_heat_apply(gs_ctx *ctx, const gs_graph *g, double t, int K, const float *V, int B,
                        float *Y);

/* Heat filter of the combinatorial Laplacian L = D - A (Sec. 3.4) with the expansion of Sec. 3.5:
 *     Y = p_K(L', s) V ~ exp(-t (D - A)) V,   L' = (2 / lam)(D - A),   s = t lam / 2,
 * where lam = 2 max_i D_ii bounds the largest eigenvalue of D - A (Gershgorin), so the spectrum of
 * L' lies in [0, 2] as Sec. 3.5 assumes, and exp(-t L) = exp(-s L').  The recurrence runs on
 * M = Id - L' (its diagonal 1 - D_ii / max_j D_jj stored with the off-diagonal A_ij / max_j D_jj)
 * with the coefficients c_k(s) of gs_cheb_coeffs.  The first call on a graph builds M (device
 * memory of nnz + n entries kept with the graph; waits for the stream once); later calls are
 * asynchronous.  lam (host double, may be NULL) receives lam.  V, Y: [n, B] as gs_heat_apply, same
 * limits.  Errors: GS_ERR_ARG, GS_ERR_UNSUPPORTED, GS_ERR_OOM. */
gs_status gs_heat_apply_combinatorial(gs_ctx *ctx, gs_graph *g, double t, int K, const float *V, int B,
                                      float *Y, double *lam);

/* Allocation-free variant of gs_heat_apply for callers that cannot allocate device memory:
 * plug-ins whose host application owns every device allocation (the library may not take memory
 * from under it), and real-time loops that must never enter the allocator, where cudaMalloc can
 * block or fail under memory pressure.  The paper has no counterpart; this is a deployment
 * convenience.
 * It computes the same Y = p_K(L, t) V (Sec. 3.5) with the same kernels, but takes the operator
 * as plain CSR device arrays (rowptr [n+1] int32 offsets, col [nnz] int32, pval [nnz] FP32 holding
 * P = D^{-1/2} A D^{-1/2}, as gs_graph_export_csr returns them once rowptr is narrowed to int32)
 * and needs no gs_ctx or gs_graph.  The CSR is trusted, not checked: rowptr must start at 0, be
 * non-decreasing and end at nnz, and every col entry must lie in [0, n); anything else reads out
 * of bounds.  Its two scratch blocks live in a fixed 8 MiB device array inside the library,
 * present on every GPU that loads it until the process exits, so n * B <= 1,048,576 (2^20) is
 * required (GS_ERR_UNSUPPORTED otherwise).  No cudaMalloc, cudaFree or other device allocation
 * happens in this call.
 *   - Works on the calling thread's current device; `stream` is a cudaStream_t as void*.
 *   - The first call on each device looks up the array's device address (cudaGetSymbolAddress);
 *     make that first call before any stream capture.
 *   - Every call shares the one scratch array: calls that overlap on the GPU (other streams,
 *     other threads) race and corrupt each other; serialise them.  Nothing in the scratch must
 *     start at zero, so stale contents from an earlier call do no harm.
 * Same limits on t, K and B as gs_heat_apply, with both V and Y on a 16-byte boundary for
 * B > 256.  Returns GS_ERR_ARG / GS_ERR_UNSUPPORTED / GS_ERR_CUDA (no message: there is no
 * context). */
gs_status gs_heat_apply_noalloc(int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *col,
                                const float *pval, double t, int K, const float *V, int B,
                                float *Y, void *stream);

/* ----------------------------------------------------------------------------- Sinkhorn --- */

/* Algorithm 1 (Geodesic Sinkhorn): v <- 1; repeat { u <- a / p_K(vol * v); v <- b / p_K(vol * u) }
 * (the division is fused into the last Chebyshev order), then the distance reduction
 *     dist[0] = W^2 = 4t sum_i vol_i (a_i ln u_i + b_i ln v_i)      (Algorithm 1's return value)
 *     dist[1] = W   = sqrt(W^2)                                     (Definition 4.1)
 * accumulated in FP64 (0 ln 0 := 0; a_i = 0 gives u_i = 0).
 *   a, b   : [n] non-negative marginals of equal mass sum(vol a) = sum(vol b) (checked on the device,
 *            see GS_OPT_CHECK_ARGS)
 *   vol    : [n] vertex weights, NULL = all ones
 *   eps    : > 0 -> stop at the first iteration j, j a multiple of 10, whose marginal error
 *            sum_i |u_i (p_K(vol * v))_i - a_i| is below eps (GS_ERR_NOT_CONVERGED at gs_sync if
 *            none); <= 0 -> run exactly `iters` iterations
 *   u, v   : [n] outputs (scalings after the last iteration done)
 *   dist   : [2] double output (device), may be NULL
 *   iters_done : [1] int32 output (device), may be NULL
 * Non-finite or negative scalings are reported as GS_ERR_NONFINITE at gs_sync.
 * Requires t > 0, K >= 1, iters >= 1.  Errors: GS_ERR_ARG. */
gs_status gs_sinkhorn(gs_ctx *ctx, const gs_graph *g, const float *a, const float *b,
                      const float *vol, double t, int K, double eps, int iters, float *u, float *v,
                      double *dist, int32_t *iters_done);

/* Geodesic Sinkhorn distance only (Definition 4.1): gs_sinkhorn with the scalings kept in the
 * context's workspace.  dist: [2] double (device) receiving W^2 and W. */
gs_status gs_distance(gs_ctx *ctx, const gs_graph *g, const float *a, const float *b,
                      const float *vol, double t, int K, double eps, int iters, double *dist);

/* Algorithm 1 in the log domain, for diffusion times small enough that the scalings of gs_sinkhorn
 * leave the FP32 range (it reports GS_ERR_NONFINITE there).  The same iteration,
 *     ln u <- ln a - ln p_K(vol * e^{ln v}),   ln v <- ln b - ln p_K(vol * e^{ln u}),   ln v = 0 at
 * the start, with the potentials held in FP64 and every vector of the Chebyshev recurrence held as
 * an FP32 mantissa with its own int32 binary exponent (each order's row sums align their terms to
 * the row's largest exponent by exact powers of two), so no value of the loop over- or underflows.
 * Result: the scalings of gs_sinkhorn as logarithms, and
 *     dist[0] = W^2 = 4t sum_i vol_i (a_i ln u_i + b_i ln v_i),   dist[1] = W = sqrt(W^2)
 * in FP64 (0 ln 0 := 0).  A fixed iteration count runs as one persistent launch (one launch per
 * Chebyshev order replayed from a CUDA graph with GS_OPT_LOOP 1, or where the graph has no
 * persistent partition); an eps stop runs one launch per order.  All arguments are in the
 * caller's node order.
 *   a, b   : [n] non-negative marginals of equal mass (device FP32; checked as in gs_sinkhorn)
 *   vol    : [n] vertex weights or NULL
 *   eps    : > 0 -> stop at the first iteration j, j a multiple of 10, whose marginal error
 *            sum_i |u_i (p_K(vol * v))_i - a_i| is below eps (computed in FP64 from the
 *            potentials; GS_ERR_NOT_CONVERGED at gs_sync if none); <= 0 -> exactly `iters`
 *   log_u, log_v : [n] double outputs (device), distinct buffers; -inf where a_i (b_i) = 0
 *   dist   : [2] double output (device), may be NULL
 *   iters_done : [1] int32 output (device), may be NULL
 * A non-positive p_K(vol * u)_i where the marginal is positive (the truncated series can dip below
 * zero) gives NaN there and GS_ERR_NONFINITE at gs_sync.  Requires t > 0, 1 <= K <= 10000,
 * iters >= 1.  Errors: GS_ERR_ARG. */
gs_status gs_sinkhorn_log(gs_ctx *ctx, const gs_graph *g, const float *a, const float *b,
                          const float *vol, double t, int K, double eps, int iters, double *log_u,
                          double *log_v, double *dist, int32_t *iters_done);

/* ---------------------------------------------------------------------------- barycenter --- */

/* Fixed-support Wasserstein barycenter (Sec. 3.3) by iterative Bregman projections with the
 * heat filter as kernel: v_i <- 1; repeat `iters` times { w_i <- mu_i / p_K(vol * v_i);
 * d_i <- v_i * p_K(vol * w_i); mu <- prod_i d_i^alpha_i; v_i <- v_i * mu / d_i }.  All m
 * distributions move through the filter as one [n, m] block; the geometric mean is a log-sum
 * accumulated in FP64 inside the last Chebyshev order.
 *   M      : [n, m] input distributions (column i is mu_i), non-negative, of equal mass
 *            sum(vol * mu_i) (not checked: with unequal masses the iteration has no fixed point
 *            and mu depends on `iters`); the barycenter keeps that mass
 *   alpha  : [m] double weights (device), >= 0, summing to 1 (checked on the device, see
 *            GS_OPT_CHECK_ARGS)
 *   vol    : [n] vertex weights or NULL
 *   mu     : [n] output barycenter
 *   v_state: [n, m] output scalings v_i after the last iteration, may be NULL
 * Requires 1 <= m <= 1024.  Errors: GS_ERR_ARG. */
gs_status gs_barycenter(gs_ctx *ctx, const gs_graph *g, const float *M, int m, const double *alpha,
                        const float *vol, double t, int K, int iters, float *mu, float *v_state);

/* Euler implicit heat kernel, the other approximation of H_t that Sec. 4 cites (backward Euler
 * with K steps, `(Id - (eps/4K) L)^{-K}` in the paper's sign convention for L):
 *     Y = (I + (t/K) L)^{-K} V,   L = I - D^{-1/2} A D^{-1/2},
 * each of the K steps a solve of the symmetric positive definite system (I + (t/K) L) x = b by
 * conjugate gradients from x = 0, all B columns at once, exactly `iters` iterations per step (a
 * column whose residual falls below tol |b| stops changing).  The condition number is at most
 * 1 + 2t/K.  For comparison with gs_heat_apply; not used by the Sinkhorn or barycenter calls.
 *   V, Y : [n, B] device FP32, row-major, caller's node order, no aliasing; 1 <= B <= 256
 * Scalars stay on the device: the call is asynchronous like the others.
 * Errors: GS_ERR_ARG. */
gs_status gs_heat_apply_implicit(gs_ctx *ctx, const gs_graph *g, double t, int K, const float *V, int B,
                                 float *Y, double tol, int iters);

/* ---------------------------------------------------------------- families of distributions --- */

/* Barycentric distance between two families of distributions (Definition 4.3):
 *     gamma(T, C) = W_{H_t}(mu*_T, mu*_C),
 * the Geodesic Sinkhorn distance (Algorithm 1, `sink_iters` iterations, as gs_distance) between
 * the barycenters of the two families (Sec. 3.3, `bary_iters` iterations each, as gs_barycenter).
 * Each barycenter is divided by its mass before the distance: the definition compares
 * distributions, and Algorithm 1 needs marginals of equal mass.
 *   MT, MC          : [n, mT] and [n, mC] device FP32, column i a member of the family
 *   alphaT, alphaC  : [mT], [mC] device FP64 weights (>= 0, summing to 1; checked on the device)
 *   vol             : [n] vertex weights or NULL (barycenters and distance alike)
 *   muT, muC        : [n] device FP32 outputs, the normalised barycenters (distinct buffers)
 *   dist            : [2] device FP64 output, (gamma^2, gamma) as gs_distance's (W^2, W)
 * Requires 1 <= mT, mC <= 1024 (as gs_barycenter), iterations >= 1.  A barycenter without
 * positive finite mass raises GS_ERR_NONFINITE at the next gs_sync.  Errors: GS_ERR_ARG,
 * GS_ERR_UNSUPPORTED. */
gs_status gs_barycentric_distance(gs_ctx *ctx, const gs_graph *g, const float *MT, int mT,
                                  const double *alphaT, const float *MC, int mC, const double *alphaC,
                                  const float *vol, double t, int K, int bary_iters, int sink_iters,
                                  float *muT, float *muC, double *dist);

/* Expected barycenter effect (Definition 4.4): tau = E_{mu*_T}[Y] - E_{mu*_C}[Y], the features'
 * expectations under the two barycenters, each measure divided by its mass (the closed form of
 * the definition: two weighted means).
 *   Y        : [n, d] device FP32 node features, row-major, in the graph's node numbering
 *   muT, muC : [n] device FP32 measures (e.g. gs_barycentric_distance's outputs)
 *   out      : [d] device FP64 output
 * Sums are FP64 in a fixed order.  A measure without positive finite mass raises
 * GS_ERR_NONFINITE at the next gs_sync.  Requires n >= 1, 1 <= d <= 65535.  Errors: GS_ERR_ARG. */
gs_status gs_barycenter_effect(gs_ctx *ctx, const float *Y, int64_t n, int d, const float *muT,
                               const float *muC, double *out);

/* ------------------------------------------------------------------------------ adjoint --- */

/* Reverse mode of Algorithm 1 unrolled over `iters` iterations (not in the paper; it serves
 * gradient-based use of the distance).  Runs the loop forward keeping the second scaling every
 * `checkpoint` iterations, then sweeps back segment by segment: each segment is recomputed from
 * its checkpoint with the filter values saved, and the transposed filter applies reuse the same
 * fused kernels because p_K(L, t) is symmetric.  Outputs
 *     dist[0..1] (device doubles) = W^2, W            (as gs_sinkhorn)
 *     grad_a, grad_b [n] (device)  = dW^2/da, dW^2/db  (of the unrolled map, a and b independent;
 *                                                       entries with zero mass use 0 ln 0 := 0)
 * Marginals are checked as in gs_sinkhorn.  Requires checkpoint >= 1.  Errors: GS_ERR_ARG. */
gs_status gs_sinkhorn_grad(gs_ctx *ctx, const gs_graph *g, const float *a, const float *b,
                           const float *vol, double t, int K, int iters, int checkpoint,
                           double *dist, float *grad_a, float *grad_b);

/* Reverse mode of gs_barycenter (Sec. 3.3) unrolled over `iters` iterations: given mubar [n]
 * (device), the adjoint of the returned barycenter, writes mu [n] (the barycenter, may be NULL)
 * and grad_alpha [m] (device doubles) = d<mubar, mu>/dalpha.  Checkpoints of the scalings every
 * `checkpoint` iterations bound the tape to `checkpoint` iterations of [n, m] blocks.
 * Same limits as gs_barycenter.  Errors: GS_ERR_ARG, GS_ERR_UNSUPPORTED. */
gs_status gs_barycenter_grad(gs_ctx *ctx, const gs_graph *g, const float *M, int m,
                             const double *alpha, const float *vol, double t, int K, int iters,
                             int checkpoint, const float *mubar, float *mu, double *grad_alpha);

/* ------------------------------------------------------------------------------ batched --- */

/* Many independent Algorithm 1 problems in one persistent launch (the batching is not in the
 * paper; it serves workloads with many small distances). Problem i has graph graphs[i] (any size,
 * any order), marginals a[i], b[i] (device [n_i]; checked as in gs_sinkhorn), diffusion time t[i] and degree K[i]; all run
 * `iters` iterations with unit vertex weights. Outputs u[i], v[i] (device [n_i]) and dist[2i],
 * dist[2i+1] (device doubles: W^2, W). `graphs`, `a`, `b`, `t`, `K`, `u`, `v` are HOST arrays of
 * length nprob. Each problem runs on one thread-block cluster whose Chebyshev orders are separated
 * by hardware cluster barriers. Requires 1 <= nprob, every K[i] >= 1, t[i] > 0. Errors:
 * GS_ERR_ARG. */
gs_status gs_sinkhorn_batched(gs_ctx *ctx, int nprob, const gs_graph *const *graphs,
                              const float *const *a, const float *const *b, const double *t,
                              const int *K, int iters, float *const *u, float *const *v,
                              double *dist);

#ifdef __cplusplus
}
#endif

#endif /* GEOSINK_H */
