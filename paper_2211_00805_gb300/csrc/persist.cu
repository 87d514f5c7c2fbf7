// Persistent form of the Sinkhorn loop (Algorithm 1) for one problem with one right-hand side.
//
// The fixed-count loop is 2 K iters Chebyshev orders; each order is a few microseconds of work
// when the graph is L2-resident, so separate launches spend most of their time starting and
// draining.  Here one cooperative launch (every block resident, guaranteed by the runtime) runs
// the whole loop: each block owns a contiguous slice of rows, and a grid barrier separates the
// orders.  The barrier is a counter plus a generation word in global memory; every wait is
// bounded by a clock budget, after which the block records GS_FLAG_TIMEOUT and the whole grid
// leaves the loop (each block's own wait runs out too), so a fault can never leave the GPU
// spinning.  Per row the arithmetic is the fused order of cheb.cu: gather through the CSR row,
// update T_k in place and the running sum, and in the last order divide the marginal by the
// filter value and write the next filter input vol * u.
//
// Buffers written by other blocks are read with ordinary (coherent) loads after the barrier; only
// the graph, which never changes during the kernel, goes through the read-only path.
#include <cuda/atomic>

#include <algorithm>

#include "cache_slices.cuh"
#include <type_traits>

#include "gs_internal.cuh"
#include "sell_row.cuh"

namespace {

constexpr int kThreads = 1024;
constexpr int kReadyStride = 32;  // one 128-byte line per block's ready counter
constexpr long long kBarrierBudget = 4000000000ll;  // clock cycles (~2 s) before giving up
// Self-test: the barrier waits for one arrival more than the grid has, so every wait runs out
// after this much shorter budget and the launch ends with GS_FLAG_TIMEOUT.
constexpr long long kSelfTestBudget = 20000000ll;

struct PersistArgs {
    int n;
    const int* rowptr;
    const int* col;
    const float* pval;
    const int* sptr;     // sliced ELL, or null (then the CSR row-split mapping is used)
    const int* scol;
    const float* sval;
    const float* a;
    const float* b;
    const float* vol;
    float* x;
    float* A;
    float* y;
    float* u;
    float* v;
    const float* coef;   // [K + 1] device
    int K;
    int iters;
    unsigned* bar;       // [0] arrivals, [1] generation
    int* flags;
    unsigned expect;     // arrivals that release a barrier (gridDim.x; one more in the self-test)
    long long budget;    // clock cycles a block waits at a barrier before giving up
    int rows_per_block;  // whole slices
    int smem_graph;      // 1: each block's slices of the sliced ELL are copied to shared memory once
                         // 2: values + 16-bit local column indices + the per-block gather cache
    const int* xc_rows;  // smem_graph == 2: block b owns rows [xc_rows[b], xc_rows[b+1])
    const int* xc_ucol;  // gather cache tables (smem_graph == 2)
    const int* xc_ucnt;
    const uint16_t* xc_lidx;
    int xc_max_e;
    int xc_max_u;
    const int* xc_deps;  // [gridDim.x][gridDim.x] blocks each block reads from (neighbour-flag sync)
    const int* xc_ndeps;
    unsigned* ready;     // [gridDim.x * kReadyStride] per-block count of published stages
    int selftest;        // neighbour-flag sync: wait for one stage more than will ever be published
    unsigned long long* tagged;  // [3][n] (value, stage + 1) words, zeroed (tagged-value sync)
};

// Returns false when the wait ran out (the caller leaves the loop).  Arrival is a relaxed atomic
// increment after a release fence; the last arriver resets the counter and bumps the generation
// with release semantics; waiters poll the generation with acquire loads, bounded by `budget`.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* flags, int* s_ok, unsigned expect,
                                             long long budget)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(bar[0]);
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> gen(bar[1]);
        const unsigned g = gen.load(cuda::memory_order_relaxed);
        cuda::atomic_thread_fence(cuda::memory_order_release, cuda::thread_scope_device);
        if (cnt.fetch_add(1u, cuda::memory_order_relaxed) == expect - 1) {
            cnt.store(0u, cuda::memory_order_relaxed);
            gen.fetch_add(1u, cuda::memory_order_release);
        } else {
            const long long t0 = clock64();
            while (gen.load(cuda::memory_order_acquire) == g) {
                if (clock64() - t0 > budget) {
                    atomicOr(flags, GS_FLAG_TIMEOUT);
                    *s_ok = 0;
                    break;
                }
            }
        }
        cuda::atomic_thread_fence(cuda::memory_order_acquire, cuda::thread_scope_device);
    }
    __syncthreads();
    return *s_ok != 0;
}

// Row functions: mode 0 is the first order (T_1 = P x, y = c_0 x + c_1 T_1), 1 a middle order, 2
// the last order (divide the marginal by the filter value, write the next input vol * u), 3 the
// only order when K = 1 (first and last at once).
template <int G>
__device__ __forceinline__ void rows_order(const PersistArgs& p, int r0, int r1, int mode, float ck,
                                           float c0, const float* cur, const float* prev,
                                           float* next, const float* num, float* out, float* xnext)
{
    const int lane = threadIdx.x & (G - 1);
    const int rows_per_pass = kThreads / G;
    for (int base = r0; base < r1; base += rows_per_pass) {
        const int row = base + (int)threadIdx.x / G;
        const bool active = row < r1;
        float s = 0.f;
        if (active) {
            const int beg = __ldg(p.rowptr + row), end = __ldg(p.rowptr + row + 1);
            int e = beg + lane;
            for (; e + G < end; e += 2 * G) {
                const int j0 = __ldg(p.col + e), j1 = __ldg(p.col + e + G);
                const float w0 = __ldg(p.pval + e), w1 = __ldg(p.pval + e + G);
                s = fmaf(w0, cur[j0], s);
                s = fmaf(w1, cur[j1], s);
            }
            if (e < end) s = fmaf(__ldg(p.pval + e), cur[__ldg(p.col + e)], s);
        }
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (!active || lane != 0) continue;
        const bool first = mode == 0 || mode == 3;
        const float tk = first ? s : fmaf(2.f, s, -prev[row]);
        const float acc = first ? fmaf(ck, tk, c0 * cur[row]) : fmaf(ck, tk, p.y[row]);
        if (mode < 2) {
            next[row] = tk;
            p.y[row] = acc;
        } else {
            const float m = num[row];
            float r = 0.f;
            if (m != 0.f) {
                r = m / acc;
                if (!(r > 0.f) || isinf(r)) atomicOr(p.flags, GS_FLAG_NONFINITE);
            }
            out[row] = r;
            xnext[row] = p.vol ? p.vol[row] * r : r;
        }
    }
}

// Thread-per-row variant over the sliced ELL copy (same arithmetic as the per-order kernel, so
// both loop modes give identical results).
__device__ __forceinline__ void rows_order_sell(const PersistArgs& p, int r0, int r1, int mode,
                                                float ck, float c0, const float* cur,
                                                const float* prev, float* next, const float* num,
                                                float* out, float* xnext)
{
    for (int row = r0 + (int)threadIdx.x; row < r1; row += kThreads) {
        const bool first = mode == 0 || mode == 3;
        const float pv = first ? 0.f : prev[row];
        const float yv = first ? c0 * cur[row] : p.y[row];
        const float s = gs_sell_row<false>(p.sptr, p.scol, p.sval, cur, row);
        const float tk = first ? s : fmaf(2.f, s, -pv);
        const float acc = fmaf(ck, tk, yv);
        if (mode < 2) {
            next[row] = tk;
            p.y[row] = acc;
        } else {
            const float m = num[row];
            float r = 0.f;
            if (m != 0.f) {
                r = m / acc;
                if (!(r > 0.f) || isinf(r)) atomicOr(p.flags, GS_FLAG_NONFINITE);
            }
            out[row] = r;
            xnext[row] = p.vol ? p.vol[row] * r : r;
        }
    }
}

// Same rows and arithmetic with the block's sliced-ELL entries resident in shared memory
// (scol_s / sval_s hold entries [e0, e0 + count) of the global arrays).
__device__ __forceinline__ void rows_order_sell_smem(const PersistArgs& p, int r0, int r1, int mode,
                                                     float ck, float c0, const float* cur,
                                                     const float* prev, float* next,
                                                     const float* num, float* out, float* xnext,
                                                     const int* scol_s, const float* sval_s, int e0)
{
    for (int row = r0 + (int)threadIdx.x; row < r1; row += kThreads) {
        const bool first = mode == 0 || mode == 3;
        const float pv = first ? 0.f : prev[row];
        const float yv = first ? c0 * cur[row] : p.y[row];
        const int sl = row / GS_SELL_C;
        const int beg = __ldg(p.sptr + sl);
        const int width = (__ldg(p.sptr + sl + 1) - beg) / GS_SELL_C;
        const int off = beg - e0 + row % GS_SELL_C;
        const float s = gs_sell_dot<false, false>(scol_s + off, sval_s + off, width, cur);
        const float tk = first ? s : fmaf(2.f, s, -pv);
        const float acc = fmaf(ck, tk, yv);
        if (mode < 2) {
            next[row] = tk;
            p.y[row] = acc;
        } else {
            const float m = num[row];
            float r = 0.f;
            if (m != 0.f) {
                r = m / acc;
                if (!(r > 0.f) || isinf(r)) atomicOr(p.flags, GS_FLAG_NONFINITE);
            }
            out[row] = r;
            xnext[row] = p.vol ? p.vol[row] * r : r;
        }
    }
}

// Rows with values and local column indices in shared memory and the neighbour values in the
// block's gather cache xc (filled from cur at the start of the order).
__device__ __forceinline__ void rows_order_cached(const PersistArgs& p, int r0, int r1, int mode,
                                                  float ck, float c0, const float* cur,
                                                  const float* prev, float* next, const float* num,
                                                  float* out, float* xnext, const uint16_t* lidx_s,
                                                  const float* sval_s, const float* xc, int e0)
{
    for (int row = r0 + (int)threadIdx.x; row < r1; row += kThreads) {
        const bool first = mode == 0 || mode == 3;
        const float pv = first ? 0.f : prev[row];
        const float yv = first ? c0 * cur[row] : p.y[row];
        const int sl = row / GS_SELL_C;
        const int beg = __ldg(p.sptr + sl);
        const int width = (__ldg(p.sptr + sl + 1) - beg) / GS_SELL_C;
        const int r = row % GS_SELL_C;
        const float s = gs_sell_dot_cached(lidx_s + (beg - e0), r, sval_s + (beg - e0) + r, width, xc);
        const float tk = first ? s : fmaf(2.f, s, -pv);
        const float acc = fmaf(ck, tk, yv);
        if (mode < 2) {
            next[row] = tk;
            p.y[row] = acc;
        } else {
            const float m = num[row];
            float r = 0.f;
            if (m != 0.f) {
                r = m / acc;
                if (!(r > 0.f) || isinf(r)) atomicOr(p.flags, GS_FLAG_NONFINITE);
            }
            out[row] = r;
            xnext[row] = p.vol ? p.vol[row] * r : r;
        }
    }
}

template <int G>
__device__ __forceinline__ void rows_any(const PersistArgs& p, int r0, int r1, int mode, float ck,
                                         float c0, const float* cur, const float* prev, float* next,
                                         const float* num, float* out, float* xnext,
                                         const int* scol_s = nullptr, const float* sval_s = nullptr,
                                         int e0 = 0, const uint16_t* lidx_s = nullptr,
                                         const int* ucol_s = nullptr, float* xc = nullptr, int ucnt = 0)
{
    if (lidx_s) {
        // stage the block's gather cache from T_{k-1}, then the rows read it from shared memory
        for (int i = threadIdx.x; i < ucnt; i += kThreads) xc[i] = cur[ucol_s[i]];
        __syncthreads();
        rows_order_cached(p, r0, r1, mode, ck, c0, cur, prev, next, num, out, xnext, lidx_s, sval_s, xc, e0);
    } else if (scol_s) rows_order_sell_smem(p, r0, r1, mode, ck, c0, cur, prev, next, num, out, xnext, scol_s, sval_s, e0);
    else if (p.sptr) rows_order_sell(p, r0, r1, mode, ck, c0, cur, prev, next, num, out, xnext);
    else rows_order<G>(p, r0, r1, mode, ck, c0, cur, prev, next, num, out, xnext);
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* mbar)
{
    gs_bulk_g2s(dst, src, bytes, mbar);
}

// Mode 2: values, local column indices and the distinct-column list of this block into shared
// memory with three bulk copies on one mbarrier (bounded wait).
__device__ bool load_cached_slices(const PersistArgs& p, int r0, int r1, float* sval_s,
                                   uint16_t* lidx_s, int* ucol_s, int* e0_out, int* ucnt_out,
                                   unsigned long long* mbar)
{
    bool timed_out = false;
    const bool ok = gs_load_cache_tables(p.sptr, p.sval, p.xc_lidx, p.xc_ucol, p.xc_ucnt, (int)blockIdx.x, r0, r1,
                                         p.budget, sval_s, lidx_s, ucol_s, e0_out, ucnt_out, mbar, &timed_out);
    if (timed_out) atomicOr(p.flags, GS_FLAG_TIMEOUT);
    return ok;
}

// Load this block's sliced-ELL entries into shared memory with two bulk copies tracked by one
// mbarrier transaction count.  The wait is bounded; false = it ran out (GS_FLAG_TIMEOUT set).
__device__ bool load_graph_slices(const PersistArgs& p, int r0, int r1, int* scol_s, float* sval_s,
                                  int* e0_out, unsigned long long* mbar)
{
    const int s0 = r0 / GS_SELL_C;
    const int s1 = (r1 + GS_SELL_C - 1) / GS_SELL_C;
    const int e0 = __ldg(p.sptr + s0);
    const int e1 = (r1 > r0) ? __ldg(p.sptr + s1) : e0;
    *e0_out = e0;
    const unsigned bytes = (unsigned)(e1 - e0) * 4u;  // a multiple of 128: slices are 32 x 4 bytes wide
    if (bytes == 0) return true;
    const unsigned m = (unsigned)__cvta_generic_to_shared(mbar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(m) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(m), "r"(2u * bytes)
                     : "memory");
        bulk_g2s(scol_s, p.scol + e0, bytes, mbar);
        bulk_g2s(sval_s, p.sval + e0, bytes, mbar);
    }
    const long long t0 = clock64();
    unsigned done = 0;
    while (!done) {
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], 0;\n"
            " selp.u32 %0, 1, 0, P;\n}\n"
            : "=r"(done)
            : "r"(m)
            : "memory");
        if (!done && clock64() - t0 > p.budget) {
            atomicOr(p.flags, GS_FLAG_TIMEOUT);
            return false;
        }
    }
    return true;
}

template <int G>
__global__ void __launch_bounds__(kThreads) sinkhorn_persistent(const PersistArgs p)
{
    __shared__ int s_ok;
    __shared__ __align__(8) unsigned long long s_mbar;
    extern __shared__ __align__(128) unsigned char p_smem[];
    if (threadIdx.x == 0) s_ok = 1;
    __syncthreads();
    const int per = p.rows_per_block;
    const int r0 = p.smem_graph == 2 ? __ldg(p.xc_rows + blockIdx.x) : min(p.n, (int)blockIdx.x * per);
    const int r1 = p.smem_graph == 2 ? __ldg(p.xc_rows + blockIdx.x + 1) : min(p.n, r0 + per);
    int e0 = 0, ucnt = 0;
    int* scol_s = nullptr;
    float* sval_s = nullptr;
    uint16_t* lidx_s = nullptr;
    int* ucol_s = nullptr;
    float* xc = nullptr;
    if (p.smem_graph == 2) {
        const int emax = (p.xc_max_e + 31) / 32 * 32, umax = (p.xc_max_u + 31) / 32 * 32;
        sval_s = reinterpret_cast<float*>(p_smem);
        lidx_s = reinterpret_cast<uint16_t*>(p_smem + (size_t)emax * 4);
        ucol_s = reinterpret_cast<int*>(p_smem + (size_t)emax * 6);
        xc = reinterpret_cast<float*>(p_smem + (size_t)emax * 6 + (size_t)umax * 4);
        if (!load_cached_slices(p, r0, r1, sval_s, lidx_s, ucol_s, &e0, &ucnt, &s_mbar)) s_ok = 0;
        __syncthreads();
        if (!s_ok) return;
    } else if (p.smem_graph) {
        const int cap = (__ldg(p.sptr + min((r0 + per + GS_SELL_C - 1) / GS_SELL_C, (p.n + GS_SELL_C - 1) / GS_SELL_C)) -
                         __ldg(p.sptr + r0 / GS_SELL_C));
        scol_s = reinterpret_cast<int*>(p_smem);
        sval_s = reinterpret_cast<float*>(p_smem + (size_t)((cap + 31) / 32 * 32) * 4);
        if (!load_graph_slices(p, r0, r1, scol_s, sval_s, &e0, &s_mbar)) s_ok = 0;
        __syncthreads();
        if (!s_ok) return;
    }
    for (int r = r0 + threadIdx.x; r < r1; r += kThreads) p.x[r] = p.vol ? p.vol[r] : 1.f;
    if (!grid_barrier(p.bar, p.flags, &s_ok, p.expect, p.budget)) return;
    float* X = p.x;
    float* Ab = p.A;
    const float c0 = p.coef[0];
    for (int it = 0; it < p.iters; ++it) {
        for (int h = 0; h < 2; ++h) {
            const float* num = h == 0 ? p.a : p.b;
            float* out = h == 0 ? p.u : p.v;
            if (p.K == 1) {
                rows_any<G>(p, r0, r1, 3, p.coef[1], c0, X, nullptr, nullptr, num, out, Ab, scol_s, sval_s, e0, lidx_s, ucol_s, xc, ucnt);
                if (!grid_barrier(p.bar, p.flags, &s_ok, p.expect, p.budget)) return;
                float* t = X; X = Ab; Ab = t;
                continue;
            }
            rows_any<G>(p, r0, r1, 0, p.coef[1], c0, X, nullptr, Ab, nullptr, nullptr, nullptr, scol_s, sval_s, e0, lidx_s, ucol_s, xc, ucnt);
            if (!grid_barrier(p.bar, p.flags, &s_ok, p.expect, p.budget)) return;
            float* prev = X;
            float* cur = Ab;
            for (int k = 2; k <= p.K; ++k) {
                if (k < p.K) {
                    rows_any<G>(p, r0, r1, 1, p.coef[k], 0.f, cur, prev, prev, nullptr, nullptr, nullptr, scol_s, sval_s, e0, lidx_s, ucol_s, xc, ucnt);
                    if (!grid_barrier(p.bar, p.flags, &s_ok, p.expect, p.budget)) return;
                    float* t = prev; prev = cur; cur = t;
                } else {
                    rows_any<G>(p, r0, r1, 2, p.coef[k], 0.f, cur, prev, nullptr, num, out, prev, scol_s, sval_s, e0, lidx_s, ucol_s, xc, ucnt);
                    if (!grid_barrier(p.bar, p.flags, &s_ok, p.expect, p.budget)) return;
                    X = prev;
                    Ab = cur;
                }
            }
        }
    }
}


// ------------------------------------------------------------------ neighbour-flag variant
// Same loop, same arithmetic as mode 2 above, with two changes.  (1) Each block keeps the
// recurrence values of its own rows (T_{k-1}, T_{k-2}, the running sum, the input x and the
// marginals) in registers, since no other block reads them; only T_k (or, after the last order,
// the next input vol * u) is published, alternately into one of two global slots.  (2) Instead of
// a barrier over the grid, block b waits before each order only for the blocks that own a column
// of its rows: "stage s published" is a per-block counter ready[b] = s + 1 written with release
// semantics after the stage's stores.  Order s reads stage s-1 from slot (s-1) & 1 and writes stage
// s into slot s & 1, which held stage s-2; waiting for ready[d] >= s on every block d it reads
// covers both the read of stage s-1 and, the operator being symmetric, the end of every read of
// stage s-2 from this block's rows (block d read it in order s-1, before publishing stage s-1).
// Every wait is bounded by the clock budget.

// Wait until every block this one reads from has published stage `need - 1`.  Bounded; false =
// the wait ran out (GS_FLAG_TIMEOUT set).
__device__ __forceinline__ bool wait_neighbours(const PersistArgs& p, int dep, unsigned need,
                                                int* s_ok)
{
    if (dep >= 0) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> f(p.ready[dep * kReadyStride]);
        if (f.load(cuda::memory_order_relaxed) < need) {
            const long long t0 = clock64();
            while (f.load(cuda::memory_order_relaxed) < need) {
                if (clock64() - t0 > p.budget) {
                    atomicOr(p.flags, GS_FLAG_TIMEOUT);
                    *s_ok = 0;
                    break;
                }
            }
        }
        cuda::atomic_thread_fence(cuda::memory_order_acquire, cuda::thread_scope_device);
    }
    __syncthreads();
    return *s_ok != 0;
}

// All of this block's stores of stage s are done: publish ready[b] = s + 1.
__device__ __forceinline__ void publish(const PersistArgs& p, unsigned stage)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        cuda::atomic_thread_fence(cuda::memory_order_release, cuda::thread_scope_device);
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> f(p.ready[blockIdx.x * kReadyStride]);
        f.store(stage + 1u, cuda::memory_order_relaxed);
    }
}

template <int RPT, int NT>
__global__ void __launch_bounds__(NT) sinkhorn_neighbour_sync(const PersistArgs p)
{
    __shared__ int s_ok;
    __shared__ __align__(8) unsigned long long s_mbar;
    extern __shared__ __align__(128) unsigned char p_smem[];
    if (threadIdx.x == 0) s_ok = 1;
    __syncthreads();
    const int r0 = __ldg(p.xc_rows + blockIdx.x), r1 = __ldg(p.xc_rows + blockIdx.x + 1);
    const int emax = (p.xc_max_e + 31) / 32 * 32, umax = (p.xc_max_u + 31) / 32 * 32;
    float* sval_s = reinterpret_cast<float*>(p_smem);
    uint16_t* lidx_s = reinterpret_cast<uint16_t*>(p_smem + (size_t)emax * 4);
    int* ucol_s = reinterpret_cast<int*>(p_smem + (size_t)emax * 6);
    float* xc = reinterpret_cast<float*>(p_smem + (size_t)emax * 6 + (size_t)umax * 4);
    int e0 = 0, ucnt = 0;
    if (!load_cached_slices(p, r0, r1, sval_s, lidx_s, ucol_s, &e0, &ucnt, &s_mbar)) s_ok = 0;
    __syncthreads();
    if (!s_ok) return;
    if (r0 >= r1 && !p.selftest) return;  // no rows: no block reads from this one

    // the block this thread waits on (one per thread; a self-test waits for its own block too)
    const int nd = __ldg(p.xc_ndeps + blockIdx.x);
    int dep = (int)threadIdx.x < nd ? __ldg(p.xc_deps + (int64_t)blockIdx.x * gridDim.x + threadIdx.x) : -1;
    if (p.selftest && (int)threadIdx.x == nd) dep = (int)blockIdx.x;
    const unsigned extra = p.selftest ? 1u : 0u;

    // own rows: sliced-ELL position, marginals, volume, recurrence state
    int off[RPT], width[RPT];
    float av[RPT], bv[RPT], vv[RPT], xo[RPT], t1[RPT], t2[RPT], yo[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int row = r0 + (int)threadIdx.x + j * NT;
        off[j] = 0;
        width[j] = 0;
        av[j] = bv[j] = 0.f;
        vv[j] = 1.f;
        if (row < r1) {
            const int sl = row / GS_SELL_C;
            const int beg = __ldg(p.sptr + sl);
            width[j] = (__ldg(p.sptr + sl + 1) - beg) / GS_SELL_C;
            off[j] = beg - e0 + row % GS_SELL_C;
            av[j] = __ldg(p.a + row);
            bv[j] = __ldg(p.b + row);
            if (p.vol) vv[j] = __ldg(p.vol + row);
        }
        xo[j] = vv[j];  // vol * (v = 1)
        t1[j] = t2[j] = yo[j] = 0.f;
    }
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int row = r0 + (int)threadIdx.x + j * NT;
        if (row < r1) p.x[row] = xo[j];
    }
    unsigned stage = 0;
    publish(p, stage);
    const float c0 = p.coef[0];
    const int K = p.K;
    for (int it = 0; it < p.iters; ++it) {
        for (int h = 0; h < 2; ++h) {
            for (int k = 1; k <= K; ++k) {
                ++stage;
                if (!wait_neighbours(p, dep, stage + extra, &s_ok)) return;
                const float* src = (stage & 1) ? p.x : p.A;  // stage s - 1 lives in slot (s - 1) & 1
                float* dst = (stage & 1) ? p.A : p.x;
                for (int i = threadIdx.x; i < ucnt; i += NT) xc[i] = __ldcg(src + ucol_s[i]);
                __syncthreads();
                const float ck = p.coef[k];
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const int row = r0 + (int)threadIdx.x + j * NT;
                    if (row >= r1) continue;
                    const float s = gs_sell_dot_cached(lidx_s + off[j] - (threadIdx.x & (GS_SELL_C - 1)),
                                                       threadIdx.x & (GS_SELL_C - 1), sval_s + off[j], width[j], xc);
                    float tk, acc;
                    if (k == 1) {
                        tk = s;
                        acc = fmaf(ck, tk, c0 * xo[j]);
                    } else {
                        tk = fmaf(2.f, s, -t2[j]);
                        acc = fmaf(ck, tk, yo[j]);
                    }
                    if (k < K) {
                        t2[j] = k == 1 ? xo[j] : t1[j];
                        t1[j] = tk;
                        yo[j] = acc;
                        dst[row] = tk;
                    } else {
                        const float m = h == 0 ? av[j] : bv[j];
                        float r = 0.f;
                        if (m != 0.f) {
                            r = m / acc;
                            if (!(r > 0.f) || isinf(r)) atomicOr(p.flags, GS_FLAG_NONFINITE);
                        }
                        (h == 0 ? p.u : p.v)[row] = r;
                        xo[j] = p.vol ? vv[j] * r : r;
                        dst[row] = xo[j];
                    }
                }
                publish(p, stage);
            }
        }
    }
}

// ------------------------------------------------------------------ tagged-value variant
// Same loop and arithmetic again, with the readiness carried by the data itself: every published
// value is one 64-bit word (FP32 bits low, stage + 1 high), written and read as a single-copy-
// atomic 64-bit access, into one of three slots (stage s in slot s mod 3; the slots are zeroed
// before the launch, so a tag of 0 is never a stage).  The default 4-byte form (W4) halves the
// exchanged bytes, which is what the staging is bound by (scattered loads, one cache line per
// few values): the tag is the stage parity in the value's last mantissa bit.  A block reading stage s - 1 simply re-reads
// any word whose tag is not yet s: no counters, no fences, and no barrier of any kind between
// blocks.  Three slots make the overwrite safe: the block writing stage s into a slot (which held
// stage s - 3) has read stage s - 1 from every block it reads from, and each of those blocks had
// finished reading stage s - 3 (in order s - 2) before it computed stage s - 1.  Should a value
// ever be overwritten early anyway, its reader would find a tag other than the one it waits for
// and its bounded wait would run out (GS_FLAG_TIMEOUT), never a silently wrong value.

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* a)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* a, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;\n" ::"l"(a), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long pack_tagged(float x, unsigned tag)
{
    return ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(x);
}


// 4-byte exchange words: the FP32 value with its last mantissa bit replaced by the stage parity
// (at most one unit in the last place on the values other blocks read; the owner keeps the exact
// value in registers).  Three slots still tell a stale word (stage s - 4) from the wanted one
// (s - 1): their parities differ, and so does an early overwrite (s + 2).
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* a)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u32(unsigned* a, unsigned v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;\n" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned pack_tag32(float x, unsigned parity)
{
    return (__float_as_uint(x) & ~1u) | parity;
}
template <bool W4>
__device__ __forceinline__ unsigned tag_of(unsigned long long w)
{
    return W4 ? (unsigned)(w & 1ull) : (unsigned)(w >> 32);
}

// A row's first WR steps of the sliced ELL held in registers for the whole loop (the operator does
// not change between orders): values wv[t], and local cache indices paired two steps to a word as
// in the shared-memory table (an odd last step alone in the low half).  Loaded once per launch.
template <int WR>
__device__ __forceinline__ void load_row_regs(const uint16_t* slice_lidx, int r, const float* vp, int width,
                                              float (&wv)[WR], unsigned (&lp)[WR / 2])
{
    const uint32_t* lp2 = reinterpret_cast<const uint32_t*>(slice_lidx) + r;
#pragma unroll
    for (int q = 0; q < WR / 2; ++q) {
        const int t = 2 * q;
        unsigned pr = 0u;
        if (t + 1 < width) pr = lp2[q * GS_SELL_C];
        else if (t < width) pr = (unsigned)slice_lidx[t * GS_SELL_C + r];
        lp[q] = pr;
        wv[t] = t < width ? vp[t * GS_SELL_C] : 0.f;
        wv[t + 1] = t + 1 < width ? vp[(t + 1) * GS_SELL_C] : 0.f;
    }
}

// The cached row sum of gs_sell_dot_cached (same products, same two accumulators, same order:
// blocks of eight steps, then pairs, then an odd last step) with steps below WR taken from
// registers and only the neighbour values read from shared memory there.  Every branch depends
// on the slice width alone, so it is uniform across the warp.
template <int WR>
__device__ __forceinline__ float row_dot_regs(const float (&wv)[WR], const unsigned (&lp)[WR / 2],
                                              const uint16_t* slice_lidx, int r, const float* vp, int width,
                                              const float* xc)
{
    static_assert(WR % 8 == 0, "register steps come in blocks of eight");
    const uint32_t* lp2 = reinterpret_cast<const uint32_t*>(slice_lidx) + r;
    const int full8 = width & ~7;
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int jb = 0; jb < WR; jb += 8) {
        if (jb < full8) {
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                const unsigned pr = lp[(jb + u) >> 1];
                s0 = fmaf(wv[jb + u], xc[pr & 0xffffu], s0);
                s1 = fmaf(wv[jb + u + 1], xc[pr >> 16], s1);
            }
        }
    }
    int j = WR;
    for (; j + 8 <= width; j += 8) {
        float w[8], x[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const unsigned pr = lp2[((j >> 1) + q) * GS_SELL_C];
            w[2 * q] = vp[(j + 2 * q) * GS_SELL_C];
            w[2 * q + 1] = vp[(j + 2 * q + 1) * GS_SELL_C];
            x[2 * q] = xc[pr & 0xffffu];
            x[2 * q + 1] = xc[pr >> 16];
        }
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            s0 = fmaf(w[u], x[u], s0);
            s1 = fmaf(w[u + 1], x[u + 1], s1);
        }
    }
    if (full8 < WR) {  // the tail (under eight steps) lies in registers: pairs, then an odd step
#pragma unroll
        for (int t = 0; t + 2 <= WR; t += 2)
            if (t >= full8 && t + 2 <= width) {
                const unsigned pr = lp[t >> 1];
                s0 = fmaf(wv[t], xc[pr & 0xffffu], s0);
                s0 = fmaf(wv[t + 1], xc[pr >> 16], s0);
            }
#pragma unroll
        for (int t = 0; t < WR; t += 2)
            if ((width & 1) && t + 1 == width) s0 = fmaf(wv[t], xc[lp[t >> 1] & 0xffffu], s0);
    } else {
        j = full8;
        for (; j + 2 <= width; j += 2) {
            const unsigned pr = lp2[(j >> 1) * GS_SELL_C];
            s0 = fmaf(vp[j * GS_SELL_C], xc[pr & 0xffffu], s0);
            s0 = fmaf(vp[(j + 1) * GS_SELL_C], xc[pr >> 16], s0);
        }
        if (j < width) s0 = fmaf(vp[j * GS_SELL_C], xc[slice_lidx[j * GS_SELL_C + r]], s0);
    }
    return s0 + s1;
}

template <int RPT, int NT, bool W4, bool GROUP, int WR = 0, int UL = 8>
__global__ void __launch_bounds__(NT) sinkhorn_tagged(const PersistArgs p)
{
    __shared__ int s_ok;
    __shared__ __align__(8) unsigned long long s_mbar;
    extern __shared__ __align__(128) unsigned char p_smem[];
    if (threadIdx.x == 0) s_ok = 1;
    __syncthreads();
    const int r0 = __ldg(p.xc_rows + blockIdx.x), r1 = __ldg(p.xc_rows + blockIdx.x + 1);
    const int emax = (p.xc_max_e + 31) / 32 * 32, umax = (p.xc_max_u + 31) / 32 * 32;
    float* sval_s = reinterpret_cast<float*>(p_smem);
    uint16_t* lidx_s = reinterpret_cast<uint16_t*>(p_smem + (size_t)emax * 4);
    int* ucol_s = reinterpret_cast<int*>(p_smem + (size_t)emax * 6);
    float* xc = reinterpret_cast<float*>(p_smem + (size_t)emax * 6 + (size_t)umax * 4);
    int e0 = 0, ucnt = 0;
    if (!load_cached_slices(p, r0, r1, sval_s, lidx_s, ucol_s, &e0, &ucnt, &s_mbar)) s_ok = 0;
    __syncthreads();
    if (!s_ok) return;
    if (r0 >= r1) return;  // no rows: nothing to publish, nothing to read
    const unsigned extra = p.selftest ? 1u : 0u;
    const size_t n = (size_t)p.n;
    unsigned* tw = reinterpret_cast<unsigned*>(p.tagged);

    int off[RPT], width[RPT];
    float av[RPT], bv[RPT], vv[RPT], xo[RPT], t1[RPT], t2[RPT], yo[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int row = r0 + (int)threadIdx.x + j * NT;
        off[j] = 0;
        width[j] = 0;
        av[j] = bv[j] = 0.f;
        vv[j] = 1.f;
        if (row < r1) {
            const int sl = row / GS_SELL_C;
            const int beg = __ldg(p.sptr + sl);
            width[j] = (__ldg(p.sptr + sl + 1) - beg) / GS_SELL_C;
            off[j] = beg - e0 + row % GS_SELL_C;
            av[j] = __ldg(p.a + row);
            bv[j] = __ldg(p.b + row);
            if (p.vol) vv[j] = __ldg(p.vol + row);
        }
        xo[j] = vv[j];  // vol * (v = 1)
        t1[j] = t2[j] = yo[j] = 0.f;
        if (row < r1) {  // stage 0, slot 0
            if (W4) st_relaxed_u32(tw + row, pack_tag32(xo[j], 0u));
            else st_relaxed_u64(p.tagged + row, pack_tagged(xo[j], 1u));
        }
    }
    static_assert(WR == 0 || RPT == 1, "register-resident rows: one row per thread");
    using Word = typename std::conditional<W4, unsigned, unsigned long long>::type;  // an exchange word
    constexpr int WRA = WR > 0 ? WR : 8;
    float wv[WRA];
    unsigned lp[WRA / 2];
    if (WR > 0)
        load_row_regs<WRA>(lidx_s + off[0] - (threadIdx.x & (GS_SELL_C - 1)), threadIdx.x & (GS_SELL_C - 1),
                           sval_s + off[0], width[0], wv, lp);
    unsigned stage = 0;
    int rslot = 0, wslot = 1;  // slots of stage - 1 and stage (mod 3) inside the order loop
    const float c0 = p.coef[0];
    const int K = p.K;
    for (int it = 0; it < p.iters; ++it) {
        for (int h = 0; h < 2; ++h) {
            for (int k = 1; k <= K; ++k) {
                ++stage;
                const unsigned long long* src = p.tagged + (size_t)rslot * n;
                unsigned long long* dst = p.tagged + (size_t)wslot * n;
                const unsigned* src4 = tw + (size_t)rslot * n;
                unsigned* dst4 = tw + (size_t)wslot * n;
                // stage s - 1 carries tag s (8-byte words) or parity (s - 1) & 1 (4-byte words);
                // the self-test waits for a tag no word will carry
                const unsigned want = W4 ? (p.selftest ? 2u : ((stage - 1u) & 1u)) : stage + extra;
                // issue up to UL loads per thread before checking any tag; words not yet carrying
                // the wanted tag are then re-read together (GROUP: each retry round costs one round
                // trip) or one at a time in list order, each stored as soon as it is ready (fewer
                // loads in flight while the owners have not published: the faster form where the
                // exchange dominates the order)
                for (int i0 = threadIdx.x; i0 < ucnt; i0 += UL * NT) {
                    Word w[UL];
#pragma unroll
                    for (int u = 0; u < UL; ++u) {
                        const int i = i0 + u * NT;
                        w[u] = i >= ucnt ? Word(0) : (W4 ? (Word)ld_relaxed_u32(src4 + ucol_s[i])
                                                        : (Word)ld_relaxed_u64(src + ucol_s[i]));
                    }
                    if (GROUP) {
                        unsigned pending = 0;
#pragma unroll
                        for (int u = 0; u < UL; ++u)
                            if (i0 + u * NT < ucnt && tag_of<W4>(w[u]) != want) pending |= 1u << u;
                        if (pending) {
                            const long long t0 = clock64();
                            do {
#pragma unroll
                                for (int u = 0; u < UL; ++u)
                                    if (pending & (1u << u))
                                        w[u] = W4 ? (Word)ld_relaxed_u32(src4 + ucol_s[i0 + u * NT])
                                                  : (Word)ld_relaxed_u64(src + ucol_s[i0 + u * NT]);
#pragma unroll
                                for (int u = 0; u < UL; ++u)
                                    if ((pending & (1u << u)) && tag_of<W4>(w[u]) == want) pending &= ~(1u << u);
                                if (pending && clock64() - t0 > p.budget) {
                                    atomicOr(p.flags, GS_FLAG_TIMEOUT);
                                    s_ok = 0;
                                    break;
                                }
                            } while (pending);
                        }
#pragma unroll
                        for (int u = 0; u < UL; ++u) {
                            const int i = i0 + u * NT;
                            if (i < ucnt) xc[i] = __uint_as_float((unsigned)w[u]);
                        }
                    } else {
#pragma unroll
                        for (int u = 0; u < UL; ++u) {
                            const int i = i0 + u * NT;
                            if (i >= ucnt) break;
                            if (tag_of<W4>(w[u]) != want) {
                                const long long t0 = clock64();
                                do {
                                    w[u] = W4 ? (Word)ld_relaxed_u32(src4 + ucol_s[i])
                                              : (Word)ld_relaxed_u64(src + ucol_s[i]);
                                    if (clock64() - t0 > p.budget) {
                                        atomicOr(p.flags, GS_FLAG_TIMEOUT);
                                        s_ok = 0;
                                        break;
                                    }
                                } while (tag_of<W4>(w[u]) != want);
                            }
                            xc[i] = __uint_as_float((unsigned)w[u]);
                        }
                    }
                }
                __syncthreads();
                if (!s_ok) return;
                const float ck = p.coef[k];
#pragma unroll
                for (int j = 0; j < RPT; ++j) {
                    const int row = r0 + (int)threadIdx.x + j * NT;
                    if (row >= r1) continue;
                    const float s =
                        WR > 0 ? row_dot_regs<WRA>(wv, lp, lidx_s + off[j] - (threadIdx.x & (GS_SELL_C - 1)),
                                                   threadIdx.x & (GS_SELL_C - 1), sval_s + off[j], width[j], xc)
                               : gs_sell_dot_cached(lidx_s + off[j] - (threadIdx.x & (GS_SELL_C - 1)),
                                                    threadIdx.x & (GS_SELL_C - 1), sval_s + off[j], width[j], xc);
                    float tk, acc;
                    if (k == 1) {
                        tk = s;
                        acc = fmaf(ck, tk, c0 * xo[j]);
                    } else {
                        tk = fmaf(2.f, s, -t2[j]);
                        acc = fmaf(ck, tk, yo[j]);
                    }
                    float pub;
                    if (k < K) {
                        t2[j] = k == 1 ? xo[j] : t1[j];
                        t1[j] = tk;
                        yo[j] = acc;
                        pub = tk;
                    } else {
                        const float m = h == 0 ? av[j] : bv[j];
                        float r = 0.f;
                        if (m != 0.f) {
                            r = m / acc;
                            if (!(r > 0.f) || isinf(r)) atomicOr(p.flags, GS_FLAG_NONFINITE);
                        }
                        (h == 0 ? p.u : p.v)[row] = r;
                        xo[j] = p.vol ? vv[j] * r : r;
                        pub = xo[j];
                    }
                    if (W4) st_relaxed_u32(dst4 + row, pack_tag32(pub, stage & 1u));
                    else st_relaxed_u64(dst + row, pack_tagged(pub, stage + 1u));
                }
                __syncthreads();  // xc is refilled by the next order
                rslot = wslot;
                wslot = wslot == 2 ? 0 : wslot + 1;
            }
        }
    }
}

constexpr int kSmemGraphMax = 200 * 1024;  // shared-memory budget for the resident graph slice
// Register-resident form of the tagged loop: blocks of up to kRegThreads rows (21 slices), one row
// per thread.  With 21 warps one SM sub-partition holds six of them, so a thread may hold 80
// registers; the first kRegSteps steps of its row stay in registers (24 steps spill).  Staging
// issues kRegLoads loads per thread per round (6,720 distinct columns in one round trip; 5,503 is
// the largest block of the 100k-point manifold graph, whose second round trip cost more than the
// registers saved).
constexpr int kRegThreads = 672;
constexpr int kRegSteps = 16;
constexpr int kRegLoads = 10;

template <int NT, bool W4, bool GROUP>
void (*tagged_kernel(int rpt))(PersistArgs)
{
    return rpt == 1 ? sinkhorn_tagged<1, NT, W4, GROUP>
                    : (rpt == 2 ? sinkhorn_tagged<2, NT, W4, GROUP> : sinkhorn_tagged<4, NT, W4, GROUP>);
}

template <int NT>
void (*gather_cache_kernel(bool tagged, bool w4, bool group, int rpt))(PersistArgs)
{
    if (tagged)
        return w4 ? (group ? tagged_kernel<NT, true, true>(rpt) : tagged_kernel<NT, true, false>(rpt))
                  : (group ? tagged_kernel<NT, false, true>(rpt) : tagged_kernel<NT, false, false>(rpt));
    return rpt == 1 ? sinkhorn_neighbour_sync<1, NT>
                    : (rpt == 2 ? sinkhorn_neighbour_sync<2, NT> : sinkhorn_neighbour_sync<4, NT>);
}

template <int G>
gs_status launch_persistent(gs_ctx* ctx, const gs_graph* g, PersistArgs& args)
{
    args.xc_rows = g->xc_rows;
    args.xc_ucol = g->xc_ucol;
    args.xc_ucnt = g->xc_ucnt;
    args.xc_lidx = g->xc_lidx;
    args.xc_max_e = g->xc_max_e;
    args.xc_max_u = g->xc_max_u;
    args.budget = ctx->barrier_selftest ? kSelfTestBudget : kBarrierBudget;
    args.selftest = ctx->barrier_selftest;
    args.xc_deps = g->xc_deps;
    args.xc_ndeps = g->xc_ndeps;
    args.ready = args.bar + kReadyStride;
    const size_t emax = (size_t)(g->xc_max_e + 31) / 32 * 32, umax = (size_t)(g->xc_max_u + 31) / 32 * 32;
    const size_t cache_smem = emax * 6 + umax * 8;

    // Gather-cache kernels with tagged-value or neighbour-flag synchronisation run on the cache
    // tables' own partition: one block of 1024 threads per SM, or two of 512.
    const int sync = gs_persist_sync_choice(ctx, g);
    const bool tagged = sync == 2 && args.tagged && 2.0 * args.K * (double)args.iters + 2.0 < 4294967295.0;
    const int bps = (g->xc_ok && ctx->num_sms > 0 && g->xc_blocks % ctx->num_sms == 0)
                        ? g->xc_blocks / ctx->num_sms : 0;
    if (ctx->persist_smem_graph == 2 && (bps == 1 || bps == 2) && (tagged || (sync == 1 && g->xc_deps))) {
        const int nt = kThreads / bps;
        const int rpt = (g->xc_rpb + nt - 1) / nt;
        if (rpt <= 4 && cache_smem <= (size_t)kSmemGraphMax / bps) {
            args.rows_per_block = g->xc_rpb;
            args.smem_graph = 2;
            const bool w4 = ctx->tag_word == 4;
            const bool group = gs_persist_sync_setting(ctx, g) != 4;
            void (*kern)(PersistArgs) = bps == 1 ? gather_cache_kernel<kThreads>(tagged, w4, group, rpt)
                                                 : gather_cache_kernel<kThreads / 2>(tagged, w4, group, rpt);
            int nt_launch = nt;
            if (bps == 1 && tagged && w4 && ctx->loop_regs && g->xc_rpb <= kRegThreads) {
                // one row per thread, each row's first kRegSteps steps in registers
                kern = group ? sinkhorn_tagged<1, kRegThreads, true, true, kRegSteps, kRegLoads>
                             : sinkhorn_tagged<1, kRegThreads, true, false, kRegSteps, kRegLoads>;
                nt_launch = kRegThreads;
            }
            if (tagged && !w4)  // 8-byte words: tag 0 is no stage
                cudaMemsetAsync(args.tagged, 0, sizeof(unsigned long long) * 3 * (size_t)args.n, ctx->stream);
            if (tagged && w4) {  // 4-byte words: slot k must not start with stage k's parity
                unsigned* tw = reinterpret_cast<unsigned*>(args.tagged);
                const size_t bytes = sizeof(unsigned) * (size_t)args.n;
                cudaMemsetAsync(tw, 0x01, bytes, ctx->stream);
                cudaMemsetAsync(tw + args.n, 0x00, bytes, ctx->stream);
                cudaMemsetAsync(tw + 2 * (size_t)args.n, 0x01, bytes, ctx->stream);
            }
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cache_smem);
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt_launch, cache_smem) == cudaSuccess &&
                per_sm >= bps) {
                ctx->barrier_selftest = 0;
                void* params[] = {&args};
                const cudaError_t e = cudaLaunchCooperativeKernel((void*)kern, dim3(g->xc_blocks), dim3(nt_launch),
                                                                  params, cache_smem, ctx->stream);
                if (e == cudaSuccess) {
                    gs_count(ctx, 1);
                    return GS_OK;
                }
            }
            cudaGetLastError();
        }
    }

    // Grid-barrier kernel: one 1024-thread block per SM over its own partition.
    const int blocks = ctx->num_sms;
    args.rows_per_block = gs_persist_rows_per_block(ctx, g->n, blocks);
    args.expect = (unsigned)blocks + (ctx->barrier_selftest ? 1u : 0u);
    size_t smem = 0;
    args.smem_graph = 0;
    if (ctx->persist_smem_graph == 2 && g->xc_ok && g->xc_blocks == blocks && cache_smem <= (size_t)kSmemGraphMax) {
        smem = cache_smem;
        args.smem_graph = 2;
    }
    if (!args.smem_graph && g->sptr && !g->sptr_host.empty() && ctx->persist_smem_graph) {
        // largest per-block entry range of the sliced ELL (host copy of its slice offsets)
        const int64_t ns = g->nslices;
        int64_t worst = 0;
        for (int b = 0; b < blocks; ++b) {
            const int64_t s0 = std::min<int64_t>(ns, (int64_t)b * args.rows_per_block / GS_SELL_C);
            const int64_t s1 = std::min<int64_t>(ns, ((int64_t)(b + 1) * args.rows_per_block + GS_SELL_C - 1) / GS_SELL_C);
            worst = std::max<int64_t>(worst, (int64_t)g->sptr_host[s1] - g->sptr_host[s0]);
        }
        const size_t need = 2 * (size_t)((worst + 31) / 32 * 32) * 4;
        if (need > 0 && need <= (size_t)kSmemGraphMax) {
            smem = need;
            args.smem_graph = 1;
        }
    }
    if (smem) cudaFuncSetAttribute(sinkhorn_persistent<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sinkhorn_persistent<G>, kThreads, smem) !=
            cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return GS_ERR_UNSUPPORTED;
    }
    ctx->barrier_selftest = 0;
    void* params[] = {&args};
    cudaError_t e = cudaLaunchCooperativeKernel((void*)sinkhorn_persistent<G>, dim3(blocks),
                                                dim3(kThreads), params, smem, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_UNSUPPORTED;
    }
    gs_count(ctx, 1);
    return GS_OK;
}

}  // namespace

// Enqueue the fixed-count loop as one persistent launch.  All vectors are in the filter's node
// order; `coef_dev` holds K+1 FP32 coefficients; `bar` has room for gs_persist_bar_words(ctx)
// unsigned words (zeroed here); `tagged` (3 n words, or null) is the tagged-value kernel's exchange buffer.
// Returns GS_ERR_UNSUPPORTED (nothing enqueued) when a cooperative launch is not possible.
gs_status gs_sinkhorn_persistent(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b,
                                 const float* vol, const float* coef_dev, int K, int iters,
                                 float* x, float* A, float* y, float* u, float* v, unsigned* bar,
                                 unsigned long long* tagged)
{
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device);
    if (!coop || g->n >= (1ll << 31)) return GS_ERR_UNSUPPORTED;
    const FilterCsr csr = gs_filter_csr(g);
    PersistArgs args;
    args.n = (int)g->n;
    args.rowptr = csr.rowptr;
    args.col = csr.col;
    args.pval = csr.pval;
    args.sptr = g->sptr;
    args.scol = g->scol;
    args.sval = g->sval;
    args.a = a;
    args.b = b;
    args.vol = vol;
    args.x = x;
    args.A = A;
    args.y = y;
    args.u = u;
    args.v = v;
    args.coef = coef_dev;
    args.K = K;
    args.iters = iters;
    args.bar = bar;
    args.flags = ctx->flags;
    args.tagged = tagged;
    cudaMemsetAsync(bar, 0, gs_persist_bar_words(ctx) * sizeof(unsigned), ctx->stream);
    const float m = g->mean_row;
    if (m <= 6.f) return launch_persistent<4>(ctx, g, args);
    if (m <= 14.f) return launch_persistent<8>(ctx, g, args);
    if (m <= 28.f) return launch_persistent<16>(ctx, g, args);
    return launch_persistent<32>(ctx, g, args);
}
