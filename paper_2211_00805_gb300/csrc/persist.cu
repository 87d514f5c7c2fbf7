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

#include "gs_internal.cuh"
#include "sell_row.cuh"

namespace {

constexpr int kThreads = 1024;
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
        const float tk = (mode == 0) ? s : fmaf(2.f, s, -prev[row]);
        const float acc = (mode == 0) ? fmaf(ck, tk, c0 * cur[row]) : fmaf(ck, tk, p.y[row]);
        if (mode != 2) {
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
        const float pv = (mode == 0) ? 0.f : prev[row];
        const float yv = (mode == 0) ? c0 * cur[row] : p.y[row];
        const float s = gs_sell_row<false>(p.sptr, p.scol, p.sval, cur, row);
        const float tk = (mode == 0) ? s : fmaf(2.f, s, -pv);
        const float acc = fmaf(ck, tk, yv);
        if (mode != 2) {
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
                                         const float* num, float* out, float* xnext)
{
    if (p.sptr) rows_order_sell(p, r0, r1, mode, ck, c0, cur, prev, next, num, out, xnext);
    else rows_order<G>(p, r0, r1, mode, ck, c0, cur, prev, next, num, out, xnext);
}

template <int G>
__global__ void __launch_bounds__(kThreads) sinkhorn_persistent(const PersistArgs p)
{
    __shared__ int s_ok;
    if (threadIdx.x == 0) s_ok = 1;
    __syncthreads();
    const int per = ((p.n + gridDim.x - 1) / gridDim.x + GS_SELL_C - 1) / GS_SELL_C * GS_SELL_C;
    const int r0 = min(p.n, (int)blockIdx.x * per), r1 = min(p.n, r0 + per);
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
                rows_any<G>(p, r0, r1, 2, p.coef[1], c0, X, nullptr, nullptr, num, out, Ab);
                if (!grid_barrier(p.bar, p.flags, &s_ok, p.expect, p.budget)) return;
                float* t = X; X = Ab; Ab = t;
                continue;
            }
            rows_any<G>(p, r0, r1, 0, p.coef[1], c0, X, nullptr, Ab, nullptr, nullptr, nullptr);
            if (!grid_barrier(p.bar, p.flags, &s_ok, p.expect, p.budget)) return;
            float* prev = X;
            float* cur = Ab;
            for (int k = 2; k <= p.K; ++k) {
                if (k < p.K) {
                    rows_any<G>(p, r0, r1, 1, p.coef[k], 0.f, cur, prev, prev, nullptr, nullptr, nullptr);
                    if (!grid_barrier(p.bar, p.flags, &s_ok, p.expect, p.budget)) return;
                    float* t = prev; prev = cur; cur = t;
                } else {
                    rows_any<G>(p, r0, r1, 2, p.coef[k], 0.f, cur, prev, nullptr, num, out, prev);
                    if (!grid_barrier(p.bar, p.flags, &s_ok, p.expect, p.budget)) return;
                    X = prev;
                    Ab = cur;
                }
            }
        }
    }
}

template <int G>
gs_status launch_persistent(gs_ctx* ctx, PersistArgs& args)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sinkhorn_persistent<G>, kThreads, 0) !=
            cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return GS_ERR_UNSUPPORTED;
    }
    const int blocks = ctx->num_sms;  // one block of kThreads per SM
    args.expect = (unsigned)blocks + (ctx->barrier_selftest ? 1u : 0u);
    args.budget = ctx->barrier_selftest ? kSelfTestBudget : kBarrierBudget;
    ctx->barrier_selftest = 0;
    void* params[] = {&args};
    cudaError_t e = cudaLaunchCooperativeKernel((void*)sinkhorn_persistent<G>, dim3(blocks),
                                                dim3(kThreads), params, 0, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GS_ERR_UNSUPPORTED;
    }
    gs_count(ctx, 1);
    return GS_OK;
}

}  // namespace

// Enqueue the fixed-count loop as one persistent launch.  All vectors are in the filter's node
// order; `coef_dev` holds K+1 FP32 coefficients; `bar` is two zeroed unsigned words.
// Returns GS_ERR_UNSUPPORTED (nothing enqueued) when a cooperative launch is not possible.
gs_status gs_sinkhorn_persistent(gs_ctx* ctx, const gs_graph* g, const float* a, const float* b,
                                 const float* vol, const float* coef_dev, int K, int iters,
                                 float* x, float* A, float* y, float* u, float* v, unsigned* bar)
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
    cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), ctx->stream);
    const float m = g->mean_row;
    if (m <= 6.f) return launch_persistent<4>(ctx, args);
    if (m <= 14.f) return launch_persistent<8>(ctx, args);
    if (m <= 28.f) return launch_persistent<16>(ctx, args);
    return launch_persistent<32>(ctx, args);
}
