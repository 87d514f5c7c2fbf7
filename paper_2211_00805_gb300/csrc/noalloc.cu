// Allocation-free heat filter for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: plug-ins whose host application owns every device
// allocation (the library may not take memory from under it), and real-time loops that must never
// enter the allocator, whose calls can block or fail under memory pressure.  gs_heat_apply_noalloc serves them: it
// takes the graph as plain CSR device arrays instead of a library-owned handle and keeps the
// Chebyshev recurrence's two scratch blocks in a fixed array compiled into this file, so it
// allocates no device memory and needs no gs_ctx.
//
// The scratch is a file-scope __device__ array.  Its host-side name is only a stand-in for the
// symbol, not a device address, so the first call on each device looks the real address up with
// cudaGetSymbolAddress while that device is current and caches it.
#include <math.h>

#include <mutex>
#include <vector>

#include "gs_internal.cuh"

namespace {

constexpr int64_t kNoAllocBlockFloats = (int64_t)1 << 20;  // n * B limit per scratch block
constexpr int kMaxDevices = 64;

// Two scratch blocks of 2^20 floats each: 8 MiB on every GPU that loads the library, held until
// the process exits.  Every call shares them; nothing in them must start at zero (each order
// writes its block before the next order reads it).
static __device__ __align__(256) float g_noalloc_scratch[2 * kNoAllocBlockFloats];
// Status bits the kernels may raise (unused by the store epilogue, but the kernels need a target).
static __device__ __align__(256) int g_noalloc_flags[4];

std::mutex g_setup_mu;
float* g_scratch_addr[kMaxDevices] = {};
int* g_flags_addr[kMaxDevices] = {};

// Once per device, with that device current: resolve the device addresses of the arrays.
gs_status noalloc_setup(int dev, float** scratch, int** flags)
{
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* s = nullptr;
        void* f = nullptr;
        if (cudaGetSymbolAddress(&s, g_noalloc_scratch) != cudaSuccess ||
            cudaGetSymbolAddress(&f, g_noalloc_flags) != cudaSuccess || !s || !f) {
            cudaGetLastError();
            return GS_ERR_CUDA;
        }
        g_scratch_addr[dev] = static_cast<float*>(s);
        g_flags_addr[dev] = static_cast<int*>(f);
    }
    *scratch = g_scratch_addr[dev];
    *flags = g_flags_addr[dev];
    return GS_OK;
}

}  // namespace

extern "C" gs_status gs_heat_apply_noalloc(int64_t n, int64_t nnz, const int32_t* rowptr,
                                           const int32_t* col, const float* pval, double t, int K,
                                           const float* V, int B, float* Y, void* stream)
{
    if (!rowptr || !col || !pval || !V || !Y || V == Y) return GS_ERR_ARG;
    if (n < 2 || nnz < 0 || nnz >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31)) return GS_ERR_ARG;
    if (!(t > 0.0) || !isfinite(t) || K < 1 || K > 10000 || B < 1) return GS_ERR_ARG;
    if (n * (int64_t)B > kNoAllocBlockFloats) return GS_ERR_UNSUPPORTED;   // n * B above 2^20
    if (!gs_filter_supports(B, ((uintptr_t)V % 16) == 0 && ((uintptr_t)Y % 16) == 0)) return GS_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return GS_ERR_CUDA;
    }
    float* scratch = nullptr;
    int* flags = nullptr;
    gs_status st = noalloc_setup(dev, &scratch, &flags);
    if (st != GS_OK) return st;

    gs_ctx ctx;  // host-side bookkeeping only; owns no device memory here
    ctx.device = dev;
    ctx.stream = static_cast<cudaStream_t>(stream);
    ctx.flags = flags;
    gs_graph g;  // a view of the caller's arrays
    g.device = dev;
    g.n = n;
    g.nnz = nnz;
    g.rowptr = const_cast<int*>(rowptr);
    g.col = const_cast<int*>(col);
    g.pval = const_cast<float*>(pval);
    g.mean_row = (float)((double)nnz / (double)n);

    std::vector<double> c((size_t)K + 1);
    gs_heat_coefficients(t, K, c.data());
    Epilogue e;
    e.kind = EPI_STORE;
    e.out = Y;
    return gs_filter_enqueue(&ctx, &g, c.data(), K, B, const_cast<float*>(V), false, scratch,
                             scratch + kNoAllocBlockFloats, Y, e, nullptr, nullptr);
}
