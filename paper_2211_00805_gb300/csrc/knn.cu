// Common graph of Sec. 4 ("a common graph using an affinity kernel") built on the GPU:
//   1. screen: for every query point, the 32 smallest FP32 squared distances |q|^2 + |c|^2 - 2 q.c
//      over all other points (register-tiled dot products, warp-held sorted candidate lists);
//   2. rerank: the 32 candidates' squared distances recomputed in FP64 by direct differences
//      (the same operation order as the definition, no contraction), sorted by (distance, index),
//      the first k kept;
//   3. sigma = median of the n*k kNN distances by an 8-pass radix select on the FP64 bit patterns
//      (mean of the two middle values when n*k is even);
//   4. symmetrise: edge set = union of the directed kNN edges, A_ij = exp(-d_ij^2 / sigma^2),
//      FP64 degrees, P_ij = A_ij / sqrt(D_ii D_jj) (Sec. 3.4), packed as CSR with ascending columns.
#include <math.h>
#include <stdint.h>

#include <vector>

#include "gs_internal.cuh"
#include "async_copy.cuh"

namespace {

constexpr int KK = 32;   // screened candidates per query
constexpr int QT = 64;   // queries per block
constexpr int CT = 64;   // candidates per tile
constexpr int DC = 32;   // feature chunk
constexpr unsigned FULL = 0xffffffffu;

inline unsigned nblk(int64_t work, int per) { return (unsigned)((work + per - 1) / per); }

__global__ void sq_norms(const float* __restrict__ X, int64_t n, int d, float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int c = 0; c < d; ++c) {
        const float v = X[i * d + c];
        s = fmaf(v, v, s);
    }
    out[i] = s;
}

// Insert (dv, iv) into the warp's sorted list (lane l holds entry l) if it beats the last entry.
__device__ __forceinline__ void list_insert(float& ld, int& li, float dv, int iv, int lane)
{
    const float last = __shfl_sync(FULL, ld, 31);
    const int lasti = __shfl_sync(FULL, li, 31);
    if (!(dv < last || (dv == last && iv < lasti))) return;
    const bool less = (ld < dv) || (ld == dv && li < iv);
    const int pos = __popc(__ballot_sync(FULL, less));
    const float ud = __shfl_up_sync(FULL, ld, 1);
    const int ui = __shfl_up_sync(FULL, li, 1);
    if (lane > pos) {
        ld = ud;
        li = ui;
    } else if (lane == pos) {
        ld = dv;
        li = iv;
    }
}

// Fold one 64 x 64 tile of squared distances into the warp's 8 sorted top-32 lists (warp w owns
// query rows 8w .. 8w+7 of the tile; lane l holds entry l of every list).
__device__ __forceinline__ void select_tile(const float (*tile)[CT + 1], int c0, int warp, int lane,
                                            float (&ld)[8], int (&li)[8])
{
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int qrow = warp * 8 + r;
        const float thr = __shfl_sync(FULL, ld[r], 31);
        const float d0 = tile[qrow][lane], d1 = tile[qrow][lane + 32];
        unsigned m0 = __ballot_sync(FULL, d0 <= thr && d0 < INFINITY);
        unsigned m1 = __ballot_sync(FULL, d1 <= thr && d1 < INFINITY);
        while (m0) {
            const int src = __ffs(m0) - 1;
            m0 &= m0 - 1;
            list_insert(ld[r], li[r], __shfl_sync(FULL, d0, src), c0 + src, lane);
        }
        while (m1) {
            const int src = __ffs(m1) - 1;
            m1 &= m1 - 1;
            list_insert(ld[r], li[r], __shfl_sync(FULL, d1, src), c0 + 32 + src, lane);
        }
    }
}

__global__ void __launch_bounds__(256) knn_screen(const float* __restrict__ X,
                                                  const float* __restrict__ norms, int n, int d,
                                                  int* __restrict__ cand)
{
    __shared__ __align__(16) float sq[DC][QT + 4];
    __shared__ __align__(16) float sc[DC][CT + 4];
    __shared__ float tile[QT][CT + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q0 = blockIdx.x * QT;
    const int tq = tid >> 4, tc = tid & 15;
    float ld[8];
    int li[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        ld[r] = INFINITY;
        li[r] = 0x7fffffff;
    }
    float qn[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gq = q0 + tq * 4 + i;
        qn[i] = gq < n ? norms[gq] : 0.f;
    }
    for (int c0 = 0; c0 < n; c0 += CT) {
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        for (int k0 = 0; k0 < d; k0 += DC) {
            for (int e = tid; e < QT * DC; e += 256) {
                const int qq = e / DC, kk = e % DC;
                const int gq = q0 + qq, gk = k0 + kk;
                sq[kk][qq] = (gq < n && gk < d) ? X[(int64_t)gq * d + gk] : 0.f;
                const int gc = c0 + qq;
                sc[kk][qq] = (gc < n && gk < d) ? X[(int64_t)gc * d + gk] : 0.f;
            }
            __syncthreads();
            const int kmax = (d - k0) < DC ? (d - k0) : DC;
            for (int kk = 0; kk < kmax; ++kk) {
                const float4 a = *reinterpret_cast<const float4*>(&sq[kk][tq * 4]);
                const float4 b = *reinterpret_cast<const float4*>(&sc[kk][tc * 4]);
                const float av[4] = {a.x, a.y, a.z, a.w};
                const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gc = c0 + tc * 4 + j;
            const float cn = gc < n ? norms[gc] : 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int gq = q0 + tq * 4 + i;
                tile[tq * 4 + i][tc * 4 + j] =
                    (gc < n && gc != gq) ? fmaf(-2.f, acc[i][j], qn[i] + cn) : INFINITY;
            }
        }
        __syncthreads();
        select_tile(tile, c0, warp, lane, ld, li);
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int gq = q0 + warp * 8 + r;
        if (gq < n) cand[(int64_t)gq * KK + lane] = li[r];
    }
}


// ------------------------------------------------------------------ tensor-core screening
// Same tiles and selection as knn_screen, but the 64 x 64 dot-product tile runs on the tensor
// cores (warp-level m16n8k8 TF32 MMA) with the 3xTF32 split: x = hi + lo with hi, lo TF32, and
// q.c ~ q_hi.c_hi + q_hi.c_lo + q_lo.c_hi, which recovers FP32-grade products.  Points are split
// once into hi / lo arrays padded to dp (a multiple of 8) features.
constexpr int TC_DC = 32;
constexpr int TC_LD = TC_DC + 4;  // shared row stride (floats): conflict-free fragment loads
constexpr int TC_SMEM = 4 * 64 * TC_LD * 4 + 64 * (CT + 1) * 4;

__device__ __forceinline__ float tf32_round(float x)
{
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__global__ void split_tf32(const float* __restrict__ X, int64_t n, int d, int dp,
                           float* __restrict__ hi, float* __restrict__ lo)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * dp) return;
    const int64_t r = i / dp;
    const int c = (int)(i - r * dp);
    const float x = c < d ? X[r * d + c] : 0.f;
    const float h = tf32_round(x);
    hi[i] = h;
    lo[i] = tf32_round(x - h);
}

__device__ __forceinline__ void mma_tf32(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(256) knn_screen_tc(const float* __restrict__ hi,
                                                     const float* __restrict__ lo,
                                                     const float* __restrict__ norms, int n,
                                                     int dp, int* __restrict__ cand)
{
    extern __shared__ __align__(16) float tc_sm[];
    float* qh = tc_sm;
    float* ql = qh + 64 * TC_LD;
    float* chh = ql + 64 * TC_LD;
    float* cll = chh + 64 * TC_LD;
    float (*tile)[CT + 1] = reinterpret_cast<float (*)[CT + 1]>(cll + 64 * TC_LD);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int q0 = blockIdx.x * QT;
    const int m0 = 16 * (warp >> 1);   // this warp's 16 query rows of the tile
    const int nb = 32 * (warp & 1);    // and its 32 candidate columns (4 n8 tiles)
    float ld[8];
    int li[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        ld[r] = INFINITY;
        li[r] = 0x7fffffff;
    }
    const float qn0 = (q0 + m0 + gid < n) ? norms[q0 + m0 + gid] : 0.f;
    const float qn1 = (q0 + m0 + gid + 8 < n) ? norms[q0 + m0 + gid + 8] : 0.f;
    for (int c0 = 0; c0 < n; c0 += CT) {
        float acc[4][4];
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[t][v] = 0.f;
        for (int k0 = 0; k0 < dp; k0 += TC_DC) {
            const int kc = (dp - k0) < TC_DC ? (dp - k0) : TC_DC;  // multiple of 8
            for (int e = tid; e < 64 * TC_DC; e += 256) {
                const int rr = e / TC_DC, kk = e % TC_DC;
                const bool kin = kk < kc;
                const int gq = q0 + rr, gc = c0 + rr;
                const int64_t oq = (int64_t)gq * dp + k0 + kk, oc = (int64_t)gc * dp + k0 + kk;
                qh[rr * TC_LD + kk] = (gq < n && kin) ? hi[oq] : 0.f;
                ql[rr * TC_LD + kk] = (gq < n && kin) ? lo[oq] : 0.f;
                chh[rr * TC_LD + kk] = (gc < n && kin) ? hi[oc] : 0.f;
                cll[rr * TC_LD + kk] = (gc < n && kin) ? lo[oc] : 0.f;
            }
            __syncthreads();
            for (int kk = 0; kk < kc; kk += 8) {
                unsigned ah[4], al[4];
                const int ra = (m0 + gid) * TC_LD + kk + tig, rb = (m0 + gid + 8) * TC_LD + kk + tig;
                ah[0] = __float_as_uint(qh[ra]);
                ah[1] = __float_as_uint(qh[rb]);
                ah[2] = __float_as_uint(qh[ra + 4]);
                ah[3] = __float_as_uint(qh[rb + 4]);
                al[0] = __float_as_uint(ql[ra]);
                al[1] = __float_as_uint(ql[rb]);
                al[2] = __float_as_uint(ql[ra + 4]);
                al[3] = __float_as_uint(ql[rb + 4]);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int cb = (nb + 8 * t + gid) * TC_LD + kk + tig;
                    const unsigned bh0 = __float_as_uint(chh[cb]), bh1 = __float_as_uint(chh[cb + 4]);
                    const unsigned bl0 = __float_as_uint(cll[cb]), bl1 = __float_as_uint(cll[cb + 4]);
                    mma_tf32(acc[t], al, bh0, bh1);
                    mma_tf32(acc[t], ah, bl0, bl1);
                    mma_tf32(acc[t], ah, bh0, bh1);
                }
            }
            __syncthreads();
        }
        // D fragment: (gid, 2tig), (gid, 2tig+1), (gid+8, 2tig), (gid+8, 2tig+1)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int rl = m0 + gid + ((v >> 1) << 3);
                const int cl = nb + 8 * t + 2 * tig + (v & 1);
                const int gq = q0 + rl, gc = c0 + cl;
                const float qn = (v >> 1) ? qn1 : qn0;
                const float cn = gc < n ? norms[gc] : 0.f;
                tile[rl][cl] = (gc < n && gc != gq) ? fmaf(-2.f, acc[t][v], qn + cn) : INFINITY;
            }
        }
        __syncthreads();
        select_tile(tile, c0, warp, lane, ld, li);
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int gq = q0 + warp * 8 + r;
        if (gq < n) cand[(int64_t)gq * KK + lane] = li[r];
    }
}

// Register-resident variant for dp <= 64 (KS = dp / 8 k-steps): each warp keeps the TF32 hi / lo
// A fragments of its 16 query rows in registers for the whole kernel, and candidate tiles (hi and
// lo, 64 rows x dp) stream through double-buffered shared memory with 16-byte cp.async copies, so
// a candidate tile is read once per block and the query rows never again.
template <int KS>
__global__ void __launch_bounds__(256, 2) knn_screen_tc_reg(const float* __restrict__ hi,
                                                             const float* __restrict__ lo,
                                                             const float* __restrict__ norms,
                                                             int n, int* __restrict__ cand)
{
    constexpr int DP = 8 * KS;
    constexpr int LDC = DP + 4;  // (LDC / 4) odd: conflict-free B-fragment loads
    extern __shared__ __align__(16) float tc_sm[];
    float* cbuf = tc_sm;  // [2 buffers][2 (hi, lo)][64][LDC]
    float (*tile)[CT + 1] = reinterpret_cast<float (*)[CT + 1]>(tc_sm + 2 * 2 * 64 * LDC);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int q0 = blockIdx.x * QT;
    const int m0 = 16 * (warp >> 1), nb = 32 * (warp & 1);
    float ld[8];
    int li[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        ld[r] = INFINITY;
        li[r] = 0x7fffffff;
    }
    // A fragments: rows (m0 + gid) and (m0 + gid + 8), columns 8s + tig and 8s + tig + 4
    unsigned ah[KS][4], al[KS][4];
    {
        const int ra = q0 + m0 + gid, rb = ra + 8;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            const int k = 8 * ks + tig;
            ah[ks][0] = ra < n ? __float_as_uint(hi[(int64_t)ra * DP + k]) : 0u;
            ah[ks][1] = rb < n ? __float_as_uint(hi[(int64_t)rb * DP + k]) : 0u;
            ah[ks][2] = ra < n ? __float_as_uint(hi[(int64_t)ra * DP + k + 4]) : 0u;
            ah[ks][3] = rb < n ? __float_as_uint(hi[(int64_t)rb * DP + k + 4]) : 0u;
            al[ks][0] = ra < n ? __float_as_uint(lo[(int64_t)ra * DP + k]) : 0u;
            al[ks][1] = rb < n ? __float_as_uint(lo[(int64_t)rb * DP + k]) : 0u;
            al[ks][2] = ra < n ? __float_as_uint(lo[(int64_t)ra * DP + k + 4]) : 0u;
            al[ks][3] = rb < n ? __float_as_uint(lo[(int64_t)rb * DP + k + 4]) : 0u;
        }
    }
    const float qn0 = (q0 + m0 + gid < n) ? norms[q0 + m0 + gid] : 0.f;
    const float qn1 = (q0 + m0 + gid + 8 < n) ? norms[q0 + m0 + gid + 8] : 0.f;

    constexpr int CHUNKS = 2 * 64 * (DP / 4);  // 16-byte pieces of one candidate tile (hi + lo)
    auto stage = [&](int c0, int buf) {
        for (int i = tid; i < CHUNKS; i += 256) {
            const int part = i / (64 * (DP / 4));          // 0 hi, 1 lo
            const int rem = i - part * 64 * (DP / 4);
            const int r = rem / (DP / 4), q = rem - r * (DP / 4);
            float* dst = cbuf + ((buf * 2 + part) * 64 + r) * LDC + 4 * q;
            const int gc = c0 + r;
            if (gc < n) {
                gs_cp_async16(dst, (part ? lo : hi) + (int64_t)gc * DP + 4 * q);
            } else {
                dst[0] = 0.f; dst[1] = 0.f; dst[2] = 0.f; dst[3] = 0.f;
            }
        }
        gs_cp_async_commit();
    };
    const int ntiles = (n + CT - 1) / CT;
    stage(0, 0);
    for (int t = 0; t < ntiles; ++t) {
        const int c0 = t * CT, buf = t & 1;
        if (t + 1 < ntiles) {
            stage(c0 + CT, buf ^ 1);
            gs_cp_async_wait<1>();
        } else {
            gs_cp_async_wait<0>();
        }
        __syncthreads();
        const float* chh = cbuf + (buf * 2 + 0) * 64 * LDC;
        const float* cll = cbuf + (buf * 2 + 1) * 64 * LDC;
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int cb = (nb + 8 * u + gid) * LDC + 8 * ks + tig;
                const unsigned bh0 = __float_as_uint(chh[cb]), bh1 = __float_as_uint(chh[cb + 4]);
                const unsigned bl0 = __float_as_uint(cll[cb]), bl1 = __float_as_uint(cll[cb + 4]);
                mma_tf32(acc[u], al[ks], bh0, bh1);
                mma_tf32(acc[u], ah[ks], bl0, bl1);
                mma_tf32(acc[u], ah[ks], bh0, bh1);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const int rl = m0 + gid + ((v >> 1) << 3);
                const int cl = nb + 8 * u + 2 * tig + (v & 1);
                const int gq = q0 + rl, gc = c0 + cl;
                const float qn = (v >> 1) ? qn1 : qn0;
                const float cn = gc < n ? norms[gc] : 0.f;
                tile[rl][cl] = (gc < n && gc != gq) ? fmaf(-2.f, acc[u][v], qn + cn) : INFINITY;
            }
        }
        __syncthreads();
        select_tile(tile, c0, warp, lane, ld, li);
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int gq = q0 + warp * 8 + r;
        if (gq < n) cand[(int64_t)gq * KK + lane] = li[r];
    }
}

template <int KS>
constexpr int tc_reg_smem() { return 2 * 2 * 64 * (8 * KS + 4) * 4 + 64 * (CT + 1) * 4; }

template <int KS>
void launch_tc_reg(gs_ctx* ctx, const float* hi, const float* lo, const float* norms, int64_t n, int* cand)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(knn_screen_tc_reg<KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc_reg_smem<KS>());
        attr = true;
    }
    knn_screen_tc_reg<KS><<<nblk(n, QT), 256, tc_reg_smem<KS>(), ctx->stream>>>(hi, lo, norms, (int)n, cand);
}

// One warp per query: FP64 direct-difference squared distances of the 32 candidates, in the
// definition's order (no fused multiply-add), rank by (distance, index), keep the first k.
// float -> double by moving the bits (exact, as the conversion is): a normal or zero float only
// widens its exponent and mantissa fields; subnormal, infinite and NaN inputs take the conversion
// instruction.  The rerank is bound by its double-precision instructions; this and the integer
// rank compares below took it from 1.94 to 1.56 ms at n = 100k (the two not measured apart).
__device__ __forceinline__ double widen_exact(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned m = u & 0x7fffffu;
    if (e == 0xffu || (e == 0u && m != 0u)) return (double)f;
    const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                    (e ? (unsigned long long)(e + 896u) << 52 : 0ull) |
                                    ((unsigned long long)m << 29);
    return __longlong_as_double((long long)bits);
}

__global__ void knn_rerank(const float* __restrict__ X, int n, int d, int k,
                           const int* __restrict__ cand, int32_t* __restrict__ idx,
                           float* __restrict__ dist, double* __restrict__ dist64)
{
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= n) return;
    const int c = cand[q * KK + lane];
    double s = INFINITY;
    if (c >= 0 && c < n && c != q) {
        s = 0.0;
        const float* xq = X + q * d;
        const float* xc = X + (int64_t)c * d;
        for (int i = 0; i < d; ++i) {
            const double diff = __dsub_rn(widen_exact(xq[i]), widen_exact(xc[i]));
            s = __dadd_rn(s, __dmul_rn(diff, diff));
        }
    }
    // s is +0, positive or +inf (NaN only from NaN coordinates), so the order of the values is the
    // order of their bit patterns: the rank is taken with integer compares
    const unsigned long long key = (unsigned long long)__double_as_longlong(s);
    int rank = 0;
    for (int j = 0; j < 32; ++j) {
        const unsigned long long kj = __shfl_sync(FULL, key, j);
        const int cj = __shfl_sync(FULL, c, j);
        rank += (kj < key) || (kj == key && cj < c);
    }
    if (rank < k) {
        const double e = sqrt(s);
        idx[q * k + rank] = c;
        if (dist) dist[q * k + rank] = (float)e;
        if (dist64) dist64[q * k + rank] = e;
    }
}

// ---------------------------------------------------------------------- radix select (FP64)
struct SelState {
    unsigned long long prefix;
    unsigned long long mask;
    long long rank;
};

__global__ void sel_init(SelState* st, long long rank, unsigned* hist)
{
    st->prefix = 0ull;
    st->mask = 0ull;
    st->rank = rank;
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
}

__global__ void sel_hist(const unsigned long long* __restrict__ keys, int64_t N,
                         const SelState* __restrict__ st, int shift, unsigned* __restrict__ hist)
{
    __shared__ unsigned h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    const unsigned long long prefix = st->prefix, mask = st->mask;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[i];
        if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 255ull], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&hist[b], h[b]);
}

__global__ void sel_pick(SelState* st, unsigned* hist, int shift)
{
    if (threadIdx.x == 0) {
        long long r = st->rank;
        int b = 0;
        for (; b < 255; ++b) {
            if (r < (long long)hist[b]) break;
            r -= hist[b];
        }
        st->prefix |= (unsigned long long)b << shift;
        st->mask |= 255ull << shift;
        st->rank = r;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0u;
}

__global__ void sel_median(const SelState* lo, const SelState* hi, int even, double* sigma)
{
    const double a = __longlong_as_double((long long)lo->prefix);
    const double b = __longlong_as_double((long long)hi->prefix);
    *sigma = even ? (a + b) / 2.0 : b;
}

__global__ void set_scalar(double* dst, double v) { *dst = v; }

// ------------------------------------------------------------------------------------- scan
// Exclusive prefix sum of int32 counts into int64 offsets out[0..n] (out[n] = total).
constexpr int SCAN_T = 1024, SCAN_I = 4, SCAN_TILE = SCAN_T * SCAN_I;

__global__ void __launch_bounds__(SCAN_T) scan_tiles(const int* __restrict__ in, int64_t n,
                                                     int64_t* __restrict__ out,
                                                     int64_t* __restrict__ sums)
{
    __shared__ int64_t wsum[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    int64_t v[SCAN_I];
    int64_t t = 0;
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        t += v[i];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = t;
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t o = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += o;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t s = wsum[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t o = __shfl_up_sync(FULL, s, off);
            if (lane >= off) s += o;
        }
        wsum[lane] = s;
    }
    __syncthreads();
    int64_t run = incl - t + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
    for (int i = 0; i < SCAN_I; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == SCAN_T - 1) sums[blockIdx.x] = run;
}

__global__ void scan_sums(int64_t* sums, int64_t nb, int64_t* total_out)
{
    if (threadIdx.x != 0) return;
    int64_t run = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const int64_t s = sums[b];
        sums[b] = run;
        run += s;
    }
    *total_out = run;
}

__global__ void scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ sums)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / SCAN_TILE];
}

}  // namespace

void gs_exclusive_scan(cudaStream_t s, const int* cnt, int64_t n, int64_t* out, int64_t* sums)
{
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    scan_tiles<<<(unsigned)nb, SCAN_T, 0, s>>>(cnt, n, out, sums);
    scan_sums<<<1, 32, 0, s>>>(sums, nb, out + n);
    scan_add<<<nblk(n, 256), 256, 0, s>>>(out, n, sums);
}

namespace {

// --------------------------------------------------------------------------- symmetrise
__global__ void in_count(const int32_t* __restrict__ idx, int64_t nk, int* __restrict__ cnt)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nk) atomicAdd(&cnt[idx[e]], 1);
}

__global__ void in_fill(const int32_t* __restrict__ idx, const double* __restrict__ d64, int64_t n,
                        int k, const int64_t* __restrict__ inptr, int* __restrict__ cursor,
                        int* __restrict__ in_src, double* __restrict__ in_d)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * k) return;
    const int j = idx[e];
    const int64_t pos = inptr[j] + atomicAdd(&cursor[j], 1);
    in_src[pos] = (int)(e / k);
    in_d[pos] = d64[e];
}

// Sort each row's (column, distance) list by column (insertion sort; rows are short).
__global__ void sort_rows_by_col(int64_t n, const int64_t* __restrict__ ptr, int stride,
                                 int* __restrict__ c, double* __restrict__ dd)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t b = ptr ? ptr[r] : r * stride;
    const int64_t e = ptr ? ptr[r + 1] : (r + 1) * stride;
    for (int64_t i = b + 1; i < e; ++i) {
        const int ci = c[i];
        const double di = dd[i];
        int64_t j = i - 1;
        while (j >= b && c[j] > ci) {
            c[j + 1] = c[j];
            dd[j + 1] = dd[j];
            --j;
        }
        c[j + 1] = ci;
        dd[j + 1] = di;
    }
}

// Union of the sorted out-list (k entries) and in-list of each row: count, or fill col/A/deg.
template <bool FILL>
__global__ void union_rows(int64_t n, int k, const int* __restrict__ oc, const double* __restrict__ od,
                           const int64_t* __restrict__ inptr, const int* __restrict__ ic,
                           const double* __restrict__ id, int* __restrict__ cnt,
                           const int64_t* __restrict__ rowptr, int* __restrict__ col,
                           float* __restrict__ aval, double* __restrict__ ed,
                           double* __restrict__ deg, const double* __restrict__ sigma)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t a = r * k;
    const int64_t ae = a + k;
    int64_t b = inptr[r];
    const int64_t be = inptr[r + 1];
    int64_t w = FILL ? rowptr[r] : 0;
    int count = 0;
    double s2 = 0.0, dg = 0.0;
    if (FILL) s2 = (*sigma) * (*sigma);
    while (a < ae || b < be) {
        int cc;
        double dv;
        if (b >= be || (a < ae && oc[a] < ic[b])) {
            cc = oc[a];
            dv = od[a];
            ++a;
        } else if (a >= ae || ic[b] < oc[a]) {
            cc = ic[b];
            dv = id[b];
            ++b;
        } else {  // mutual edge: the same pair, the same FP64 distance
            cc = oc[a];
            dv = od[a];
            ++a;
            ++b;
        }
        ++count;
        if (FILL) {
            const double A = exp(-(dv * dv) / s2);
            col[w] = cc;
            aval[w] = (float)A;
            ed[w] = A;
            dg += A;
            ++w;
        }
    }
    if (!FILL) cnt[r] = count;
    if (FILL) deg[r] = dg;
}

__global__ void normalise_from_fp64(int64_t n, const int* __restrict__ rowptr,
                                    const int* __restrict__ col, const double* __restrict__ ea,
                                    const double* __restrict__ deg, float* __restrict__ pval,
                                    int* __restrict__ bad)
{
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const double di = deg[row];
    if (lane == 0 && !(di > 0.0)) atomicOr(bad, 1);
    for (int e = rowptr[row] + lane; e < rowptr[row + 1]; e += 32)
        pval[e] = (float)(ea[e] / sqrt(di * deg[col[e]]));
}

__global__ void rowptr_to32(int64_t n1, const int64_t* __restrict__ in, int* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n1) out[i] = (int)in[i];
}

}  // namespace

// Screen selection and the workspace the kNN stage takes from the front of the context's buffer:
// 2 tensor-memory kernel (tcgen05; d + 2 <= 64), 1 warp-level TF32 MMA (d >= 16), 0 CUDA cores.
struct KnnPlan {
    WsPlan p;
    size_t inorm = 0, icand = 0, ihi = 0, ilo = 0, iumma = 0, iord = 0, ord_bytes = 0;
    int mode = 0;
};

static KnnPlan knn_plan(const gs_ctx* ctx, int64_t n, int d)
{
    KnnPlan k;
    if (ctx->knn_tensor_cores == 2 && gs_knn_umma_bytes(n, d) > 0 && gs_knn_umma_available()) k.mode = 2;
    else if (ctx->knn_tensor_cores >= 1 && d >= 16) k.mode = 1;
    const int dp = (d + 7) / 8 * 8;
    k.inorm = k.p.add(sizeof(float) * n);
    k.icand = k.p.add(sizeof(int) * n * KK);
    if (k.mode == 1) {
        k.ihi = k.p.add(sizeof(float) * n * dp);
        k.ilo = k.p.add(sizeof(float) * n * dp);
    }
    if (k.mode == 2) {
        k.iumma = k.p.add(gs_knn_umma_bytes(n, d));
        k.ord_bytes = gs_points_order_bytes(ctx, n, d);  // the screen's spatial order of the points
        if (k.ord_bytes) k.iord = k.p.add(k.ord_bytes);
    }
    return k;
}

size_t gs_knn_ws_bytes(const gs_ctx* ctx, int64_t n, int d) { return knn_plan(ctx, n, d).p.total; }

gs_status gs_knn_launch(gs_ctx* ctx, const float* X, int64_t n, int d, int k, int32_t* idx,
                        float* dist, double* dist64, const int* ord)
{
    const KnnPlan kp = knn_plan(ctx, n, d);
    const int dp = (d + 7) / 8 * 8;
    gs_status st = gs_ws_ensure(ctx, kp.p.total);
    if (st != GS_OK) return st;
    float* norms = ws_at<float>(ctx, kp.p, kp.inorm);
    int* cand = ws_at<int>(ctx, kp.p, kp.icand);
    sq_norms<<<nblk(n, 256), 256, 0, ctx->stream>>>(X, n, d, norms);
    gs_count(ctx, 1);
    bool screened = false;
    if (kp.mode == 2) {
        int* own = nullptr;
        if (!ord && kp.ord_bytes &&
            (st = gs_points_order(ctx, X, n, d, ws_at<void>(ctx, kp.p, kp.iord), kp.ord_bytes, &own)) != GS_OK)
            return st;
        st = gs_knn_screen_umma(ctx, X, norms, n, d, ws_at<unsigned char>(ctx, kp.p, kp.iumma), ord ? ord : own,
                                cand);
        if (st == GS_OK) screened = true;
        else if (st != GS_ERR_UNSUPPORTED) return st;
    }
    if (!screened && kp.mode == 1) {
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(knn_screen_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
            attr = true;
        }
        float* hi = ws_at<float>(ctx, kp.p, kp.ihi);
        float* lo = ws_at<float>(ctx, kp.p, kp.ilo);
        split_tf32<<<nblk(n * dp, 256), 256, 0, ctx->stream>>>(X, n, d, dp, hi, lo);
        switch (dp / 8) {
            case 2: launch_tc_reg<2>(ctx, hi, lo, norms, n, cand); break;
            case 3: launch_tc_reg<3>(ctx, hi, lo, norms, n, cand); break;
            case 4: launch_tc_reg<4>(ctx, hi, lo, norms, n, cand); break;
            case 5: launch_tc_reg<5>(ctx, hi, lo, norms, n, cand); break;
            case 6: launch_tc_reg<6>(ctx, hi, lo, norms, n, cand); break;
            case 7: launch_tc_reg<7>(ctx, hi, lo, norms, n, cand); break;
            case 8: launch_tc_reg<8>(ctx, hi, lo, norms, n, cand); break;
            default:
                knn_screen_tc<<<nblk(n, QT), 256, TC_SMEM, ctx->stream>>>(hi, lo, norms, (int)n, dp, cand);
        }
        gs_count(ctx, 2);
        screened = true;
    }
    if (!screened) {
        knn_screen<<<nblk(n, QT), 256, 0, ctx->stream>>>(X, norms, (int)n, d, cand);
        gs_count(ctx, 1);
    }
    knn_rerank<<<nblk(n * 32, 256), 256, 0, ctx->stream>>>(X, (int)n, d, k, cand, idx, dist, dist64);
    gs_count(ctx, 1);
    return gs_cuda_check(ctx, cudaGetLastError(), "kNN launch");
}

gs_status gs_build_graph_impl(gs_ctx* ctx, const float* X, int64_t n, int d, int k, float sigma,
                              gs_graph** out)
{
    const int64_t nk = n * k;
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE + 1;
    // one workspace plan for every stage (the knn stage reuses the front of the workspace)
    WsPlan plan;
    const size_t i_knn = plan.add(gs_knn_ws_bytes(ctx, n, d));
    const size_t i_idx = plan.add(sizeof(int) * nk), i_d64 = plan.add(sizeof(double) * nk),
                 i_cnt = plan.add(sizeof(int) * n), i_cur = plan.add(sizeof(int) * n),
                 i_inp = plan.add(sizeof(int64_t) * (n + 1)), i_ins = plan.add(sizeof(int) * nk),
                 i_ind = plan.add(sizeof(double) * nk), i_rp = plan.add(sizeof(int64_t) * (n + 1)),
                 i_sum = plan.add(sizeof(int64_t) * nb), i_ed = plan.add(sizeof(double) * 2 * nk),
                 i_sel = plan.add(sizeof(SelState) * 2), i_hist = plan.add(sizeof(unsigned) * 256),
                 i_sig = plan.add(sizeof(double) * 2), i_bad = plan.add(sizeof(int));
    (void)i_knn;
    gs_status st = gs_ws_ensure(ctx, plan.total);
    if (st != GS_OK) return st;
    cudaStream_t s = ctx->stream;
    int* idx = ws_at<int>(ctx, plan, i_idx);
    double* d64 = ws_at<double>(ctx, plan, i_d64);
    int* cnt = ws_at<int>(ctx, plan, i_cnt);
    int* cur = ws_at<int>(ctx, plan, i_cur);
    int64_t* inptr = ws_at<int64_t>(ctx, plan, i_inp);
    int* in_src = ws_at<int>(ctx, plan, i_ins);
    double* in_d = ws_at<double>(ctx, plan, i_ind);
    int64_t* rp64 = ws_at<int64_t>(ctx, plan, i_rp);
    int64_t* sums = ws_at<int64_t>(ctx, plan, i_sum);
    double* ed = ws_at<double>(ctx, plan, i_ed);
    SelState* sel = ws_at<SelState>(ctx, plan, i_sel);
    unsigned* hist = ws_at<unsigned>(ctx, plan, i_hist);
    double* sig = ws_at<double>(ctx, plan, i_sig);
    int* bad = ws_at<int>(ctx, plan, i_bad);

    // 0: the points' coordinate bisection into the persistent loop's partition, used by the kNN
    // screen's sweep and by the node order; in its own allocation (the stages below reuse the
    // workspace)
    void* obuf = nullptr;
    int* ord = nullptr;
    const size_t obytes = gs_points_order_bytes(ctx, n, d);
    if (obytes && cudaMalloc(&obuf, obytes) != cudaSuccess) {
        cudaGetLastError();
        obuf = nullptr;  // the kNN and the reordering compute their own
    }
    struct FreeOnExit {
        void* p;
        ~FreeOnExit() { cudaFree(p); }
    } free_obuf{obuf};
    if (obuf && (st = gs_points_order(ctx, X, n, d, obuf, obytes, &ord)) != GS_OK) return st;

    // 1-2: kNN (front of the workspace holds norms and candidates)
    if ((st = gs_knn_launch(ctx, X, n, d, k, idx, nullptr, d64, ord)) != GS_OK) return st;

    // 3: sigma
    if (sigma > 0.f) {
        set_scalar<<<1, 1, 0, s>>>(sig, (double)sigma);
        gs_count(ctx, 1);
    } else {
        const long long N = nk;
        const long long rhi = N / 2, rlo = (N % 2 == 0) ? N / 2 - 1 : N / 2;
        const long long ranks[2] = {rlo, rhi};
        const unsigned hb = nblk(N, 256) < 1024 ? nblk(N, 256) : 1024;
        for (int which = 0; which < 2; ++which) {
            sel_init<<<1, 256, 0, s>>>(sel + which, ranks[which], hist);
            for (int shift = 56; shift >= 0; shift -= 8) {
                sel_hist<<<hb, 256, 0, s>>>(reinterpret_cast<const unsigned long long*>(d64), N,
                                            sel + which, shift, hist);
                sel_pick<<<1, 256, 0, s>>>(sel + which, hist, shift);
            }
        }
        sel_median<<<1, 1, 0, s>>>(sel, sel + 1, (int)(N % 2 == 0), sig);
        gs_count(ctx, 2 * 17 + 1);
    }

    // 4: in-lists, sorted out-lists, union count
    cudaMemsetAsync(cnt, 0, sizeof(int) * n, s);
    cudaMemsetAsync(cur, 0, sizeof(int) * n, s);
    in_count<<<nblk(nk, 256), 256, 0, s>>>(idx, nk, cnt);
    gs_exclusive_scan(s, cnt, n, inptr, sums);
    in_fill<<<nblk(nk, 256), 256, 0, s>>>(idx, d64, n, k, inptr, cur, in_src, in_d);
    sort_rows_by_col<<<nblk(n, 128), 128, 0, s>>>(n, inptr, 0, in_src, in_d);
    sort_rows_by_col<<<nblk(n, 128), 128, 0, s>>>(n, nullptr, k, idx, d64);
    union_rows<false><<<nblk(n, 128), 128, 0, s>>>(n, k, idx, d64, inptr, in_src, in_d, cnt,
                                                    nullptr, nullptr, nullptr, nullptr, nullptr,
                                                    nullptr);
    gs_exclusive_scan(s, cnt, n, rp64, sums);
    gs_count(ctx, 11);
    int64_t nnz = 0;
    double hsig[1] = {0.0};
    cudaMemcpyAsync(&nnz, rp64 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(hsig, sig, sizeof(double), cudaMemcpyDeviceToHost, s);
    if ((st = gs_cuda_check(ctx, cudaStreamSynchronize(s), "graph build (sizes)")) != GS_OK) return st;
    if (nnz >= ((int64_t)1 << 31)) return gs_fail(ctx, GS_ERR_UNSUPPORTED, "graph has >= 2^31 edges");
    if (!(hsig[0] > 0.0) || !isfinite(hsig[0]))
        return gs_fail(ctx, GS_ERR_ARG, "sigma is not positive (duplicate points?)");

    gs_graph* g = nullptr;
    if ((st = gs_graph_alloc(ctx, n, nnz, &g)) != GS_OK) return st;
    g->sigma = hsig[0];
    rowptr_to32<<<nblk(n + 1, 256), 256, 0, s>>>(n + 1, rp64, g->rowptr);
    union_rows<true><<<nblk(n, 128), 128, 0, s>>>(n, k, idx, d64, inptr, in_src, in_d, nullptr,
                                                   rp64, g->col, g->aval, ed, g->deg, sig);
    cudaMemsetAsync(bad, 0, sizeof(int), s);
    normalise_from_fp64<<<nblk(n * 32, 256), 256, 0, s>>>(n, g->rowptr, g->col, ed, g->deg, g->pval, bad);
    gs_count(ctx, 3);
    int hbad = 0;
    cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if ((st = gs_cuda_check(ctx, cudaStreamSynchronize(s), "graph build")) != GS_OK) {
        gs_graph_destroy(g);
        return st;
    }
    if (hbad) {
        gs_graph_destroy(g);
        return gs_fail(ctx, GS_ERR_ARG, "graph has a node with zero degree");
    }
    if ((st = gs_graph_reorder(ctx, g, X, d, ord)) != GS_OK) {
        gs_graph_destroy(g);
        return st;
    }
    *out = g;
    return GS_OK;
}
