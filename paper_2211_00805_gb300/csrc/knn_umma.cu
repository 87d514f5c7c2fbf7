// kNN candidate screen on the fifth-generation tensor cores (tcgen05 + TMA + TMEM).
//
// The graph of Sec. 4 needs, for every point, its k nearest neighbours among all n points; the
// distance tile |q - c|^2 = |q|^2 + |c|^2 - 2 q.c is a dense contraction over the features.  The
// norms are folded into that contraction by augmenting the vectors,
//     q' = (q, 1, |q|^2),   c' = (-2 c, |c|^2, 1),   q'.c' = |q - c|^2,
// so the tensor cores produce the squared distances directly.  FP32-grade products come from the
// 3xTF32 split x = hi + lo (both TF32): q'.c' ~ lo(q').hi(c') + hi(q').lo(c') + hi(q').hi(c'),
// accumulated in FP32 in tensor memory.  The screen keeps, per query, the 32 smallest screened
// distances (ties to the lower index); the FP64 rerank in knn.cu then fixes the exact k-list.
//
// One CTA owns 128 queries (the MMA's M) and streams all candidates in tiles of 256 (its N: the
// widest MMA, which does the most work per instruction).  All CTAs sweep the candidate tiles in
// the same order, so the CTAs resident at one time read the same tile and it is served from L2
// after its first fetch:
//   warp 0    TMA producer: the query operands once, then the candidates unit by unit (one unit =
//             the hi and lo boxes of one 32-feature K-block of one tile, 64 KB) into two shared
//             stages, so one unit's copy runs while the MMAs read the other (a stage is refilled
//             once the MMAs have released it);
//   warp 1    TMEM owner and MMA issuer (one thread): per unit 3 MMAs of 128 x 256 x 8 for each
//             of its k-steps (3 x ceil((d+2)/8) per tile) into one of two TMEM accumulators, then
//             commits to the stage's "empty" barrier and, after a tile's last unit, to the
//             accumulator's "full" barrier;
//   warps 2-5 epilogue: thread = query row = TMEM lane; reads the tile's 256 distances
//             (tcgen05.ld, 128 at a time), tests them against its current threshold in a compact
//             loop, inserts the rare hits into its top-32 list in shared memory (four groups of
//             eight with their maxima, so an insertion rescans eight entries), frees the
//             accumulator.
// Operands are K-major with the 128-byte swizzle that TMA writes and the MMA descriptors read.
// Every wait is bounded by a clock budget; a timeout sets GS_FLAG_TIMEOUT and the CTA drains its
// own copies and MMAs (bounded again) before it frees tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "gs_internal.cuh"

namespace {

constexpr int UM = 128;                 // queries per CTA (MMA M = TMEM lanes)
constexpr int UN = 256;                 // candidates per tile (MMA N = accumulator columns)
constexpr int UKB = 32;                 // features per K-block: one 128-byte swizzle row of FP32
constexpr int UTHREADS = 192;           // 6 warps
constexpr int BOXA = UM * 128;          // bytes of one query K-block box (128 rows x 128 B)
constexpr int BOX = UN * 128;           // bytes of one candidate K-block box (128 rows x 128 B)
constexpr int STAGES = 2;               // candidate units (one K-block of one tile) in shared memory
constexpr int NACC = 2;                 // accumulators in tensor memory
constexpr int UHALF = 128;              // columns the epilogue reads per pass (registers)
constexpr int LIST = 32;                // screened candidates per query
constexpr int TMEM_COLS = NACC * UN;    // 512 columns: all of tensor memory
constexpr long long kBudget = 2000000000ll;  // clock cycles per wait (~1 s)

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(b)) : "memory");
}
// Wait for the phase of parity `par` to complete; false when the budget runs out.  Each try_wait
// may suspend the thread in hardware until the phase completes (or a 20 us hint passes), so the
// waiting producer and MMA threads take fewer issue slots from the epilogue warps.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned par)
{
    const uint32_t a = su32(b);
    long long t0 = -1;
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, P;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(par), "r"(20000u)
            : "memory");
        if (done) return true;
        const long long t = clock64();
        if (t0 < 0) t0 = t;
        else if (t - t0 > kBudget) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}


// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address (16-byte units)
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused when swizzled)
    d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                           // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                           // swizzle: 128 B
    return d;
}

// Instruction descriptor, kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t umma_idesc_tf32(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
        "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// Per-thread top-32 list in shared memory, entry e of query row r at [e * UM + r], kept as four
// groups of eight whose worst entries (largest (distance, index)) are cached per group in scalar
// registers (no indexed register arrays, so nothing goes to local memory).
struct TopList {
    float* d;
    int* i;
    int row;
    float gd0, gd1, gd2, gd3;
    int gi0, gi1, gi2, gi3, gp0, gp1, gp2, gp3;
    float thr;  // distance of the worst entry overall
    int thr_i;  // its index
    int wg;     // its group

    __device__ __forceinline__ static bool worse(float da, int ia, float db, int ib)
    {
        return da > db || (da == db && ia > ib);
    }
    __device__ __forceinline__ void init(float* dl, int* il, int r)
    {
        d = dl;
        i = il;
        row = r;
        for (int e = 0; e < LIST; ++e) {
            d[e * UM + r] = INFINITY;
            i[e * UM + r] = 0x7fffffff;
        }
        gd0 = gd1 = gd2 = gd3 = INFINITY;
        gi0 = gi1 = gi2 = gi3 = 0x7fffffff;
        gp0 = gp1 = gp2 = gp3 = 0;
        thr = INFINITY;
        thr_i = 0x7fffffff;
        wg = 0;
    }

    // Replace the worst entry by (dv, iv), rescan its group, find the new worst group.  A
    // candidate enters when it ranks before the worst entry in the (distance, index) order.
    __device__ __forceinline__ void insert(float dv, int iv)
    {
        const int g = wg;
        const int p = g == 0 ? gp0 : (g == 1 ? gp1 : (g == 2 ? gp2 : gp3));
        const int base = g * 8;
        d[(base + p) * UM + row] = dv;
        i[(base + p) * UM + row] = iv;
        float md = d[base * UM + row];
        int mi = i[base * UM + row], mp = 0;
#pragma unroll
        for (int e = 1; e < 8; ++e) {
            const float de = d[(base + e) * UM + row];
            const int ie = i[(base + e) * UM + row];
            if (worse(de, ie, md, mi)) {
                md = de;
                mi = ie;
                mp = e;
            }
        }
        if (g == 0) { gd0 = md; gi0 = mi; gp0 = mp; }
        else if (g == 1) { gd1 = md; gi1 = mi; gp1 = mp; }
        else if (g == 2) { gd2 = md; gi2 = mi; gp2 = mp; }
        else { gd3 = md; gi3 = mi; gp3 = mp; }
        float bd = gd0;
        int bi = gi0, w = 0;
        if (worse(gd1, gi1, bd, bi)) { bd = gd1; bi = gi1; w = 1; }
        if (worse(gd2, gi2, bd, bi)) { bd = gd2; bi = gi2; w = 2; }
        if (worse(gd3, gi3, bd, bi)) { bd = gd3; bi = gi3; w = 3; }
        wg = w;
        thr = bd;
        thr_i = bi;
    }
};

template <int KB>
struct UmmaLayout {
    static constexpr int A = 0;                                  // [hi, lo][KB] query boxes
    static constexpr int B = A + 2 * KB * BOXA;                  // [stage][hi, lo] boxes of one K-block
    static constexpr int LD = B + STAGES * 2 * BOX;              // list distances [32][UM]
    static constexpr int LI = LD + LIST * UM * 4;                // list indices [32][UM]
    static constexpr int NBAR = 2 + 2 * STAGES + 2 * NACC;
    static constexpr int BAR = LI + LIST * UM * 4;               // NBAR mbarriers
    static constexpr int TSLOT = BAR + NBAR * 8;                 // TMEM address
    static constexpr int BYTES = TSLOT + 16;
    static constexpr int ALLOC = BYTES + 1024;                   // slack for 1024-byte alignment
};

template <int KB>
__global__ void __launch_bounds__(UTHREADS, 1)
    knn_screen_umma(const __grid_constant__ CUtensorMap tq_hi, const __grid_constant__ CUtensorMap tq_lo,
                    const __grid_constant__ CUtensorMap tc_hi, const __grid_constant__ CUtensorMap tc_lo,
                    int n, int ksteps, const int* __restrict__ ord, int* __restrict__ cand,
                    int* __restrict__ flags)
{
    using L = UmmaLayout<KB>;
    extern __shared__ unsigned char um_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(um_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    __shared__ int s_ok;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
    uint64_t* full_a = bar + 0;
    uint64_t* drain = bar + 1;
    uint64_t* full = bar + 2;                    // [STAGES]
    uint64_t* empty = full + STAGES;             // [STAGES]
    uint64_t* accf = empty + STAGES;             // [NACC]
    uint64_t* acce = accf + NACC;                // [NACC]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::TSLOT);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q0 = blockIdx.x * UM;
    const int ntiles = (n + UN - 1) / UN;
    const int nunits = ntiles * KB;
    // Points in the bisection order (ord: position -> point): each CTA starts its sweep at the tile
    // holding its own queries, whose neighbours mostly lie in the same part of the bisection, so its
    // top-32 thresholds fall within the first tiles and later tiles rarely insert.  Points in the
    // caller's order: all CTAs sweep in the same order.  Either way the CTAs resident at one time
    // read few distinct tiles, served from L2.
    const int rot = ord ? (int)(((int64_t)blockIdx.x * UM / UN) % ntiles) : 0;
    auto tile_of = [rot, ntiles](int t) { const int u = t + rot; return u >= ntiles ? u - ntiles : u; };

    if (threadIdx.x == 0) {
        s_ok = 1;
        mbar_init(full_a, 1);
        mbar_init(drain, 1);
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, 1);  // one MMA commit
        }
        for (int i = 0; i < NACC; ++i) {
            mbar_init(accf + i, 1);
            mbar_init(acce + i, 4 * 32);
        }
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            bool ok = true;
            mbar_expect_tx(full_a, 2 * KB * BOXA);
            for (int kb = 0; kb < KB; ++kb) {
                tma_load_2d(sm + L::A + kb * BOXA, &tq_hi, kb * UKB, q0, full_a);
                tma_load_2d(sm + L::A + (KB + kb) * BOXA, &tq_lo, kb * UKB, q0, full_a);
            }
            // unit u = K-block u % KB of tile u / KB: its hi and lo boxes into stage u % STAGES,
            // so the next unit's copy runs while the MMAs read the other stage
            int issued = 0;
            for (int u = 0; u < nunits; ++u) {
                const int s = u % STAGES;
                if (u >= STAGES && !mbar_wait(empty + s, ((u / STAGES) - 1) & 1)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(full + s, 2 * BOX);
                unsigned char* st = sm + L::B + s * 2 * BOX;
                const int y = tile_of(u / KB) * UN, kb = u % KB;
                tma_load_2d(st, &tc_hi, kb * UKB, y, full + s);
                tma_load_2d(st + BOX, &tc_lo, kb * UKB, y, full + s);
                issued = u + 1;
            }
            // every copy into this CTA has landed and the MMAs have released the last stages
            // before the CTA may exit
            for (int u = (issued > STAGES ? issued - STAGES : 0); u < issued; ++u) {
                if (!mbar_wait(full + u % STAGES, (u / STAGES) & 1)) ok = false;
                if (!mbar_wait(empty + u % STAGES, (u / STAGES) & 1)) ok = false;
            }
            if (!mbar_wait(full_a, 0)) ok = false;
            if (!ok) {
                atomicOr(flags, GS_FLAG_TIMEOUT);
                s_ok = 0;
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc_tf32(UM, UN);
            bool ok = mbar_wait(full_a, 0);
            const uint32_t a_hi = su32(sm + L::A), a_lo = su32(sm + L::A + KB * BOXA);
            for (int u = 0; ok && u < nunits; ++u) {
                const int s = u % STAGES, t = u / KB, kb = u % KB, b = t % NACC;
                if (!mbar_wait(full + s, (u / STAGES) & 1)) { ok = false; break; }
                if (kb == 0 && t >= NACC && !mbar_wait(acce + b, ((t / NACC) - 1) & 1)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tbase + (uint32_t)(b * UN);
                const uint32_t b_hi = su32(sm + L::B + s * 2 * BOX);
                const uint32_t b_lo = b_hi + BOX;
                const int ks1 = 4 * kb + 4 < ksteps ? 4 * kb + 4 : ksteps;  // this K-block's k-steps
                for (int ks = 4 * kb; ks < ks1; ++ks) {
                    const uint32_t offa = (uint32_t)(kb * BOXA + (ks & 3) * 32);
                    const uint32_t offb = (uint32_t)((ks & 3) * 32);
                    const uint64_t ah = sw128_desc(a_hi + offa), al = sw128_desc(a_lo + offa);
                    const uint64_t bh = sw128_desc(b_hi + offb), bl = sw128_desc(b_lo + offb);
                    umma_tf32(d_tmem, al, bh, idesc, ks > 0 ? 1u : 0u);
                    umma_tf32(d_tmem, ah, bl, idesc, 1u);
                    umma_tf32(d_tmem, ah, bh, idesc, 1u);
                }
                umma_commit(empty + s);
                if (kb == KB - 1) umma_commit(accf + b);
            }
            // all MMAs issued by this thread have completed before tensor memory is freed
            umma_commit(drain);
            if (!mbar_wait(drain, 0)) ok = false;
            if (!ok) {
                atomicOr(flags, GS_FLAG_TIMEOUT);
                s_ok = 0;
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int quad = warp & 3;  // TMEM lanes this warp may read: [32 quad, 32 quad + 32)
        const int row = quad * 32 + lane;
        const int q = q0 + row;
        TopList tl;
        tl.init(reinterpret_cast<float*>(sm + L::LD), reinterpret_cast<int*>(sm + L::LI), row);
        // rows past n (zero-filled by TMA) score 0 against everything: they test nothing
        if (q >= n) tl.thr = -INFINITY;
        const int qo = (q < n && ord) ? __ldg(ord + q) : q;  // the query's own index
        bool ok = true;
        for (int t = 0; t < ntiles; ++t) {
            const int b = t % NACC;
            // warp-uniform outcome: the tensor-memory loads below are warp-collective
            if (!__all_sync(0xffffffffu, mbar_wait(accf + b, (t / NACC) & 1))) { ok = false; break; }
            tc_fence_after();
            const uint32_t ta = tbase + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * UN);
            for (int hb = 0; hb < UN; hb += UHALF) {  // one pass per UHALF columns
                float v[UHALF / 32][32];
                __syncwarp();
#pragma unroll
                for (int h = 0; h < UHALF / 32; ++h) tmem_ld32(ta + (uint32_t)(hb + 32 * h), v[h]);
                tmem_wait_ld();
                // per chunk of 32: the minimum (a depth-5 tree; the chunks' trees are independent, so
                // they overlap) against the threshold; most chunks have no hit, and the rare hits
                // are inserted one at a time through a single copy of the insertion code
                float mn[UHALF / 32];
#pragma unroll
                for (int h = 0; h < UHALF / 32; ++h) {
                    float m16[16], m8[8], m4[4];
#pragma unroll
                    for (int j = 0; j < 16; ++j) m16[j] = fminf(v[h][j], v[h][j + 16]);
#pragma unroll
                    for (int j = 0; j < 8; ++j) m8[j] = fminf(m16[j], m16[j + 8]);
#pragma unroll
                    for (int j = 0; j < 4; ++j) m4[j] = fminf(m8[j], m8[j + 4]);
                    mn[h] = fminf(fminf(m4[0], m4[2]), fminf(m4[1], m4[3]));
                }
#pragma unroll
                for (int h = 0; h < UHALF / 32; ++h) {
                    if (!(mn[h] <= tl.thr)) continue;
                    const int cbase = tile_of(t) * UN + hb + 32 * h;
                    uint32_t hits = 0;
#pragma unroll
                    for (int j = 0; j < 32; ++j) hits |= (v[h][j] <= tl.thr) ? (1u << j) : 0u;
                    while (hits) {
                        const int j = __ffs(hits) - 1;
                        hits &= hits - 1;
                        float dv = v[h][0];
#pragma unroll
                        for (int jj = 1; jj < 32; ++jj) dv = (jj == j) ? v[h][jj] : dv;
                        const int ci = cbase + j;
                        if (ci >= n || ci == q || !(dv <= tl.thr)) continue;
                        const int co = ord ? __ldg(ord + ci) : ci;  // the candidate's own index
                        if (dv < tl.thr || co < tl.thr_i) tl.insert(dv, co);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acce + b);
        }
        if (!ok) {
            atomicOr(flags, GS_FLAG_TIMEOUT);
            s_ok = 0;
        }
        if (q < n) {
            for (int e = 0; e < LIST; ++e) cand[(int64_t)qo * LIST + e] = tl.i[e * UM + row];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(TMEM_COLS)
                     : "memory");
    }
}

// Augmented 3xTF32 operands: rows [n][32 KB] of q' = (x, 1, |x|^2) and c' = (-2x, |x|^2, 1), row r
// holding point ord[r] (or r).
__global__ void umma_operands(const float* __restrict__ X, const float* __restrict__ norms, int64_t n,
                              int d, int w, const int* __restrict__ ord, float* __restrict__ qh,
                              float* __restrict__ ql, float* __restrict__ ch, float* __restrict__ cl)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * w) return;
    const int64_t rr = e / w;
    const int j = (int)(e - rr * w);
    const int64_t r = ord ? (int64_t)ord[rr] : rr;
    float qv = 0.f, cv = 0.f;
    if (j < d) {
        const float x = X[r * d + j];
        qv = x;
        cv = -2.f * x;
    } else if (j == d) {
        qv = 1.f;
        cv = norms[r];
    } else if (j == d + 1) {
        qv = norms[r];
        cv = 1.f;
    }
    unsigned h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(qv));
    float hv = __uint_as_float(h);
    qh[e] = hv;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(qv - hv));
    ql[e] = __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(cv));
    hv = __uint_as_float(h);
    ch[e] = hv;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(cv - hv));
    cl[e] = __uint_as_float(h);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

bool make_map(CUtensorMap* m, const float* base, int64_t n, int w, int rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)w, (cuuint64_t)n};
    const cuuint64_t strides[1] = {(cuuint64_t)w * sizeof(float)};
    const cuuint32_t box[2] = {UKB, (cuuint32_t)rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KB>
gs_status launch_umma(gs_ctx* ctx, const CUtensorMap* maps, int64_t n, int ksteps, const int* ord, int* cand)
{
    using L = UmmaLayout<KB>;
    static int ready = 0;  // 1 usable, -1 not
    if (!ready) {
        ready = cudaFuncSetAttribute(knn_screen_umma<KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::ALLOC) ==
                        cudaSuccess
                    ? 1
                    : -1;
        cudaGetLastError();
    }
    if (ready < 0) return GS_ERR_UNSUPPORTED;
    const unsigned grid = (unsigned)((n + UM - 1) / UM);
    knn_screen_umma<KB><<<grid, UTHREADS, L::ALLOC, ctx->stream>>>(maps[0], maps[1], maps[2], maps[3], (int)n,
                                                                   ksteps, ord, cand, ctx->flags);
    if (cudaGetLastError() != cudaSuccess) return GS_ERR_UNSUPPORTED;
    gs_count(ctx, 1);
    return GS_OK;
}

}  // namespace

bool gs_knn_umma_available() { return tensor_map_encoder() != nullptr; }

// Bytes of workspace the tensor-memory screen needs for n points of dimension d (0: not usable).
size_t gs_knn_umma_bytes(int64_t n, int d)
{
    if (d + 2 > 2 * UKB || n < 2 || n >= ((int64_t)1 << 31)) return 0;
    const int w = d + 2 <= UKB ? UKB : 2 * UKB;
    return 4 * ((size_t)n * w * sizeof(float) + 256);
}

// Screen the 32 nearest candidates of every point with the tensor-memory kernel.  `ws` holds
// gs_knn_umma_bytes(n, d) bytes (256-byte aligned); `norms` are the FP32 squared norms; `ord`
// (position -> point, or null) lays the points out in a spatial order for the sweep; lists and
// tie-breaking use the points' own indices either way.
// Returns GS_ERR_UNSUPPORTED (nothing enqueued) when the shape or the driver does not allow it.
gs_status gs_knn_screen_umma(gs_ctx* ctx, const float* X, const float* norms, int64_t n, int d,
                             unsigned char* ws, const int* ord, int* cand)
{
    if (!gs_knn_umma_bytes(n, d) || !tensor_map_encoder()) return GS_ERR_UNSUPPORTED;
    const int kb = d + 2 <= UKB ? 1 : 2;
    const int w = kb * UKB;
    const size_t arr = ((size_t)n * w * sizeof(float) + 255) / 256 * 256;
    float* qh = reinterpret_cast<float*>(ws);
    float* ql = reinterpret_cast<float*>(ws + arr);
    float* ch = reinterpret_cast<float*>(ws + 2 * arr);
    float* cl = reinterpret_cast<float*>(ws + 3 * arr);
    CUtensorMap maps[4];
    if (!make_map(&maps[0], qh, n, w, UM) || !make_map(&maps[1], ql, n, w, UM) || !make_map(&maps[2], ch, n, w, UN) ||
        !make_map(&maps[3], cl, n, w, UN))
        return GS_ERR_UNSUPPORTED;
    umma_operands<<<(unsigned)((n * w + 255) / 256), 256, 0, ctx->stream>>>(X, norms, n, d, w, ord, qh, ql, ch, cl);
    gs_count(ctx, 1);
    const int ksteps = (d + 2 + 7) / 8;
    return kb == 1 ? launch_umma<1>(ctx, maps, n, ksteps, ord, cand) : launch_umma<2>(ctx, maps, n, ksteps, ord, cand);
}
