// Per-block gather cache for the persistent Sinkhorn loop.
//
// The persistent kernel gives block b a contiguous range of whole slices of rows, [rows[b],
// rows[b+1]), the ranges holding about equal numbers of sliced-ELL entries.  In the one-column filter each nonzero gathers cur[col]; within one block many
// nonzeros share a column.  This pass lists, once per graph, the distinct columns of every block's
// sliced-ELL entries (sorted) and rewrites each entry's column as a 16-bit index into that list.
// Per Chebyshev order the block then copies cur[] at its distinct columns into shared memory (one
// load per distinct column, in increasing address order) and every nonzero reads its neighbour
// value from shared memory.  The same pass lists, per block, the other blocks that own one of those
// columns: the blocks whose results this block reads in every order (and, the pattern being
// symmetric, the blocks that read this block's results), which is what the persistent loop waits
// for between orders instead of a barrier over the whole grid.
#include <stdint.h>

#include <new>

#include "gs_internal.cuh"

namespace {

constexpr int kXcMaxEntries = 32768;  // sort capacity per block (and the 16-bit index range)
constexpr int kXcMaxBlocks = 1024;    // partition blocks (one per SM)

__global__ void __launch_bounds__(1024) xcache_build(const int* __restrict__ sptr,
                                                     const int* __restrict__ scol, int64_t nslices,
                                                     const int* __restrict__ rows, int64_t n, int P,
                                                     int* __restrict__ ucol, int* __restrict__ ucnt,
                                                     uint16_t* __restrict__ lidx,
                                                     int* __restrict__ deps, int* __restrict__ ndeps)
{
    extern __shared__ int keys[];  // [P]
    __shared__ int wsum[32];
    __shared__ int mark[kXcMaxBlocks];
    __shared__ int s_rows[kXcMaxBlocks + 1];
    __shared__ int s_nd;
    const int tid = threadIdx.x, b = blockIdx.x;
    const int nb = (int)gridDim.x;
    for (int i = tid; i <= nb; i += blockDim.x) s_rows[i] = rows[i];
    __syncthreads();
    const int64_t r0 = s_rows[b];
    const int64_t r1 = s_rows[b + 1];
    if (r0 >= r1) {
        if (tid == 0) ucnt[b] = 0;
        if (tid == 0) ndeps[b] = 0;
        return;
    }
    const int64_t s0 = r0 / GS_SELL_C;
    int64_t s1 = (r1 + GS_SELL_C - 1) / GS_SELL_C;
    s1 = s1 < nslices ? s1 : nslices;
    const int e0 = sptr[s0], e1 = sptr[s1];
    const int E = e1 - e0;
    if (E > P) {  // sized from the largest block, so this cannot happen; never write past keys[]
        if (tid == 0) ucnt[b] = -1;
        if (tid == 0) ndeps[b] = 0;
        return;
    }
    __shared__ int s_bad;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int i = tid; i < P; i += blockDim.x) {
        const int c = i < E ? scol[e0 + i] : 0x7fffffff;
        if (i < E && (c < 0 || c >= n)) s_bad = 1;
        keys[i] = c;
    }
    __syncthreads();
    if (s_bad) {  // a column outside [0, n): no cache for this graph
        if (tid == 0) ucnt[b] = -1;
        if (tid == 0) ndeps[b] = 0;
        return;
    }
    // bitonic sort, ascending
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const int a = keys[i], c = keys[ixj];
                    if ((a > c) == up) {
                        keys[i] = c;
                        keys[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    // distinct values: exclusive scan of "first of a run" flags over contiguous chunks per thread
    const int chunk = (P + blockDim.x - 1) / blockDim.x;
    const int i0 = tid * chunk, i1 = (i0 + chunk) < P ? (i0 + chunk) : P;
    int cnt = 0;
    for (int i = i0; i < i1; ++i)
        cnt += (keys[i] != 0x7fffffff) && (i == 0 || keys[i] != keys[i - 1]);
    int incl = cnt;
    const int lane = tid & 31, w = tid >> 5;
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += o;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        int v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, v, off);
            if (lane >= off) v += o;
        }
        wsum[lane] = v;  // inclusive prefix over warps
    }
    __syncthreads();
    int pos = incl - cnt + (w > 0 ? wsum[w - 1] : 0);
    for (int i = i0; i < i1; ++i) {
        if ((keys[i] != 0x7fffffff) && (i == 0 || keys[i] != keys[i - 1])) ucol[e0 + pos++] = keys[i];
    }
    const int total = wsum[(blockDim.x >> 5) - 1];
    if (tid == 0) ucnt[b] = total;
    __syncthreads();
    // each entry's position in the block's distinct list (binary search; the list is sorted)
    for (int e = e0 + tid; e < e1; e += blockDim.x) {
        const int c = scol[e];
        int lo = 0, hi = total - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (ucol[e0 + mid] < c) lo = mid + 1;
            else hi = mid;
        }
        lidx[e] = (uint16_t)lo;
    }
    // blocks owning one of the distinct columns (other than this one), in increasing order
    for (int i = tid; i < nb; i += blockDim.x) mark[i] = 0;
    if (tid == 0) s_nd = 0;
    __syncthreads();
    for (int i = tid; i < total; i += blockDim.x) {
        const int c = ucol[e0 + i];
        int lo = 0, hi = nb - 1;  // the block o with rows[o] <= c < rows[o + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_rows[mid] <= c) lo = mid;
            else hi = mid - 1;
        }
        if (lo != b) mark[lo] = 1;
    }
    __syncthreads();
    if (tid < 32) {
        for (int base = 0; base < nb; base += 32) {
            const int i = base + tid;
            const bool m = i < nb && mark[i];
            const unsigned bal = __ballot_sync(0xffffffffu, m);
            if (m) deps[(int64_t)b * nb + s_nd + __popc(bal & ((1u << tid) - 1u))] = i;
            __syncwarp();
            if (tid == 0) s_nd += __popc(bal);
            __syncwarp();
        }
        if (tid == 0) ndeps[b] = s_nd;
    }
}


// Bank assignment of the gather-cache slots.  Slot i of a block's cache sits in shared-memory bank
// i mod 32, and a slice's step conflicts where two lanes read different slots of one bank; no
// order of the entries within the rows can do better than the slice's most-used bank.  The slots
// of every aligned group of 32 distinct columns may be permuted freely: a warp's staging loads
// still cover the same 32 columns (the same cache lines) and its staging stores still hit 32
// distinct banks.  Within each group the columns with the most entries choose first, each taking
// the free bank least used so far by the slices it occurs in, which evens out every slice's bank
// counts.  Four warps take four consecutive groups per round against the counts of the rounds
// before (so the result does not depend on timing), then add their choices to the counts.
constexpr int kAssignMaxSlices = 64;  // blocks with more slices keep the sorted slots
constexpr int kAssignWarps = 4;

__global__ void __launch_bounds__(32 * kAssignWarps) xcache_bank_assign(const int* __restrict__ sptr, int64_t nslices,
                                                                        const int* __restrict__ rows,
                                                                        const int* __restrict__ ucnt,
                                                                        int* __restrict__ ucol,
                                                                        uint16_t* __restrict__ lidx)
{
    extern __shared__ int a_smem[];
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t r0 = rows[b], r1 = rows[b + 1];
    const int U = ucnt[b];
    if (r0 >= r1 || U <= 1) return;
    const int64_t s0 = r0 / GS_SELL_C;
    int64_t s1 = (r1 + GS_SELL_C - 1) / GS_SELL_C;
    s1 = s1 < nslices ? s1 : nslices;
    const int nsl = (int)(s1 - s0);
    if (nsl > kAssignMaxSlices) return;
    const int e0 = sptr[s0], E = sptr[s1] - e0;
    int* off = a_smem;                                       // [U + 1] column -> its entries
    int* cur = off + (U + 1);                                // [U] fill cursors, then new slots
    unsigned* bank_use = reinterpret_cast<unsigned*>(cur + U);         // [nsl][32]
    int* cost_s = reinterpret_cast<int*>(bank_use + nsl * 32);         // [kAssignWarps][32][32]
    unsigned char* ent_slice = reinterpret_cast<unsigned char*>(cost_s + kAssignWarps * 1024);  // [E]
    const int nt = 32 * kAssignWarps;
    // the slices each column occurs in (with multiplicity), grouped by column
    for (int i = tid; i <= U; i += nt) off[i] = 0;
    for (int i = tid; i < nsl * 32; i += nt) bank_use[i] = 0;
    __syncthreads();
    for (int e = tid; e < E; e += nt) atomicAdd(&off[lidx[e0 + e] + 1], 1);
    __syncthreads();
    if (w == 0) {  // inclusive scan of off[1..U]
        int carry = 0;
        for (int base = 1; base <= U; base += 32) {
            const int i = base + lane;
            int v = i <= U ? off[i] : 0;
            for (int d = 1; d < 32; d <<= 1) {
                const int o = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d) v += o;
            }
            if (i <= U) off[i] = v + carry;
            carry += __shfl_sync(0xffffffffu, v, 31);
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = tid; i < U; i += nt) cur[i] = off[i];
    __syncthreads();
    for (int sl = w; sl < nsl; sl += kAssignWarps) {
        const int e1 = sptr[s0 + sl + 1] - e0;
        for (int e = sptr[s0 + sl] - e0 + lane; e < e1; e += 32)
            ent_slice[atomicAdd(&cur[lidx[e0 + e]], 1)] = (unsigned char)sl;
    }
    __syncthreads();
    int* cost = cost_s + w * 1024;  // [column in group][bank]
    for (int r0g = 0; r0g < U; r0g += 32 * kAssignWarps) {
        const int g0 = r0g + 32 * w;
        const int k = g0 < U ? min(32, U - g0) : 0;
        const int my = g0 + lane;
        int bank = lane;
        if (k > 0) {
            // every column's cost per bank against the counts of the earlier rounds
            for (int c = 0; c < k; ++c) {
                int sum = 0;
                for (int q = off[g0 + c]; q < off[g0 + c + 1]; ++q) sum += (int)bank_use[ent_slice[q] * 32 + lane];
                cost[c * 32 + lane] = sum;
            }
            // rank of this lane's column: more entries first, ties to the lower column
            const int weight = lane < k ? off[my + 1] - off[my] : -1;
            int rank = 0;
            for (int j = 0; j < 32; ++j) {
                const int wj = __shfl_sync(0xffffffffu, weight, j);
                rank += (wj > weight) || (wj == weight && j < lane);
            }
            __syncwarp();
            unsigned freeb = k == 32 ? 0xffffffffu : ((1u << k) - 1u);
            for (int it = 0; it < k; ++it) {
                const int col = __ffs(__ballot_sync(0xffffffffu, rank == it)) - 1;
                int key = ((freeb >> lane) & 1u) ? (cost[col * 32 + lane] << 5) | lane : 0x7fffffff;
                for (int d = 16; d > 0; d >>= 1) key = min(key, __shfl_xor_sync(0xffffffffu, key, d));
                const int bk = key & 31;
                if (lane == col) bank = bk;
                freeb &= ~(1u << bk);
            }
        }
        __syncthreads();
        if (lane < k) {
            for (int q = off[my]; q < off[my + 1]; ++q) atomicAdd(&bank_use[ent_slice[q] * 32 + bank], 1u);
        }
        // move the group's columns to their slots; cur[] maps old slot -> new slot
        const int c = lane < k ? ucol[e0 + my] : 0;
        __syncwarp();
        if (lane < k) {
            ucol[e0 + g0 + bank] = c;
            cur[my] = g0 + bank;
        }
        __syncthreads();
    }
    for (int e = tid; e < E; e += nt) lidx[e0 + e] = (uint16_t)cur[lidx[e0 + e]];
}

// Bank-aware order of the entries of every 32-row slice.  In the persistent loop a warp sums one
// slice, lane = row, step j = the j-th stored entry of every row, reading the neighbour value from
// the block's gather cache at its 16-bit local index; lanes whose indices share a shared-memory
// bank (index mod 32) serialise.  The entries of a row may be summed in any order, so the steps
// are a free choice: an assignment of steps to the entries in which every row uses each step once
// and, ideally, every bank at most once per step.  That is an edge colouring of the bipartite
// multigraph rows x banks with as many colours as the slice is wide, which exists whenever no
// bank has more entries than that (Koenig's edge-colouring theorem); the construction adds the
// edges one at a time, and where no colour is free at both ends it swaps the two colours along
// the alternating path from the bank end (Kempe chain), which in a bipartite graph never reaches
// the row end.  Entries beyond a full bank take any colour left free at their row (a conflict).
// One thread per slice; the steps go to `step`, and a second pass moves column, value and local
// index together, so every kernel reading the sliced ELL sums each row in the same (new) order.
constexpr int kSchedMaxWidth = 64;
constexpr unsigned char kNone = 0xff;

__host__ __device__ inline int lowest_bit(unsigned long long m)
{
#ifdef __CUDA_ARCH__
    return __ffsll((long long)m) - 1;
#else
    return __builtin_ctzll(m);
#endif
}

// Steps for one slice of width W (1..64): lx = the slice's local indices ([W][32], entry j of row
// l at j * 32 + l), st = the step of every entry (same layout).  Always a permutation of the steps
// within every row: should the construction ever leave a row incomplete, the slice keeps its order.
struct ColourWork {
    unsigned char lane_at[32][kSchedMaxWidth];  // row l, colour c -> entry j (or none)
    unsigned char bank_at[32][kSchedMaxWidth];  // bank b, colour c -> row (or none); then counts
    unsigned long long lane_free[32], bank_free[32], over[32];
    int deg[32];
    unsigned char worst[kSchedMaxWidth];
    unsigned char pl[64], pj[64], pb[64], pc[64];  // an alternating path
    unsigned char bank_of[kSchedMaxWidth][32];     // bank of entry j of row l
};

__host__ __device__ inline void colour_slice(const uint16_t* lx, int W, unsigned char* st, ColourWork& wk)
{
    auto& lane_at = wk.lane_at;
    auto& bank_at = wk.bank_at;
    auto& lane_free = wk.lane_free;
    auto& bank_free = wk.bank_free;
    auto& over = wk.over;
    auto& deg = wk.deg;
    const unsigned long long full = W == 64 ? ~0ull : ((1ull << W) - 1ull);
    for (int i = 0; i < 32; ++i) {
        lane_free[i] = full;
        bank_free[i] = full;
        over[i] = 0ull;
        deg[i] = 0;
        for (int c = 0; c < W; ++c) {
            lane_at[i][c] = kNone;
            bank_at[i][c] = kNone;
        }
    }
    auto& bank_of = wk.bank_of;
    for (int e = 0; e < W * 32; ++e) bank_of[e >> 5][e & 31] = (unsigned char)(lx[e] & 31);
    for (int j = 0; j < W; ++j)
        for (int l = 0; l < 32; ++l) {
            const int bk = bank_of[j][l];
            if (++deg[bk] > W) over[l] |= 1ull << j;  // entries beyond a full bank: left for the end
        }
    for (int j = 0; j < W; ++j) {
        for (int l = 0; l < 32; ++l) {
            if ((over[l] >> j) & 1ull) continue;
            const int bk = bank_of[j][l];
            const unsigned long long both = lane_free[l] & bank_free[bk];
            int c;
            if (both) {
                c = lowest_bit(both);
            } else {
                const int a = lowest_bit(lane_free[l]);    // free at the row, used at the bank
                const int bb = lowest_bit(bank_free[bk]);  // free at the bank, used at the row
                // the a/bb path from the bank: bank -a-> row -bb-> bank -a-> ...; swap a and bb on it
                auto& pl = wk.pl;
                auto& pj = wk.pj;
                auto& pb = wk.pb;
                auto& pc = wk.pc;
                int len = 0;
                int vb = bk;
                while (len < 63) {
                    const int x = bank_at[vb][a];
                    if (x == kNone) break;
                    pl[len] = (unsigned char)x; pj[len] = lane_at[x][a]; pb[len] = (unsigned char)vb; pc[len] = (unsigned char)a;
                    ++len;
                    const int jy = lane_at[x][bb];
                    if (jy == kNone) break;
                    const int y = bank_of[jy][x];
                    pl[len] = (unsigned char)x; pj[len] = (unsigned char)jy; pb[len] = (unsigned char)y; pc[len] = (unsigned char)bb;
                    ++len;
                    vb = y;
                }
                for (int q = 0; q < len; ++q) {
                    lane_at[pl[q]][pc[q]] = kNone;
                    bank_at[pb[q]][pc[q]] = kNone;
                }
                for (int q = 0; q < len; ++q) {
                    const int nc = pc[q] == a ? bb : a;
                    lane_at[pl[q]][nc] = pj[q];
                    bank_at[pb[q]][nc] = pl[q];
                }
                const unsigned long long m = (1ull << a) | (1ull << bb);
                for (int q = 0; q < len; ++q) {
                    unsigned long long lf = lane_free[pl[q]] | m, bf = bank_free[pb[q]] | m;
                    if (lane_at[pl[q]][a] != kNone) lf &= ~(1ull << a);
                    if (lane_at[pl[q]][bb] != kNone) lf &= ~(1ull << bb);
                    if (bank_at[pb[q]][a] != kNone) bf &= ~(1ull << a);
                    if (bank_at[pb[q]][bb] != kNone) bf &= ~(1ull << bb);
                    lane_free[pl[q]] = lf;
                    bank_free[pb[q]] = bf;
                }
                if (!((lane_free[l] & bank_free[bk]) >> a & 1ull)) {  // not in a bipartite graph
                    over[l] |= 1ull << j;
                    continue;
                }
                c = a;
            }
            lane_at[l][c] = (unsigned char)j;
            bank_at[bk][c] = (unsigned char)l;
            lane_free[l] &= ~(1ull << c);
            bank_free[bk] &= ~(1ull << c);
        }
    }
    // the rest: the colour free at the row that raises the step's worst bank multiplicity least
    // (ties: the lower colour), so that the unavoidable conflicts share steps
    auto& mult = wk.bank_at;  // bank b, colour c -> entries (the rows are no longer needed)
    auto& worst = wk.worst;
    for (int c = 0; c < W; ++c) {
        worst[c] = 0;
        for (int b = 0; b < 32; ++b) {
            mult[b][c] = bank_at[b][c] != kNone ? 1 : 0;
            worst[c] = mult[b][c] > worst[c] ? mult[b][c] : worst[c];
        }
    }
    for (int l = 0; l < 32; ++l) {
        unsigned long long o = over[l];
        while (o) {
            const int j = lowest_bit(o);
            o &= o - 1ull;
            if (!lane_free[l]) break;
            const int bk = bank_of[j][l];
            int best = -1, best_inc = 1 << 30;
            for (unsigned long long f = lane_free[l]; f; f &= f - 1ull) {
                const int c = lowest_bit(f);
                const int inc = mult[bk][c] + 1 > worst[c] ? mult[bk][c] + 1 - worst[c] : 0;
                if (inc < best_inc) {
                    best_inc = inc;
                    best = c;
                    if (inc == 0) break;  // the lowest colour that costs nothing
                }
            }
            lane_at[l][best] = (unsigned char)j;
            lane_free[l] &= ~(1ull << best);
            if (mult[bk][best] < 255) mult[bk][best] += 1;
            if (mult[bk][best] > worst[best]) worst[best] = mult[bk][best];
        }
    }
    bool ok = true;
    for (int l = 0; l < 32 && ok; ++l) {
        unsigned long long seen = 0ull;
        for (int c = 0; c < W; ++c) {
            const int j = lane_at[l][c];
            if (j == kNone || j >= W || ((seen >> j) & 1ull)) {
                ok = false;
                break;
            }
            seen |= 1ull << j;
        }
    }
    for (int l = 0; l < 32; ++l)
        for (int c = 0; c < W; ++c) {
            if (ok) st[lane_at[l][c] * 32 + l] = (unsigned char)c;
            else st[c * 32 + l] = (unsigned char)c;
        }
}

// One slice per warp, worked by its first lane, its working arrays in shared memory (a few KB:
// in local memory they would not stay in L1).  Slices sharing a warp would serialise their
// data-dependent path searches; the kernel's time is the slowest slice's.
constexpr int kColourSlices = 4;  // per block

__global__ void __launch_bounds__(32 * kColourSlices) sell_bank_colour(const int* __restrict__ sptr, int64_t nslices,
                                                                       const uint16_t* __restrict__ lidx,
                                                                       unsigned char* __restrict__ step)
{
    extern __shared__ __align__(16) unsigned char c_smem[];
    ColourWork* wk = reinterpret_cast<ColourWork*>(c_smem);
    if ((threadIdx.x & 31) != 0) return;
    const int w = threadIdx.x >> 5;
    const int64_t sl = (int64_t)blockIdx.x * kColourSlices + w;
    if (sl >= nslices) return;
    const int base = sptr[sl];
    const int W = (sptr[sl + 1] - base) / 32;
    if (W < 1 || W > kSchedMaxWidth) return;
    colour_slice(lidx + base, W, step + base, wk[w]);
}

// Moves every entry of a slice to its step (from copies of the three arrays; slices too wide for
// the colouring keep their order) and writes the local indices in the paired layout the cached
// row sums read: steps 2q and 2q + 1 of row l in the 32-bit word q * 32 + l of the slice, an odd
// last step at its plain position.
__global__ void sell_apply_steps(const int* __restrict__ sptr, int64_t nslices, const unsigned char* __restrict__ step,
                                 const int* __restrict__ c_in, const float* __restrict__ v_in,
                                 const uint16_t* __restrict__ l_in, int* __restrict__ scol,
                                 float* __restrict__ sval, uint16_t* __restrict__ lidx)
{
    const int64_t sl = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (sl >= nslices) return;
    const int l = threadIdx.x & 31;
    const int base = sptr[sl];
    const int W = (sptr[sl + 1] - base) / 32;
    if (W < 1) return;
    const bool coloured = W <= kSchedMaxWidth;
    for (int j = 0; j < W; ++j) {
        const int e = base + j * 32 + l;
        const int t = coloured ? (int)step[e] : j;
        const int d = base + t * 32 + l;
        scol[d] = c_in[e];
        sval[d] = v_in[e];
        lidx[t < (W & ~1) ? base + (t >> 1) * 64 + 2 * l + (t & 1) : d] = l_in[e];
    }
}

}  // namespace

// Build the cache tables for the partition `rows` (whole slices per block).  Leaves g->xc_ok false
// when a block has more than kXcMaxEntries entries (the loop then uses its other forms).
static gs_status build_tables(gs_ctx* ctx, gs_graph* g, const std::vector<int>& rows)
{
    const int blocks = (int)rows.size() - 1;
    const int64_t ns = g->nslices;
    const std::vector<int>& sp = g->sptr_host;
    int64_t worst = 0, most_rows = 0;
    for (int b = 0; b < blocks; ++b) {
        const int64_t r0 = rows[(size_t)b], r1 = rows[(size_t)b + 1];
        if (r1 <= r0) continue;
        const int64_t s0 = r0 / GS_SELL_C, s1 = std::min<int64_t>(ns, (r1 + GS_SELL_C - 1) / GS_SELL_C);
        worst = std::max<int64_t>(worst, (int64_t)sp[(size_t)s1] - sp[(size_t)s0]);
        most_rows = std::max<int64_t>(most_rows, r1 - r0);
    }
    if (worst > kXcMaxEntries || worst == 0) return GS_OK;
    int P = 1;
    while (P < worst) P <<= 1;
    const size_t tot = (size_t)(g->sell_nnz > 0 ? g->sell_nnz : 1);
    cudaError_t e = cudaSuccess;
    if (!g->xc_ucol) e = cudaMalloc(&g->xc_ucol, sizeof(int) * tot);
    if (e == cudaSuccess && !g->xc_lidx) e = cudaMalloc(&g->xc_lidx, sizeof(uint16_t) * tot);
    if (e == cudaSuccess && !g->xc_ucnt) e = cudaMalloc(&g->xc_ucnt, sizeof(int) * blocks);
    if (e == cudaSuccess && !g->xc_deps) e = cudaMalloc(&g->xc_deps, sizeof(int) * (size_t)blocks * blocks);
    if (e == cudaSuccess && !g->xc_ndeps) e = cudaMalloc(&g->xc_ndeps, sizeof(int) * blocks);
    if (e == cudaSuccess && !g->xc_rows) e = cudaMalloc(&g->xc_rows, sizeof(int) * ((size_t)blocks + 1));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GS_OK;  // the cache is an optimisation; run without it
    }
    g->xc_rows_host = rows;
    cudaMemcpyAsync(g->xc_rows, g->xc_rows_host.data(), sizeof(int) * ((size_t)blocks + 1), cudaMemcpyHostToDevice,
                    ctx->stream);
    cudaMemsetAsync(g->xc_ucol, 0, sizeof(int) * tot, ctx->stream);
    cudaFuncSetAttribute(xcache_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(P * sizeof(int)));
    xcache_build<<<blocks, 1024, P * sizeof(int), ctx->stream>>>(g->sptr, g->scol, ns, g->xc_rows, g->n, P,
                                                                   g->xc_ucol, g->xc_ucnt, g->xc_lidx,
                                                                   g->xc_deps, g->xc_ndeps);
    gs_count(ctx, 1);
    g->xc_ucnt_host.assign((size_t)blocks, 0);
    std::vector<int> nd((size_t)blocks, 0);
    cudaMemcpyAsync(g->xc_ucnt_host.data(), g->xc_ucnt, sizeof(int) * blocks, cudaMemcpyDeviceToHost,
                    ctx->stream);
    cudaMemcpyAsync(nd.data(), g->xc_ndeps, sizeof(int) * blocks, cudaMemcpyDeviceToHost, ctx->stream);
    gs_status st = gs_cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "gather-cache tables");
    if (st != GS_OK) return st;
    for (int v : g->xc_ucnt_host)
        if (v < 0) return GS_OK;
    g->xc_blocks = blocks;
    g->xc_rpb = (int)most_rows;
    g->xc_max_e = (int)worst;
    g->xc_max_u = *std::max_element(g->xc_ucnt_host.begin(), g->xc_ucnt_host.end());
    g->xc_max_deps = *std::max_element(nd.begin(), nd.end());
    g->xc_ok = true;
    return GS_OK;
}

// Split whole slices into `blocks` contiguous ranges of about equal total weight.
static std::vector<int> balanced_rows(const std::vector<double>& w, int64_t n, int blocks)
{
    const size_t ns = w.size();
    std::vector<double> cum(ns + 1, 0.0);
    for (size_t s = 0; s < ns; ++s) cum[s + 1] = cum[s] + w[s];
    std::vector<int> rows((size_t)blocks + 1, 0);
    size_t s = 0;
    for (int b = 1; b < blocks; ++b) {
        const double target = cum[ns] * b / blocks;
        while (s < ns && cum[s] < target) ++s;
        rows[(size_t)b] = (int)std::min<int64_t>(n, (int64_t)s * GS_SELL_C);
    }
    rows[(size_t)blocks] = (int)n;
    return rows;
}

// Build the cache tables for a partition of the rows into `blocks` contiguous ranges of whole
// slices with about equal per-order work, so that no block of the persistent loop lags its
// neighbours.  A block's work is its sums (proportional to its sliced-ELL entries) plus its
// staging (proportional to its distinct columns, about four times as costly per item, measured);
// the distinct counts are known only once the tables exist, so the ranges are first balanced on
// entries, then re-balanced on entries plus four times the block's distinct count spread over
// its slices, and the tables rebuilt.  Then the entries of every slice are put in bank-aware order.
std::vector<int> gs_equal_slice_rows(int64_t n, int blocks)
{
    const int64_t ns = (n + GS_SELL_C - 1) / GS_SELL_C;
    return balanced_rows(std::vector<double>((size_t)ns, 1.0), n, blocks);
}

gs_status gs_graph_build_xcache(gs_ctx* ctx, gs_graph* g, int blocks, const std::vector<int>* parts)
{
    g->xc_ok = false;
    if (!g->sptr || g->sptr_host.empty() || blocks < 1 || blocks > kXcMaxBlocks) return GS_OK;
    const int64_t ns = g->nslices;
    const std::vector<int>& sp = g->sptr_host;
    std::vector<double> w((size_t)ns);
    for (int64_t i = 0; i < ns; ++i) w[(size_t)i] = (double)(sp[(size_t)i + 1] - sp[(size_t)i]);
    const bool fixed = parts != nullptr && (int)parts->size() == blocks + 1;
    gs_status st = build_tables(ctx, g, fixed ? *parts : balanced_rows(w, g->n, blocks));
    if (st != GS_OK || !g->xc_ok) return st;
    constexpr double kStageWeight = 4.0;
    for (int b = 0; b < blocks; ++b) {
        const int64_t s0 = g->xc_rows_host[(size_t)b] / GS_SELL_C;
        const int64_t s1 = std::min<int64_t>(ns, (g->xc_rows_host[(size_t)b + 1] + GS_SELL_C - 1) / GS_SELL_C);
        const double eb = (double)(sp[(size_t)s1] - sp[(size_t)s0]);
        if (eb <= 0.0) continue;
        const double per_entry = kStageWeight * g->xc_ucnt_host[(size_t)b] / eb;
        for (int64_t i = s0; i < s1; ++i) w[(size_t)i] *= 1.0 + per_entry;
    }
    const std::vector<int> rows = fixed ? *parts : balanced_rows(w, g->n, blocks);
    if (rows != g->xc_rows_host) {
        g->xc_ok = false;
        if ((st = build_tables(ctx, g, rows)) != GS_OK || !g->xc_ok) return st;
    }
    // cache slots spread over the banks, then the entries of each slice in bank-aware order (all
    // readers of the sliced ELL follow it)
    {
        int max_sl = 0;
        for (int b = 0; b < blocks; ++b) {
            const int64_t s0 = g->xc_rows_host[(size_t)b] / GS_SELL_C;
            const int64_t s1 = std::min<int64_t>(ns, (g->xc_rows_host[(size_t)b + 1] + GS_SELL_C - 1) / GS_SELL_C);
            max_sl = std::max<int>(max_sl, (int)(s1 - s0));
        }
        const size_t smem = sizeof(int) * (2 * (size_t)g->xc_max_u + 1) +
                            sizeof(unsigned) * 32 * (size_t)std::min(max_sl, kAssignMaxSlices) +
                            sizeof(int) * kAssignWarps * 1024 + (size_t)g->xc_max_e + 16;
        if (smem <= 200 * 1024) {
            cudaFuncSetAttribute(xcache_bank_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            xcache_bank_assign<<<blocks, 32 * kAssignWarps, smem, ctx->stream>>>(g->sptr, ns, g->xc_rows, g->xc_ucnt,
                                                                 g->xc_ucol, g->xc_lidx);
            gs_count(ctx, 1);
        }
    }
    {
        const size_t ne = (size_t)g->sell_nnz;
        WsPlan plan;
        const size_t i_step = plan.add(ne), i_c = plan.add(sizeof(int) * ne), i_v = plan.add(sizeof(float) * ne),
                     i_l = plan.add(sizeof(uint16_t) * ne);
        if ((st = gs_ws_ensure(ctx, plan.total)) != GS_OK) return st;
        unsigned char* stp = ws_at<unsigned char>(ctx, plan, i_step);
        int* c_in = ws_at<int>(ctx, plan, i_c);
        float* v_in = ws_at<float>(ctx, plan, i_v);
        uint16_t* l_in = ws_at<uint16_t>(ctx, plan, i_l);
        cudaStream_t s = ctx->stream;
        cudaMemcpyAsync(c_in, g->scol, sizeof(int) * ne, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(v_in, g->sval, sizeof(float) * ne, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(l_in, g->xc_lidx, sizeof(uint16_t) * ne, cudaMemcpyDeviceToDevice, s);
        cudaFuncSetAttribute(sell_bank_colour, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(ColourWork) * kColourSlices));
        sell_bank_colour<<<(unsigned)((ns + kColourSlices - 1) / kColourSlices), 32 * kColourSlices,
                           sizeof(ColourWork) * kColourSlices, s>>>(g->sptr, ns, l_in, stp);
        sell_apply_steps<<<(unsigned)((ns + 7) / 8), 256, 0, s>>>(g->sptr, ns, stp, c_in, v_in, l_in, g->scol,
                                                                   g->sval, g->xc_lidx);
        gs_count(ctx, 2);
    }
    return gs_cuda_check(ctx, cudaGetLastError(), "gather-cache tables");
}

extern "C" gs_status gs_sell_step_order(const uint16_t* idx, int W, unsigned char* steps)
{
    if (idx == nullptr || steps == nullptr || W < 1 || W > kSchedMaxWidth) return GS_ERR_ARG;
    ColourWork* wk = new (std::nothrow) ColourWork;
    if (wk == nullptr) return GS_ERR_OOM;
    colour_slice(idx, W, steps, *wk);
    delete wk;
    return GS_OK;
}
