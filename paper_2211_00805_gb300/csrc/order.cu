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

// ------------------------------------------------------------------ coordinate bisection
// For a graph built from points, the nodes are ordered by recursive bisection of the point set:
// every segment of the order is split at a prescribed rank along its principal direction, so the
// final segments, one per block of the persistent loop, are compact regions of the point cloud
// (far fewer neighbours outside a block than the slabs of a breadth-first order).  The direction
// is estimated from an evenly spaced sample of the segment (mean, then power iteration), every
// point is projected and binned, and the split takes the bins below the rank's bin, and inside
// that bin the points in their current order, so it is exact and deterministic.
constexpr int kRcbBins = 4096;
constexpr int kRcbChunk = 1024;
constexpr int kRcbMaxDim = 128;   // larger dimensions keep the breadth-first order
constexpr int kRcbSampleFloats = 24576;  // sample size x dimension held in shared memory
constexpr int kRcbPower = 8;
constexpr int kRcbMaxPart = 4096;  // rows of a part for the in-part degree sort

struct RcbSeg {
    int beg, len, left;  // positions [beg, beg + len); the first `left` go to the left child
    int chunk0, nchunk;  // its chunks of kRcbChunk positions
};
struct RcbChunk {
    int seg, beg, count;
};

constexpr int kRcbStatThreads = 1024;

__global__ void __launch_bounds__(kRcbStatThreads) rcb_stats(const float* __restrict__ X, int d, const int* __restrict__ ord,
                                                 const RcbSeg* __restrict__ segs, float* __restrict__ mean,
                                                 float* __restrict__ dir, float* __restrict__ range)
{
    extern __shared__ float r_smem[];
    const RcbSeg sg = segs[blockIdx.x];
    const int S = min(sg.len, kRcbSampleFloats / d);
    float* Y = r_smem;            // [S][d]
    float* mu = Y + S * d;        // [d]
    float* v = mu + d;            // [d]
    float* w = v + d;             // [d]
    float* pr = w + d;            // [S]
    int* node = reinterpret_cast<int*>(pr + S);  // [S]
    __shared__ float s_norm;
    __shared__ float part[kRcbStatThreads];  // per (dimension, sample phase) partial sums
    const int R = d < kRcbStatThreads ? kRcbStatThreads / d : 1;  // sample phases per dimension
    for (int i = threadIdx.x; i < S; i += blockDim.x) node[i] = ord[sg.beg + (int)(((long long)i * sg.len) / S)];
    __syncthreads();
#pragma unroll 4
    for (int e = threadIdx.x; e < S * d; e += blockDim.x) {
        const int i = e / d, j = e - i * d;
        Y[e] = X[(int64_t)node[i] * d + j];
    }
    __syncthreads();
    // column sums over the samples: thread (j, r) adds samples r, r + R, ..., then the R partials
    // of each column are added in phase order
    auto column_sums = [&](const float* wt, float* out) {
        for (int t = threadIdx.x; t < d * R; t += blockDim.x) {
            const int j = t % d, r = t / d;
            float acc = 0.f;
            for (int i = r; i < S; i += R) acc = wt ? fmaf(wt[i], Y[i * d + j], acc) : acc + Y[i * d + j];
            if (R > 1) part[t] = acc;
            else out[j] = acc;
        }
        __syncthreads();
        if (R > 1) {
            for (int j = threadIdx.x; j < d; j += blockDim.x) {
                float acc = 0.f;
                for (int r = 0; r < R; ++r) acc += part[r * d + j];
                out[j] = acc;
            }
            __syncthreads();
        }
    };
    column_sums(nullptr, mu);
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        mu[j] /= (float)S;
        v[j] = 1.f + 0.01f * (float)(j % 7);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < S * d; e += blockDim.x) Y[e] -= mu[e % d];
    __syncthreads();
    for (int it = 0; it <= kRcbPower; ++it) {
        for (int i = threadIdx.x; i < S; i += blockDim.x) {
            float acc = 0.f;
            for (int j = 0; j < d; ++j) acc = fmaf(Y[i * d + j], v[j], acc);
            pr[i] = acc;
        }
        __syncthreads();
        if (it == kRcbPower) break;
        column_sums(pr, w);
        if (threadIdx.x == 0) {
            float nn = 0.f;
            for (int j = 0; j < d; ++j) nn = fmaf(w[j], w[j], nn);
            s_norm = sqrtf(nn);
        }
        __syncthreads();
        if (s_norm > 0.f)
            for (int j = threadIdx.x; j < d; j += blockDim.x) v[j] = w[j] / s_norm;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        float lo = pr[0], hi = pr[0];
        for (int i = 1; i < S; ++i) {
            lo = fminf(lo, pr[i]);
            hi = fmaxf(hi, pr[i]);
        }
        range[2 * blockIdx.x] = lo;
        range[2 * blockIdx.x + 1] = hi;
    }
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        mean[(int64_t)blockIdx.x * d + j] = mu[j];
        dir[(int64_t)blockIdx.x * d + j] = v[j];
    }
}

__global__ void __launch_bounds__(kRcbChunk) rcb_bin(const float* __restrict__ X, int d, const int* __restrict__ ord,
                                                     const RcbChunk* __restrict__ chunks, const float* __restrict__ mean,
                                                     const float* __restrict__ dir, const float* __restrict__ range,
                                                     uint16_t* __restrict__ bin, int* __restrict__ hist)
{
    extern __shared__ float b_smem[];  // [d] mean, [d] direction
    const RcbChunk ch = chunks[blockIdx.x];
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        b_smem[j] = mean[(int64_t)ch.seg * d + j];
        b_smem[d + j] = dir[(int64_t)ch.seg * d + j];
    }
    __syncthreads();
    if ((int)threadIdx.x >= ch.count) return;
    const int pos = ch.beg + threadIdx.x;
    const float* x = X + (int64_t)ord[pos] * d;
    float acc = 0.f;
    for (int j = 0; j < d; ++j) acc = fmaf(x[j] - b_smem[j], b_smem[d + j], acc);
    const float lo = range[2 * ch.seg], hi = range[2 * ch.seg + 1];
    int b = 0;
    if (hi > lo) {
        const float f = (acc - lo) / (hi - lo) * (float)kRcbBins;
        b = f > 0.f ? (f < (float)(kRcbBins - 1) ? (int)f : kRcbBins - 1) : 0;  // NaN -> bin 0
    }
    bin[pos] = (uint16_t)b;
    atomicAdd(&hist[(int64_t)ch.seg * kRcbBins + b], 1);
}

// per segment: the bin holding rank `left` (sel[0]) and how many of that bin go left (sel[1])
__global__ void __launch_bounds__(256) rcb_select(const RcbSeg* __restrict__ segs, const int* __restrict__ hist,
                                                  int* __restrict__ sel)
{
    __shared__ int part[256];
    const int* h = hist + (int64_t)blockIdx.x * kRcbBins;
    constexpr int per = kRcbBins / 256;
    int c = 0;
    for (int q = 0; q < per; ++q) c += h[threadIdx.x * per + q];
    part[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int left = segs[blockIdx.x].left;
        int below = 0, t = 0;
        while (t < 255 && below + part[t] < left) below += part[t++];
        int b = t * per;
        while (b < kRcbBins - 1 && below + h[b] < left) below += h[b++];
        sel[2 * blockIdx.x] = b;
        sel[2 * blockIdx.x + 1] = left - below;
    }
}

__device__ __forceinline__ int rcb_block_excl(int flag, int* warp_tot, int* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, flag);
    if (lane == 0) warp_tot[w] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            const int t = warp_tot[i];
            warp_tot[i] = run;
            run += t;
        }
        *total = run;
    }
    __syncthreads();
    const int r = warp_tot[w] + __popc(m & ((1u << lane) - 1u));
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kRcbChunk) rcb_count(const RcbChunk* __restrict__ chunks, const uint16_t* __restrict__ bin,
                                                       const int* __restrict__ sel, int* __restrict__ cnt)
{
    __shared__ int wt[kRcbChunk / 32];
    __shared__ int tot;
    const RcbChunk ch = chunks[blockIdx.x];
    const bool act = (int)threadIdx.x < ch.count;
    const int b = act ? bin[ch.beg + threadIdx.x] : 0;
    const int bs = sel[2 * ch.seg];
    rcb_block_excl(act && b < bs, wt, &tot);
    const int lt = tot;
    rcb_block_excl(act && b == bs, wt, &tot);
    if (threadIdx.x == 0) {
        cnt[2 * blockIdx.x] = lt;
        cnt[2 * blockIdx.x + 1] = tot;
    }
}

// per chunk: equal-bin elements before it in its segment, and its left / right output bases
__global__ void rcb_bases(const RcbSeg* __restrict__ segs, const RcbChunk* __restrict__ chunks, int nseg,
                          const int* __restrict__ sel, const int* __restrict__ cnt, int* __restrict__ base)
{
    const int sgi = blockIdx.x * blockDim.x + threadIdx.x;
    if (sgi >= nseg) return;
    const RcbSeg sg = segs[sgi];
    const int need = sel[2 * sgi + 1];
    int eq = 0, lb = 0, rb = 0;
    for (int c = sg.chunk0; c < sg.chunk0 + sg.nchunk; ++c) {
        const int lt = cnt[2 * c], e = cnt[2 * c + 1];
        const int eq_left = need - eq <= 0 ? 0 : (need - eq >= e ? e : need - eq);
        base[3 * c] = eq;
        base[3 * c + 1] = lb;
        base[3 * c + 2] = rb;
        eq += e;
        lb += lt + eq_left;
        rb += chunks[c].count - lt - eq_left;
    }
}

__global__ void __launch_bounds__(kRcbChunk) rcb_scatter(const RcbChunk* __restrict__ chunks,
                                                         const RcbSeg* __restrict__ segs, const int* __restrict__ ord,
                                                         const uint16_t* __restrict__ bin, const int* __restrict__ sel,
                                                         const int* __restrict__ base, int* __restrict__ ord_new)
{
    __shared__ int wt[kRcbChunk / 32];
    __shared__ int tot;
    const RcbChunk ch = chunks[blockIdx.x];
    const RcbSeg sg = segs[ch.seg];
    const bool act = (int)threadIdx.x < ch.count;
    const int pos = ch.beg + threadIdx.x;
    const int b = act ? bin[pos] : 0;
    const int bs = sel[2 * ch.seg], need = sel[2 * ch.seg + 1];
    const int eq_rank = rcb_block_excl(act && b == bs, wt, &tot);
    const bool L = act && (b < bs || (b == bs && base[3 * blockIdx.x] + eq_rank < need));
    const int l_rank = rcb_block_excl(L, wt, &tot);
    if (!act) return;
    const int r_rank = (int)threadIdx.x - l_rank;
    const int dst = L ? sg.beg + base[3 * blockIdx.x + 1] + l_rank : sg.beg + sg.left + base[3 * blockIdx.x + 2] + r_rank;
    ord_new[dst] = ord[pos];
}

__global__ void rcb_iota(int64_t n, int* __restrict__ ord)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) ord[i] = (int)i;
}

// The part (block of the persistent loop's partition) of every node: part_of[perm[pos]] = b for the
// positions pos of part b.
__global__ void part_of_fill(const int* __restrict__ parts, const int* __restrict__ perm, int* __restrict__ part_of)
{
    const int beg = parts[blockIdx.x], end = parts[blockIdx.x + 1];
    for (int i = beg + threadIdx.x; i < end; i += blockDim.x) part_of[perm[i]] = blockIdx.x;
}

// Order inside each part: eight degree classes, largest degrees first (rows of similar degree
// share a slice, so the sliced ELL pads little); inside a class by the smallest other part holding
// one of the row's neighbours, so the rows one neighbouring block reads sit together and its
// staging loads of their exchanged values touch fewer 32-byte sectors; then by decreasing degree,
// then in the order given.  (Against the plain degree sort: 2.22 against 2.27 us per order of the
// persistent loop on the 100k manifold graph, the same partition.)  Rank counting in shared
// memory, one block per part.
constexpr int kDegreeClasses = 8;
// by_reader = 0: decreasing degree only (then in the order given).
__global__ void __launch_bounds__(256) part_reader_sort(const int* __restrict__ parts, int nparts, int by_reader,
                                                        const int* __restrict__ perm_in,
                                                        const int* __restrict__ rowptr, const int* __restrict__ col,
                                                        const int* __restrict__ part_of, int* __restrict__ perm_out)
{
    extern __shared__ int psm[];  // degree [len], reader [len], class [len]
    const int beg = parts[blockIdx.x], len = parts[blockIdx.x + 1] - beg;
    int* pdeg = psm;
    int* prd = psm + len;
    int* pcls = psm + 2 * len;
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const int node = perm_in[beg + i];
        const int e0 = rowptr[node], e1 = rowptr[node + 1];
        int r = nparts;
        for (int e = by_reader ? e0 : e1; e < e1; ++e) {
            const int q = part_of[col[e]];
            if (q != (int)blockIdx.x && q < r) r = q;
        }
        pdeg[i] = e1 - e0;
        prd[i] = r;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const int di = pdeg[i];
        int above = 0;  // rows of larger degree: equal degrees share a class
        for (int j = 0; j < len; ++j) above += pdeg[j] > di;
        pcls[i] = by_reader ? (int)((int64_t)above * kDegreeClasses / len) : 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const int ci = pcls[i], ri = prd[i], di = pdeg[i];
        int rank = 0;
        for (int j = 0; j < len; ++j) {
            const int cj = pcls[j], rj = prd[j], dj = pdeg[j];
            rank += cj < ci || (cj == ci && (rj < ri || (rj == ri && (dj > di || (dj == di && j < i)))));
        }
        perm_out[beg + rank] = perm_in[beg + i];
    }
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

// Recursive coordinate bisection of the points X [n, d] into the parts [parts[b], parts[b+1]) of
// the order: *result (ord or ord2, n ints each) receives position -> point.  Every level is a
// handful of launches with no host synchronisation.
static gs_status rcb_points(gs_ctx* ctx, const float* X, int64_t n, int d, const std::vector<int>& parts,
                            int* ord, int* ord2, void* scratch, size_t scratch_bytes, int** result)
{
    cudaStream_t s = ctx->stream;
    const int P = (int)parts.size() - 1;
    const int max_chunks = (int)((n + kRcbChunk - 1) / kRcbChunk) + P;
    // scratch layout
    size_t off = 0;
    auto take = [&](size_t bytes) {
        void* q = static_cast<char*>(scratch) + off;
        off = (off + bytes + 255) & ~size_t(255);
        return q;
    };
    uint16_t* bin = static_cast<uint16_t*>(take(sizeof(uint16_t) * (size_t)n));
    int* hist = static_cast<int*>(take(sizeof(int) * (size_t)P * kRcbBins));
    float* mean = static_cast<float*>(take(sizeof(float) * (size_t)P * d));
    float* dir = static_cast<float*>(take(sizeof(float) * (size_t)P * d));
    float* range = static_cast<float*>(take(sizeof(float) * 2 * (size_t)P));
    int* sel = static_cast<int*>(take(sizeof(int) * 2 * (size_t)P));
    int* cnt = static_cast<int*>(take(sizeof(int) * 2 * (size_t)max_chunks));
    int* base = static_cast<int*>(take(sizeof(int) * 3 * (size_t)max_chunks));
    RcbSeg* segs_d = static_cast<RcbSeg*>(take(sizeof(RcbSeg) * (size_t)P));
    RcbChunk* chunks_d = static_cast<RcbChunk*>(take(sizeof(RcbChunk) * (size_t)max_chunks));
    if (off > scratch_bytes) return gs_fail(ctx, GS_ERR_OOM, "bisection scratch");

    const int S_max = kRcbSampleFloats / d;
    const size_t stats_smem = sizeof(float) * ((size_t)S_max * d + 3 * (size_t)d + 2 * (size_t)S_max);
    cudaFuncSetAttribute(rcb_stats, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stats_smem);
    rcb_iota<<<nblk(n, 256), 256, 0, s>>>(n, ord);
    gs_count(ctx, 1);
    struct Node {
        int beg, len, pa, pb;
    };
    std::vector<Node> cur{{0, (int)n, 0, P}};
    std::vector<RcbSeg> segs;
    std::vector<RcbChunk> chunks;
    while (true) {
        std::vector<Node> next;
        segs.clear();
        chunks.clear();
        for (const Node& nd : cur) {
            if (nd.pb - nd.pa <= 1) continue;
            const int mid = (nd.pa + nd.pb) / 2;
            const int left = parts[(size_t)mid] - parts[(size_t)nd.pa];
            next.push_back({nd.beg, left, nd.pa, mid});
            next.push_back({nd.beg + left, nd.len - left, mid, nd.pb});
            if (left <= 0 || left >= nd.len) continue;  // nothing moves
            const int nc = (nd.len + kRcbChunk - 1) / kRcbChunk;
            segs.push_back({nd.beg, nd.len, left, (int)chunks.size(), nc});
            for (int c = 0; c < nc; ++c)
                chunks.push_back({(int)segs.size() - 1, nd.beg + c * kRcbChunk, std::min(kRcbChunk, nd.len - c * kRcbChunk)});
        }
        if (next.empty()) break;
        const int ns = (int)segs.size(), nc = (int)chunks.size();
        if (ns > 0) {
            // pageable copies: staged before the calls return, so the vectors may change afterwards
            cudaMemcpyAsync(segs_d, segs.data(), sizeof(RcbSeg) * ns, cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(chunks_d, chunks.data(), sizeof(RcbChunk) * nc, cudaMemcpyHostToDevice, s);
            cudaMemsetAsync(hist, 0, sizeof(int) * (size_t)ns * kRcbBins, s);
            rcb_stats<<<ns, kRcbStatThreads, stats_smem, s>>>(X, d, ord, segs_d, mean, dir, range);
            rcb_bin<<<nc, kRcbChunk, sizeof(float) * 2 * d, s>>>(X, d, ord, chunks_d, mean, dir, range, bin, hist);
            rcb_select<<<ns, 256, 0, s>>>(segs_d, hist, sel);
            rcb_count<<<nc, kRcbChunk, 0, s>>>(chunks_d, bin, sel, cnt);
            rcb_bases<<<(ns + 127) / 128, 128, 0, s>>>(segs_d, chunks_d, ns, sel, cnt, base);
            cudaMemcpyAsync(ord2, ord, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, s);
            rcb_scatter<<<nc, kRcbChunk, 0, s>>>(chunks_d, segs_d, ord, bin, sel, base, ord2);
            gs_count(ctx, 6);
            std::swap(ord, ord2);
        }
        cur.swap(next);
    }
    *result = ord;
    return gs_cuda_check(ctx, cudaGetLastError(), "coordinate bisection");
}

// Scratch bytes of rcb_points for n points of dimension d in P parts.
static size_t rcb_scratch_bytes(int64_t n, int d, int64_t P)
{
    const int64_t chunks = (n + kRcbChunk - 1) / kRcbChunk + P;
    return (size_t)(2 * n + 4 * P * kRcbBins + 8 * P * (d > 0 ? d : 1) + 16 * P + 20 * chunks + 12 * chunks +
                    24 * P + 4 * (P + 1) + 16 * 256);
}

// The persistent loop's partition of n rows when the points can be bisected into it (each part
// small enough for the in-part degree sort), else empty.
static std::vector<int> rcb_parts(const gs_ctx* ctx, int64_t n, int d)
{
    const int blocks = gs_persist_cache_blocks(ctx);
    if (d < 1 || d > kRcbMaxDim || blocks < 2 || n < 2) return {};
    std::vector<int> parts = gs_equal_slice_rows(n, blocks);
    for (int b = 0; b < blocks; ++b)
        if (parts[(size_t)b + 1] - parts[(size_t)b] > kRcbMaxPart) return {};
    return parts;
}

size_t gs_points_order_bytes(const gs_ctx* ctx, int64_t n, int d)
{
    const std::vector<int> parts = rcb_parts(ctx, n, d);
    if (parts.empty()) return 0;
    return sizeof(int) * 2 * (size_t)n + 256 + rcb_scratch_bytes(n, d, (int64_t)parts.size() - 1);
}

gs_status gs_points_order(gs_ctx* ctx, const float* X, int64_t n, int d, void* buf, size_t bytes, int** ord)
{
    *ord = nullptr;
    const std::vector<int> parts = rcb_parts(ctx, n, d);
    if (parts.empty() || bytes < gs_points_order_bytes(ctx, n, d)) return GS_OK;
    int* a = static_cast<int*>(buf);
    int* b = a + n;
    void* scratch = static_cast<char*>(buf) + ((sizeof(int) * 2 * (size_t)n + 255) & ~(size_t)255);
    return rcb_points(ctx, X, n, d, parts, a, b, scratch, rcb_scratch_bytes(n, d, (int64_t)parts.size() - 1), ord);
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

gs_status gs_graph_reorder(gs_ctx* ctx, gs_graph* g, const float* X, int d, const int* points_order)
{
    const int64_t n = g->n, nnz = g->nnz;
    WsPlan plan;
    const size_t i_owner = plan.add(sizeof(int) * n), i_cnt = plan.add(sizeof(int) * n),
                 i_offs = plan.add(sizeof(int64_t) * (n + 1)),
                 i_sums = plan.add(sizeof(int64_t) * (n / 4096 + 2)), i_int = plan.add(sizeof(int) * 4),
                 i_p64 = plan.add(sizeof(int64_t) * (n + 1)), i_hflag = plan.add(sizeof(int) * n),
                 i_h64 = plan.add(sizeof(int64_t) * (n + 1));
    // coordinate bisection scratch (bins, histograms, per-segment statistics, chunk tables)
    const int64_t P_ = gs_persist_cache_blocks(ctx);
    const size_t rcb_bytes = (X != nullptr && !points_order) ? rcb_scratch_bytes(n, d, P_) : 0;
    const size_t i_rcb = plan.add(rcb_bytes > 0 ? rcb_bytes : 1);
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
    // points given: recursive coordinate bisection into the persistent loop's partition (when the
    // parts fit the in-part sort); otherwise the breadth-first order
    const int blocks = gs_persist_cache_blocks(ctx);
    const std::vector<int> parts = X != nullptr ? rcb_parts(ctx, n, d) : std::vector<int>();
    const bool rcb = !parts.empty();
    if (rcb) {
        // the bisection order of the points (given, or computed here), then inside each part the
        // degree-class and reader order
        const int* ord = points_order;
        if (!ord) {
            int* res = nullptr;
            if ((st = rcb_points(ctx, X, n, d, parts, owner, cnt, ws_at<void>(ctx, plan, i_rcb), rcb_bytes, &res)) !=
                GS_OK)
                return st;
            ord = res;
        }
        const int P = (int)parts.size() - 1;
        int maxpart = 0;
        for (int b = 0; b < P; ++b) maxpart = std::max(maxpart, parts[(size_t)b + 1] - parts[(size_t)b]);
        int* parts_d = reinterpret_cast<int*>(p64);  // free until the permuted CSR below (P + 1 <= n + 1)
        cudaMemcpyAsync(parts_d, parts.data(), sizeof(int) * ((size_t)P + 1), cudaMemcpyHostToDevice, s);
        int* part_of = hflag;  // n ints, free until the long-row flags below
        part_of_fill<<<P, 256, 0, s>>>(parts_d, ord, part_of);
        cudaFuncSetAttribute(part_reader_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(int) * 3 * maxpart));
        part_reader_sort<<<P, 256, sizeof(int) * 3 * std::max(maxpart, 1), s>>>(parts_d, P, ctx->node_order, ord,
                                                                                  g->rowptr, g->col, part_of, g->perm);
        gs_count(ctx, 2);
        g->levels = 0;
        invert_perm<<<nblk(n, 256), 256, 0, s>>>(n, g->perm, g->iperm);
        gs_count(ctx, 1);
    } else {
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
    return gs_graph_build_xcache(ctx, g, blocks, rcb ? &parts : nullptr);
}
