// Autotuner: picks, per graph and column count, the fastest Chebyshev-order kernel variant (and
// for one column the Sinkhorn loop mode) by timing them on the graph itself, and stores the choice
// in the graph handle.  Calls on that graph use the stored choice whenever the context's own
// option is left at automatic.
#include <vector>

#include "gs_internal.cuh"

namespace {

__global__ void fill_ones(int64_t count, float* __restrict__ x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) x[i] = 1.f / (1.f + (float)(i % 97));
}

}  // namespace

gs_status gs_autotune_impl(gs_ctx* ctx, gs_graph* g, int B, int K, int* choice_out)
{
    const int64_t n = g->n;
    const size_t blk = sizeof(float) * (size_t)n * (size_t)B;
    WsPlan plan;
    const size_t iV = plan.add(blk), iY = plan.add(blk), iA = plan.add(blk), iBb = plan.add(blk);
    gs_status st = gs_ws_ensure(ctx, plan.total);
    if (st != GS_OK) return st;
    float* V = ws_at<float>(ctx, plan, iV);
    float* Y = ws_at<float>(ctx, plan, iY);
    float* bufA = ws_at<float>(ctx, plan, iA);
    float* bufB = ws_at<float>(ctx, plan, iBb);
    const int64_t count = n * (int64_t)B;
    fill_ones<<<(unsigned)((count + 255) / 256), 256, 0, ctx->stream>>>(count, V);
    gs_count(ctx, 1);
    std::vector<double> c((size_t)K + 1);
    gs_heat_coefficients(1.0, K, c.data());

    // candidates: (order variant, lanes) where lanes is the RHS tile width of the row-group
    // kernels (lanes per row; each lane walks ceil(B / (lanes x vec)) chunks) for B > 1, and the
    // threads per row of the row-split kernel for B == 1 (0: the variant's own mapping)
    struct Cand {
        int kernel, lanes;
    };
    std::vector<Cand> cands;
    if (B == 1) {
        cands = {{GS_KERNEL_RANGED, 0}, {GS_KERNEL_SM_RANGE, 0}, {GS_KERNEL_SPLIT, 2}, {GS_KERNEL_SPLIT, 4},
                 {GS_KERNEL_SPLIT, 8}, {GS_KERNEL_SELL, 0},     {GS_KERNEL_VECTOR, 0}, {GS_KERNEL_ASYNC, 0}};
    } else {
        const int vec = (B % 4 == 0) ? 4 : 1;  // the workspace blocks below are 16-byte aligned
        int full = B / vec;
        if (full > 32) full = 32;
        int p2 = 1;
        while (p2 * 2 <= full) p2 *= 2;
        full = p2;
        std::vector<int> widths = {full};
        if (full >= 2 && (B + (full / 2) * vec - 1) / ((full / 2) * vec) <= 8) widths.push_back(full / 2);
        for (int w : widths) {
            cands.push_back({GS_KERNEL_VECTOR, w});
            cands.push_back({GS_KERNEL_RANGED, w});
        }
        if (B == 32 || B == 64 || B == 128) {
            cands.push_back({GS_KERNEL_GROUP_WARP, 0});
            cands.push_back({GS_KERNEL_GROUP_VEC4, 0});
        }
        if (B % 4 == 0 && B <= 128) {
            cands.push_back({GS_KERNEL_STAGED, 0});
            cands.push_back({GS_KERNEL_ASYNC, 0});
        }
    }
    int* knob = (B == 1) ? &ctx->b1_kernel : &ctx->blk_kernel;
    const int saved = *knob, saved_lanes = ctx->lanes_override;
    const int saved_tb1 = g->tuned_b1, saved_tblk = g->tuned_blk, saved_tB = g->tuned_blk_B;
    const int saved_split = g->tuned_split, saved_tlanes = g->tuned_lanes;
    g->tuned_b1 = 0;
    g->tuned_blk = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    Cand best = cands[0];
    float best_ms = 1e30f;
    for (const Cand& cd : cands) {
        *knob = cd.kernel;
        ctx->lanes_override = cd.lanes;
        Epilogue e;
        e.kind = EPI_STORE;
        e.out = Y;
        // warm once, then time three applies
        st = gs_filter_enqueue(ctx, g, c.data(), K, B, V, false, bufA, bufB, Y, e, nullptr, nullptr);
        if (st != GS_OK) break;
        cudaEventRecord(e0, ctx->stream);
        for (int r = 0; r < 3 && st == GS_OK; ++r)
            st = gs_filter_enqueue(ctx, g, c.data(), K, B, V, false, bufA, bufB, Y, e, nullptr, nullptr);
        cudaEventRecord(e1, ctx->stream);
        if (st != GS_OK) break;
        if ((st = gs_cuda_check(ctx, cudaEventSynchronize(e1), "autotune timing")) != GS_OK) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = cd;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *knob = saved;
    ctx->lanes_override = saved_lanes;
    if (st != GS_OK) {
        g->tuned_b1 = saved_tb1;
        g->tuned_blk = saved_tblk;
        g->tuned_blk_B = saved_tB;
        g->tuned_split = saved_split;
        g->tuned_lanes = saved_tlanes;
        return st;
    }
    if (B == 1) {
        ctx->tuned_b1 = best.kernel;
        g->tuned_b1 = best.kernel;
        g->tuned_split = best.lanes;
        g->tuned_blk = saved_tblk;
        g->tuned_blk_B = saved_tB;
    } else {
        g->tuned_b1 = saved_tb1;
        g->tuned_blk = best.kernel;
        g->tuned_lanes = best.lanes;
        g->tuned_blk_B = B;
    }
    TuneRecord rec;
    rec.n = n;
    rec.nnz = g->nnz;
    rec.B = B;
    rec.K = K;
    rec.kernel = best.kernel;
    rec.lanes = best.lanes;
    for (auto it = ctx->tune_log.begin(); it != ctx->tune_log.end(); ++it)
        if (it->n == rec.n && it->nnz == rec.nnz && it->B == B && it->K == K) {
            ctx->tune_log.erase(it);
            break;
        }
    if (ctx->tune_log.size() >= 64) ctx->tune_log.erase(ctx->tune_log.begin());
    ctx->tune_log.push_back(rec);
    const int best_kernel = best.kernel;
    if (choice_out) *choice_out = best_kernel;
    if (B != 1) return GS_OK;

    // one column: also time the fixed-count Sinkhorn loop both ways (persistent / graph replay)
    float* ab = nullptr;
    if (cudaMalloc(&ab, sizeof(float) * 2 * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return GS_OK;  // keep the kernel choice; the loop stays on its default
    }
    fill_ones<<<(unsigned)((2 * n + 255) / 256), 256, 0, ctx->stream>>>(2 * n, ab);
    gs_count(ctx, 1);
    const int saved_loop = ctx->loop_mode, saved_sync = ctx->persist_sync;
    // candidates: the persistent loop with each block synchronisation (grid barrier, neighbour
    // flags, tagged values re-read in groups, tagged values re-read one at a time), then graph replay
    constexpr int kSyncs[5] = {0, 1, 2, 4, -1};
    float loop_ms[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    int saved_flags = 0;  // the synthetic loop's status must not reach the caller's next gs_sync
    cudaStreamSynchronize(ctx->stream);
    cudaMemcpy(&saved_flags, ctx->flags, sizeof(int), cudaMemcpyDeviceToHost);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int c = 0; c < 5 && st == GS_OK; ++c) {
        ctx->loop_mode = kSyncs[c] >= 0 ? 0 : 1;
        ctx->persist_sync = kSyncs[c] >= 0 ? kSyncs[c] : saved_sync;
        for (int rep = 0; rep < 2 && st == GS_OK; ++rep) {  // first run warms (graph capture)
            cudaEventRecord(e0, ctx->stream);
            st = gs_sinkhorn_impl(ctx, g, ab, ab + n, nullptr, 1.0, K, 0.0, 10, nullptr, nullptr,
                                  nullptr, nullptr);
            cudaEventRecord(e1, ctx->stream);
            if (st == GS_OK) st = gs_cuda_check(ctx, cudaEventSynchronize(e1), "autotune loop timing");
            if (st == GS_OK) cudaEventElapsedTime(&loop_ms[c], e0, e1);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->loop_mode = saved_loop;
    ctx->persist_sync = saved_sync;
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ab);
    cudaMemcpy(ctx->flags, &saved_flags, sizeof(int), cudaMemcpyHostToDevice);
    if (st != GS_OK) return st;
    int best_c = 0;
    for (int c = 1; c < 5; ++c)
        if (loop_ms[c] < loop_ms[best_c]) best_c = c;
    g->tuned_loop = kSyncs[best_c] >= 0 ? 1 : 2;
    ctx->tuned_loop = g->tuned_loop;
    int best_p = 0;
    for (int c = 1; c < 4; ++c)
        if (loop_ms[c] < loop_ms[best_p]) best_p = c;
    const int best_s = kSyncs[best_p];
    g->tuned_sync = best_s;
    for (auto& r : ctx->tune_log)
        if (r.n == n && r.nnz == g->nnz && r.B == 1 && r.K == K) {
            r.loop = g->tuned_loop;
            r.sync = best_s;
        }
    ctx->tuned_sync = best_s;
    return GS_OK;
}
