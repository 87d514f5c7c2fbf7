"""Run one heat-filter workload a few times, for profilers (ncu) and quick timing.

    python -m paper_2211_00805_gb300.profile_run --case b1   # 100k-point manifold graph, B = 1, K = 30
    python -m paper_2211_00805_gb300.profile_run --case b32  # 200k-point cluster graph, B = 32, K = 40
    python -m paper_2211_00805_gb300.profile_run --case b1 --log-sinkhorn 20  # log-domain loop

Builds the case's graph on the GPU, then applies the filter ``--reps`` times through the C ABI and
prints the mean time per apply (CUDA events) and its algorithmic bandwidth.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import torch  # noqa: E402

from paper_2211_00805_gb300 import binding as gs  # noqa: E402
from paper_2211_00805_gb300 import workloads as W  # noqa: E402

CASES = {
    "b1": dict(kind="manifold", n=100_000, latent=10, ambient=50, seed=2, k=15, K=30, t=5.0, B=1),
    "b32": dict(kind="clusters", n=200_000, dim=30, seed=3, k=10, K=40, t=10.0, B=32),
    "b64": dict(kind="manifold", n=500_000, latent=6, ambient=40, seed=4, k=10, K=40, t=8.0, B=64),
}


def algorithmic_bytes(n, nnz, K, B):
    graph = 8 * nnz + 4 * (n + 1)
    return K * graph + 12 * n * B + (K - 2) * 20 * n * B + 16 * n * B


def time_apply(ctx, g, c, V, Y, reps):
    gs.gs_heat_apply(ctx, g, c["t"], c["K"], V, out=Y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        gs.gs_heat_apply(ctx, g, c["t"], c["K"], V, out=Y)
    e1.record()
    torch.cuda.synchronize()
    gs.gs_sync(ctx)
    return e0.elapsed_time(e1) / reps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", choices=sorted(CASES), default="b1")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--variant", type=int, default=0,
                    help="order-kernel variant (gs_set_option GS_OPT_B1_KERNEL / GS_OPT_BLK_KERNEL)")
    ap.add_argument("--sweep", action="store_true", help="time every variant of the case")
    ap.add_argument("--autotune", action="store_true",
                    help="run gs_autotune on the case's graph and time the tuned filter (choices printed)")
    ap.add_argument("--configs", default="0,0,2,2;0,0,2,1;0,0,2,0;0,0,1,0;1,6,1,0",
                    help="with --sinkhorn: ';'-separated loop mode,kernel,smem graph,sync tuples")
    ap.add_argument("--sinkhorn", type=int, default=0,
                    help="also time this many Sinkhorn iterations in both loop modes (B = 1 cases)")
    ap.add_argument("--log-sinkhorn", type=int, default=0,
                    help="also time this many iterations of the log-domain loop (gs_sinkhorn_log, B = 1 cases)")
    ap.add_argument("--n", type=int, default=0, help="override the case's point count")
    ap.add_argument("--bps", default="1", help="with --sinkhorn: ','-separated GS_OPT_PERSIST_BLOCKS values "
                    "(one graph built per value; timings interleaved)")
    ap.add_argument("--loop-regs", type=int, default=1,
                    help="with --sinkhorn: GS_OPT_LOOP_REGS (1: rows' first entries in registers, 0: off)")
    ap.add_argument("--knn-modes", default="2,1,0", help="with --knn: GS_OPT_KNN_TENSOR values to time")
    ap.add_argument("--knn", action="store_true",
                    help="time the kNN graph builder (tensor-core and CUDA-core screens) instead")
    args = ap.parse_args()
    c = dict(CASES[args.case])
    if args.n:
        c["n"] = args.n
    dev = torch.device("cuda", 0)
    ctx = gs.Context(0)
    if args.knn:
        X, _ = W.tanh_manifold(c["n"], c.get("latent", 10), c.get("ambient", 50), c["seed"])
        Xd = torch.from_numpy(X).to(dev)
        for tensor in [int(m) for m in args.knn_modes.split(",")]:
            gs.gs_set_option(ctx, gs.GS_OPT_KNN_TENSOR, tensor)
            gs.gs_knn(ctx, Xd, c["k"])
            for what, fn in (("knn", lambda: gs.gs_knn(ctx, Xd, c["k"])),
                             ("build_graph", lambda: gs.gs_build_graph(ctx, Xd, c["k"]).close())):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(args.reps):
                    fn()
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.reps
                pairs = c["n"] * (c["n"] - 1)
                print(json.dumps({"case": args.case, "what": what, "tensor_cores": tensor, "ms": ms,
                                  "n": c["n"], "d": X.shape[1],
                                  "dot_TFLOPs": 2.0 * pairs * X.shape[1] / (ms / 1e3) / 1e12}), flush=True)
        gs.gs_sync(ctx)
        return
    if c["kind"] == "manifold":
        X, Z = W.tanh_manifold(c["n"], c["latent"], c["ambient"], c["seed"])
    else:
        X, _ = W.cluster_curves(c["n"], c["dim"], seed=c["seed"])
    graphs = {}
    for bps in [int(b) for b in args.bps.split(",")]:
        gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_BLOCKS, bps)
        graphs[bps] = gs.gs_build_graph(ctx, torch.from_numpy(X).to(dev), c["k"])
        print(json.dumps({"case": args.case, "bps": bps, "layout": gs.gs_graph_layout(graphs[bps])}), flush=True)
    gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_BLOCKS, 1)
    g = next(iter(graphs.values()))
    V = torch.rand((c["n"], c["B"]), generator=torch.Generator().manual_seed(0)).to(dev)
    Y = torch.empty_like(V)
    option = gs.GS_OPT_B1_KERNEL if c["B"] == 1 else gs.GS_OPT_BLK_KERNEL
    variants = ([0, 1, 2, 3, 5, 6, 7] if c["B"] == 1 else [0, 2, 3, 4, 5, 8, 9]) if args.sweep else [args.variant]
    byts = algorithmic_bytes(c["n"], g.nnz, c["K"], c["B"])
    for var in variants:
        gs.gs_set_option(ctx, option, var)
        ms = time_apply(ctx, g, c, V, Y, args.reps)
        print(json.dumps({"case": args.case, "variant": var, "n": c["n"], "nnz": g.nnz, "B": c["B"],
                          "K": c["K"], "apply_ms": ms, "order_us": ms * 1e3 / c["K"],
                          "GBps": byts / (ms / 1e3) / 1e9, "bytes_per_order": byts / c["K"]}), flush=True)
    gs.gs_set_option(ctx, option, args.variant)
    if args.autotune:
        gs.gs_set_option(ctx, option, 0)
        choice = gs.gs_autotune(ctx, g, c["B"], c["K"])
        ms = time_apply(ctx, g, c, V, Y, args.reps)
        print(json.dumps({"case": args.case, "autotuned": gs.gs_autotune_choices(ctx, g, c["B"], c["K"]),
                          "choice": choice, "apply_ms": ms, "order_us": ms * 1e3 / c["K"],
                          "GBps": byts / (ms / 1e3) / 1e9}), flush=True)
        gs.gs_set_option(ctx, option, args.variant)
    if args.sinkhorn and c["B"] == 1:
        # loop modes x one-column kernel variants, interleaved three times, medians reported
        a = torch.full((c["n"],), 1.0 / c["n"], device=dev)
        configs = [(bps,) + tuple(int(x) for x in c.split(",")) for c in args.configs.split(";")
                   for bps in graphs]
        times = {cfg: [] for cfg in configs}
        gs.gs_set_option(ctx, gs.GS_OPT_LOOP_REGS, args.loop_regs)
        for rnd in range(4):
            for bps, mode, var, sg, sy in configs:
                g = graphs[bps]
                gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SYNC, sy)
                gs.gs_set_option(ctx, gs.GS_OPT_LOOP, mode)
                gs.gs_set_option(ctx, gs.GS_OPT_B1_KERNEL, var)
                gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SMEM_GRAPH, sg)
                gs.gs_sinkhorn(ctx, g, a, a, c["t"], c["K"], args.sinkhorn)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                gs.gs_sinkhorn(ctx, g, a, a, c["t"], c["K"], args.sinkhorn)
                e1.record()
                torch.cuda.synchronize()
                gs.gs_sync(ctx)
                if rnd > 0:
                    times[(bps, mode, var, sg, sy)].append(e0.elapsed_time(e1))
        for (bps, mode, var, sg, sy), ts in times.items():
            ms = sorted(ts)[len(ts) // 2]
            print(json.dumps({"case": args.case, "sinkhorn_loop_mode": mode, "b1_variant": var,
                              "smem_graph": sg, "sync": sy, "bps": bps, "loop_regs": args.loop_regs,
                              "iters": args.sinkhorn, "ms_median": ms,
                              "iters_per_s": args.sinkhorn / (ms / 1e3),
                              "order_us": ms * 1e3 / (2 * c["K"] * args.sinkhorn)}), flush=True)
        gs.gs_set_option(ctx, gs.GS_OPT_LOOP, 2)
        gs.gs_set_option(ctx, gs.GS_OPT_B1_KERNEL, 0)
        gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SMEM_GRAPH, 2)
        gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SYNC, 1)
        gs.gs_set_option(ctx, gs.GS_OPT_LOOP_REGS, 1)
    if args.log_sinkhorn and c["B"] == 1:
        a = torch.full((c["n"],), 1.0 / c["n"], device=dev)
        it = args.log_sinkhorn
        gs.gs_sinkhorn_log(ctx, g, a, a, c["t"], c["K"], it)  # warm (workspace, capture stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.reps):
            gs.gs_sinkhorn_log(ctx, g, a, a, c["t"], c["K"], it)
        e1.record()
        torch.cuda.synchronize()
        gs.gs_sync(ctx)
        ms = e0.elapsed_time(e1) / args.reps
        print(json.dumps({"case": args.case, "log_sinkhorn_iters": it, "ms": ms,
                          "iters_per_s": it / (ms / 1e3), "order_us": ms * 1e3 / (2 * c["K"] * it)}), flush=True)

if __name__ == "__main__":
    main()
