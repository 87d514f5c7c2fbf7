#!/usr/bin/env python
"""Geodesic Sinkhorn benchmark on one GB300 (or N replicas, one per GPU, under torchrun).

Workload (one "step" = the whole hot path once): 100,000 points on a 10-d latent manifold in R^50
(latents N(0, I_10) through a fixed random 2-layer tanh map, isotropic noise 0.01), k = 15
symmetric kNN graph with Gaussian weights (sigma = median kNN distance), the Chebyshev heat
filter with K = 30, t = 5 inside 500 Sinkhorn iterations between two softmax bumps, and the FP64
distance reduction.  Metric: Sinkhorn iterations per second (whole job: graph build included).

Also reported: the roofline of the fused Chebyshev order kernel inside the timed region, an
HBM-bound filter measurement on the 200,000-point cluster workload with 32 right-hand sides,
the end-to-end number with host buffers, clocks during the timed region, launch counts and the
FP64 oracle timed on the host cores (bounded sample, scaled).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2211_00805_gb300 import workloads as W  # noqa: E402

METRIC = "Sinkhorn iters/s & SpMM HBM GB/s, batched/adjoint vs plain at rtol 1e-4"
UNIT = "Sinkhorn iters/s"
WORKLOAD = dict(name="manifold-100k-R50: Geodesic Sinkhorn distance, graph build included",
                n=100_000, latent=10, ambient=50, seed=2, k=15, K=30, t=5.0, iters=500)
HBM_CASES = {
    "spmm_hbm": dict(name="clusters-200k-R30, B=32 heat filter", kind="clusters", n=200_000, dim=30,
                     m=32, k=10, K=40, t=10.0, seed=3, tag="order_blk_clusters200k_B32", node_order=0),
    "spmm_hbm_b64": dict(name="manifold-500k-R40, B=64 heat filter", kind="manifold", n=500_000,
                         latent=6, ambient=40, m=64, k=10, K=40, t=8.0, seed=4,
                         tag="order_blk_manifold500k_B64", node_order=1),
}
L2_FLUSH_BYTES = 256 << 20
EXCHANGE_FLOOR_US = 1.446  # µs per Chebyshev order, 100k-point manifold graph (see roofline)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the HBM-bound filter case")
    return ap.parse_args()


# ------------------------------------------------------------------------------ algorithmic bytes
def apply_bytes(n: int, nnz: int, K: int, B: int, last_streams: int) -> int:
    """Bytes one K-order filter apply must move: each order reads the CSR (4 B column + 4 B value
    per nonzero, 4 B per row pointer) and gathers the previous block once (4nB); order 1 also
    writes T_1 and y (12nB in total with the gather); orders 2..K-1 read T_{k-2} and y and write
    T_k and y (20nB with the gather); the last order streams `last_streams` n x B blocks."""
    graph = 8 * nnz + 4 * (n + 1)
    if K == 1:
        return graph + 4 * n * B * last_streams
    return K * graph + 12 * n * B + (K - 2) * 20 * n * B + 4 * n * B * last_streams


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def ncu_traffic(kernel_tag: str, source: str = "cheb.cu"):
    """DRAM bytes per launch from the committed ncu summary, or None if the kernel's source file
    changed since the counters were taken (the summary records the hash it was taken on)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    src = os.path.join(ROOT, "paper_2211_00805_gb300", "csrc", source)
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        for line in open(path):
            parts = line.split()
            if len(parts) >= 3 and parts[0] == kernel_tag and parts[1] == h:
                return float(parts[2])
    except OSError:
        pass
    return None


# ------------------------------------------------------------------------------------- clocks
CLOCK_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


def summarise_clocks(text: str):
    """Median SM clock, the largest max clock and the throttle reasons seen Active, from
    ``nvidia-smi --format=csv,noheader,nounits`` lines of ClockSampler.FIELDS; None without samples."""
    sm, smax, reasons = [], [], set()
    for line in text.strip().splitlines():
        p = [x.strip() for x in line.split(",")]
        if len(p) < 8:
            continue
        try:
            sm.append(float(p[0]))
            smax.append(float(p[1]))
        except ValueError:
            continue
        for nm, val in zip(CLOCK_REASONS, p[4:8]):
            if val.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        import threading
        self.proc = None
        self.lines = []
        self.first = threading.Event()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            self.first.set()
            return
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()
        # the sampler's start-up (NVML initialisation) must not overlap the timed region
        self.first.wait(timeout=5.0)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line)
            self.first.set()
        self.first.set()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self.reader.join(timeout=5)
        return summarise_clocks("".join(self.lines))


# ------------------------------------------------------------------------------- CPU oracle
def oracle_sample(cfg=WORKLOAD, small_n=10_000, knn_rows=2400, iters_small=150):
    """The FP64 oracle, as it stands, on a bounded sample of the workload, scaled to the full
    step.  kNN: ``knn_rows`` query rows of the full point cloud (every row costs the same n d
    work), scaled by n / rows.  Graph assembly and Sinkhorn iterations: the same generator at
    ``small_n`` points; the assembly scaled by n / small_n, one iteration by the edge-count ratio
    (each iteration is 2 K sparse products over all edges), times the full iteration count."""
    import oracle
    X, Z = W.tanh_manifold(cfg["n"], cfg["latent"], cfg["ambient"], cfg["seed"])
    X64 = X.astype(np.float64)
    rows = np.random.default_rng(0).choice(cfg["n"], knn_rows, replace=False)
    t0 = time.perf_counter()
    oracle.knn(X64, cfg["k"], rows=rows)
    t_knn = (time.perf_counter() - t0) * cfg["n"] / knn_rows

    ps = W.manifold_pair(n=small_n, latent=cfg["latent"], ambient=cfg["ambient"], seed=cfg["seed"],
                         k=cfg["k"], K=cfg["K"], t=cfg["t"], iters=iters_small)
    Xs = ps.X.astype(np.float64)
    idx, dist = oracle.knn(Xs, ps.k)
    t0 = time.perf_counter()
    s = oracle.median_sigma(dist)
    rp, col, A = oracle.affinity_graph(idx, dist, s)
    deg, L = oracle.laplacian(rp, col, A)
    Ls = oracle.shifted(L)
    t_graph = (time.perf_counter() - t0) * cfg["n"] / small_n
    b = oracle.cheb_coefficients(ps.t, ps.K)
    t0 = time.perf_counter()
    oracle.sinkhorn(Ls, b, ps.a.astype(np.float64), ps.b.astype(np.float64), ps.t, iters_small)
    t_iter_small = (time.perf_counter() - t0) / iters_small
    nnz_small = len(col)
    nnz_full_est = nnz_small * cfg["n"] / small_n
    t_iters = t_iter_small * nnz_full_est / nnz_small * cfg["iters"]
    total = t_knn + t_graph + t_iters
    sample = (f"oracle kNN on {knn_rows} of {cfg['n']} query rows (x{cfg['n'] / knn_rows:.0f}); graph "
              f"assembly + {iters_small} Sinkhorn iterations of the same generator at n={small_n} "
              f"(nnz={nnz_small}), scaled by n and by nnz to n={cfg['n']}, {cfg['iters']} iterations; "
              f"est. full step {total:.1f} s = kNN {t_knn:.1f} + graph {t_graph:.1f} + "
              f"iterations {t_iters:.1f}")
    return {"value": cfg["iters"] / total, "unit": UNIT, "cores": oracle.num_threads(),
            "kind": "oracle", "sample": sample, "est_step_s": total}


def oracle_sample_cfg3(small_n=20_000, knn_rows=1200, iters_small=2, iters=300):
    """The FP64 oracle on a bounded sample of the barycenter workload (200k cluster points in R^30,
    k = 10, 32 distributions, K = 40, t = 10, 300 iterations), scaled: kNN on ``knn_rows`` query rows
    of the full cloud (x n / rows), graph assembly and ``iters_small`` barycenter iterations of the
    same generator at ``small_n`` points, scaled by n and by the edge count."""
    import oracle
    cfg = W.clusters_barycenter()
    n = cfg["X"].shape[0]
    X64 = cfg["X"].astype(np.float64)
    rows = np.random.default_rng(0).choice(n, knn_rows, replace=False)
    t0 = time.perf_counter()
    oracle.knn(X64, cfg["k"], rows=rows)
    t_knn = (time.perf_counter() - t0) * n / knn_rows
    cs = W.clusters_barycenter(n=small_n)
    t0 = time.perf_counter()
    Ls, ex = oracle.build_graph(cs["X"].astype(np.float64), cs["k"])
    t_graph = (time.perf_counter() - t0) * n / small_n  # includes the small kNN: an overestimate
    b = oracle.cheb_coefficients(cs["t"], cs["K"])
    t0 = time.perf_counter()
    oracle.barycenter(Ls, b, cs["M"].astype(np.float64), cs["alpha"], iters_small)
    t_it = (time.perf_counter() - t0) / iters_small
    nnz_full_est = len(ex["col"]) * n / small_n
    t_iters = t_it * nnz_full_est / len(ex["col"]) * iters
    total = t_knn + t_graph + t_iters
    return {"value": iters / t_iters, "unit": "barycenter iters/s (graph build excluded)",
            "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"kNN on {knn_rows} of {n} query rows; graph + {iters_small} barycenter iterations "
                       f"of the same generator at n={small_n}, scaled by nnz to n={n}; est. "
                       f"{t_iters:.0f} s for {iters} iterations, {total:.0f} s with the graph build")}


def oracle_sample_cfg5(small_n=10_000, iters_small=4, iters=200):
    """The FP64 oracle on a bounded sample of the differentiation workload (500k manifold points in
    R^40, 64 inputs, K = 40, t = 8, 200 + 200 iterations): forward (barycenter + distance) and
    forward + reverse (``barycenter_distance_grad``) at ``iters_small`` iterations each on
    ``small_n`` points of the same generator, per iteration, scaled by the edge count to the full
    size and 200 iterations."""
    import oracle
    c = W.manifold_barycenter_grad(n=small_n, bary_iters=iters_small, sink_iters=iters_small)
    Ls, ex = oracle.build_graph(c["X"].astype(np.float64), c["k"])
    b = oracle.cheb_coefficients(c["t"], c["K"])
    M, src = c["M"].astype(np.float64), c["src"].astype(np.float64)
    t0 = time.perf_counter()
    mu = oracle.barycenter(Ls, b, M, c["alpha"], iters_small)
    oracle.sinkhorn(Ls, b, src, mu, c["t"], iters_small)
    t_f = (time.perf_counter() - t0) / iters_small
    t0 = time.perf_counter()
    oracle.barycenter_distance_grad(Ls, b, src, M, c["alpha"], c["t"], iters_small, iters_small)
    t_g = (time.perf_counter() - t0) / iters_small
    scale = 500_000 / small_n  # edge count grows with n (k fixed)
    return {"value": 1.0 / (t_g * scale * iters), "unit": "gradient evaluations/s (200 + 200 iterations)",
            "cores": oracle.num_threads(), "kind": "oracle",
            "forward_s_est": t_f * scale * iters, "forward_plus_reverse_s_est": t_g * scale * iters,
            "sample": (f"{iters_small} iterations of each loop at n={small_n} of the same generator "
                       f"(nnz={len(ex['col'])}), scaled by n to 500,000 and to {iters} iterations")}


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest value across ranks (each rank times its own replica; the job takes the slowest)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def static_config(world: int, nnz=None):
    """The workload description both arms print (no timings in it)."""
    cfg = WORKLOAD
    out = {"workload": cfg["name"], "n": cfg["n"], "d": cfg["ambient"], "k": cfg["k"], "K": cfg["K"],
           "t": cfg["t"], "iters": cfg["iters"], "parallelism": "replicas" if world > 1 else "single GPU",
           "l2": "256 MB buffer written between timed steps (GPU arm)"}
    if nnz is not None:
        out["nnz"] = int(nnz)
    return out


def reference_shares(n: int, iters: int, S: int):
    """Split one step into S shares: consecutive query-row ranges covering 0..n-1 once, and
    iteration counts summing to `iters`."""
    rows = [np.arange(i * n // S, (i + 1) * n // S) for i in range(S)]
    its = [iters // S + (1 if i < iters % S else 0) for i in range(S)]
    return rows, its


def run_reference(args, rank, world):
    """The FP64 oracle, as it stands, on the headline workload.  The full step (kNN over all n
    query rows, graph assembly, 500 Sinkhorn iterations, distance) is split into `steps` equal
    shares of real work: step i runs the kNN of its n / steps query rows and iters / steps Sinkhorn
    iterations on the full 100k-point oracle graph (built once before the timed region), plus the
    graph assembly's measured time / steps.  The timed shares add up to one whole step, so the
    value is iterations per second of the full workload without extrapolation from a smaller one."""
    if rank != 0:
        return
    import oracle
    cfg = WORKLOAD
    p = W.manifold_pair(n=cfg["n"], latent=cfg["latent"], ambient=cfg["ambient"], seed=cfg["seed"],
                        k=cfg["k"], K=cfg["K"], t=cfg["t"], iters=cfg["iters"])
    X64 = p.X.astype(np.float64)
    n = cfg["n"]
    t0 = time.perf_counter()
    idx, dist = oracle.knn(X64, cfg["k"])
    t_knn_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    s = oracle.median_sigma(dist)
    rp, col, A = oracle.affinity_graph(idx, dist, s)
    deg, L = oracle.laplacian(rp, col, A)
    Ls = oracle.shifted(L)
    t_assembly = time.perf_counter() - t0
    b = oracle.cheb_coefficients(cfg["t"], cfg["K"])
    a64, b64 = p.a.astype(np.float64), p.b.astype(np.float64)
    S = max(1, args.steps)
    rows, its = reference_shares(n, cfg["iters"], S)

    def share(i):
        oracle.knn(X64, cfg["k"], rows=rows[i])
        if its[i]:
            oracle.sinkhorn(Ls, b, a64, b64, cfg["t"], its[i])

    for w in range(args.warmup):
        share(w % S)
    t0 = time.perf_counter()
    for i in range(S):
        share(i)
    wall = time.perf_counter() - t0
    step_s = wall + t_assembly  # one whole step: every share once, plus the graph assembly
    value = cfg["iters"] / step_s
    sample = (f"the full step split into {S} shares of real work: kNN of n/{S} query rows and "
              f"{cfg['iters']}/{S} Sinkhorn iterations per share on the full n={n} oracle graph "
              f"(nnz={len(col)}); graph assembly timed once ({t_assembly:.2f} s) and added; the oracle's "
              f"full kNN outside the timed region took {t_knn_setup:.1f} s")
    cb = {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle", "sample": sample}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3 / S,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded tanh-manifold generator; no dataset)",
            "config": static_config(world, len(col)), "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall, "whole_step_s": step_s}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------ ours
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2211_00805_gb300 import binding as gs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    ctx = gs.Context(local_rank, stream)
    cfg = WORKLOAD
    p = W.manifold_pair(n=cfg["n"], latent=cfg["latent"], ambient=cfg["ambient"], seed=cfg["seed"],
                        k=cfg["k"], K=cfg["K"], t=cfg["t"], iters=cfg["iters"])
    X = torch.from_numpy(p.X).to(dev)
    a = torch.from_numpy(p.a).to(dev)
    b = torch.from_numpy(p.b).to(dev)
    n = cfg["n"]
    u = torch.empty(n, dtype=torch.float32, device=dev)
    v = torch.empty(n, dtype=torch.float32, device=dev)
    dist = torch.empty(2, dtype=torch.float64, device=dev)
    itd = torch.empty(1, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(Xd, ad, bd, ev=None):
        if ev is not None:
            ev[0].record(stream)
        g = gs.gs_build_graph(ctx, Xd, cfg["k"])
        if ev is not None:
            ev[1].record(stream)
        gs.gs_sinkhorn(ctx, g, ad, bd, cfg["t"], cfg["K"], cfg["iters"], u=u, v=v, dist=dist,
                       iters_done=itd)
        if ev is not None:
            ev[2].record(stream)
        nnz = g.nnz
        g.close()
        return nnz

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for i in range(args.warmup):
        nnz = step(X, a, b)
    gs.gs_sync(ctx)
    w2 = float(dist[0].item())
    # the project's autotuner, once, on a graph of this workload: its one-column kernel and loop
    # choices are kept by the context and used by the timed steps' freshly built graphs
    gt = gs.gs_build_graph(ctx, X, cfg["k"])
    tuned = {"b1_kernel": gs.gs_autotune(ctx, gt, 1, cfg["K"]),
             "loop_mode": gs.gs_get_option(ctx, gs.GS_OPT_LOOP),
             "persist_sync": gs.gs_get_option(ctx, gs.GS_OPT_PERSIST_SYNC)}
    gt.close()
    for i in range(2):
        nnz = step(X, a, b)

    # first uses initialise lazily (NVTX; the fill kernel's module, ~0.25 s): not in the timed region
    torch.cuda.nvtx.range_push("gs_warm")
    torch.cuda.nvtx.range_pop()
    flush.fill_(0.0)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clocks = ClockSampler(local_rank) if rank == 0 else None  # up and sampling before the barrier
    barrier()
    l0 = gs.gs_launch_count(ctx)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(args.steps):
        flush.fill_(float(i))  # L2 flush: 256 MB write between steps
        torch.cuda.nvtx.range_push("gs_timed_step")
        nnz = step(X, a, b, evs[i])
        torch.cuda.nvtx.range_pop()
    t_end.record(stream)
    barrier()
    launches = gs.gs_launch_count(ctx) - l0
    clk = clocks.stop() if clocks else None
    gs.gs_sync(ctx)
    total_ms = t_start.elapsed_time(t_end)
    graph_ms = [e[0].elapsed_time(e[1]) for e in evs]
    sink_ms = [e[1].elapsed_time(e[2]) for e in evs]
    # span of every step, from its start to the next step's start (the last to the end event)
    step_ms = [evs[i][0].elapsed_time(evs[i + 1][0]) for i in range(len(evs) - 1)]
    step_ms.append(evs[-1][0].elapsed_time(t_end))
    total_ms = max_over_ranks(total_ms, world, dev)
    value = cfg["iters"] * args.steps * world / (total_ms / 1e3)

    # roofline of the dominant kernel of the step: the Sinkhorn loop's Chebyshev orders (B = 1)
    sink_s = statistics.mean(sink_ms) / 1e3
    peak, peak_kind = measured_peaks()
    roofline = loop_roofline(n, nnz, cfg["K"], cfg["iters"], sink_s, tuned, peak, peak_kind)

    extras = {}
    if not args.no_extras:
        for key, case in HBM_CASES.items():
            extras[key] = hbm_case(gs, ctx, dev, stream, peak, peak_kind, case)
        extras["barycenter_cfg3"] = barycenter_case(gs, ctx, dev, stream, peak, peak_kind)
        extras["batched_cfg4"] = batched_case(gs, ctx, dev, stream)
        extras["adjoint_cfg5"] = adjoint_case(gs, ctx, dev, stream)
        extras["barycentric_distance"] = families_case(gs, ctx, dev, stream)
        extras["implicit_vs_chebyshev"] = implicit_case(gs, ctx, dev, stream)
        extras["log_domain_sinkhorn"] = logdomain_case(gs, ctx, dev, stream)
        extras["combinatorial_filter"] = combinatorial_case(gs, ctx, dev, stream)
        extras["matmul_peaks"] = matmul_peaks(dev, stream)
        extras["knn_screen"] = knn_case(gs, ctx, dev, stream, X, cfg, extras["matmul_peaks"])

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    Xh = torch.from_numpy(p.X).pin_memory()
    ah = torch.from_numpy(p.a).pin_memory()
    bh = torch.from_numpy(p.b).pin_memory()
    uh = torch.empty(n, dtype=torch.float32).pin_memory()
    vh = torch.empty(n, dtype=torch.float32).pin_memory()
    dh = torch.empty(2, dtype=torch.float64).pin_memory()
    Xd, ad, bd = torch.empty_like(X), torch.empty_like(a), torch.empty_like(b)

    def e2e_step():
        Xd.copy_(Xh, non_blocking=True)
        ad.copy_(ah, non_blocking=True)
        bd.copy_(bh, non_blocking=True)
        step(Xd, ad, bd)
        uh.copy_(u, non_blocking=True)
        vh.copy_(v, non_blocking=True)
        dh.copy_(dist, non_blocking=True)

    e2e_step()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    h2d = Xh.numel() * 4 + ah.numel() * 4 + bh.numel() * 4
    d2h = uh.numel() * 4 + vh.numel() * 4 + dh.numel() * 8
    e2e = {"value": cfg["iters"] * args.steps * world / (e2e_ms / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample()
        cpu.pop("est_step_s", None)
        if not args.no_extras:
            extras["cpu_baselines"] = {"barycenter_cfg3": oracle_sample_cfg3(),
                                       "adjoint_cfg5": oracle_sample_cfg5()}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded tanh-manifold generator; no dataset)",
            "config": static_config(world, nnz),
            "timing": {"graph_build_ms": statistics.mean(graph_ms),
                       "sinkhorn_ms": statistics.mean(sink_ms),
                       "sinkhorn_only_iters_per_s": cfg["iters"] / sink_s,
                       "step_ms_min_median_max": [min(step_ms), statistics.median(step_ms), max(step_ms)],
                       "W2": w2, "autotune": tuned},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "gpu_launches_per_step": launches / args.steps,
            "clocks": clk,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)


def loop_roofline(n, nnz, K, iters, sink_s, tuned, peak, peak_kind):
    """The `roofline` object of the Sinkhorn loop (B = 1) run in `sink_s` seconds: one persistent
    launch per loop (loop mode 0) or one launch per Chebyshev order (mode 1).  `achieved` counts the
    byte model of every order; the persistent form adds its fraction of the exchange floor."""
    per_apply = apply_bytes(n, nnz, K, 1, last_streams=6)  # gather, T_{K-2}, y, num, out, xnext
    orders = 2 * K * iters
    order_us = sink_s / orders * 1e6
    achieved = 2 * iters * per_apply / sink_s / 1e9
    if tuned["loop_mode"] == 0:
        tr = ncu_traffic("sinkhorn_persistent_manifold100k_500it", "persist.cu")
        name = {0: "sinkhorn_persistent", 1: "sinkhorn_neighbour_sync", 2: "sinkhorn_tagged"}[tuned["persist_sync"]]
        kern = {"kernel": f"{name} (whole {iters}-iteration loop, one cooperative launch)",
                "bytes_per_launch": 2 * iters * per_apply, "launch_us": sink_s * 1e6,
                # the loop's own floor: the same launch with each row's sum replaced by one staged
                # neighbour value (staging, tagged words and both block barriers kept), 500
                # iterations of this workload timed with CUDA events on a GB300; that copy skips
                # the arithmetic, so it is not part of the library and not re-timed here
                "exchange_floor_us_per_order": EXCHANGE_FLOOR_US,
                "frac_of_exchange_floor": EXCHANGE_FLOOR_US / order_us}
    else:
        tr = ncu_traffic("order_b1_manifold100k")
        kern = {"kernel": "fused Chebyshev order kernel (B=1), one launch per order",
                "bytes_per_launch": per_apply / K, "launch_us": order_us}
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": tr, **kern, "order_us": order_us,
            "peak_kind": f"{peak_kind} hbm_gbs",
            "note": "working set (~19 MB) is L2-resident; see spmm_hbm for the HBM-bound case"}


def hbm_case(gs, ctx, dev, stream, peak, peak_kind, c, reps=5):
    """Heat filter with B columns on a graph whose per-order working set exceeds L2: achieved
    algorithmic GB/s of the fused order kernel (CUDA events around `reps` applies)."""
    import torch
    if c["kind"] == "clusters":
        X, labels = W.cluster_curves(c["n"], c["dim"], seed=c["seed"])
        M = W.cluster_unions(labels, c["m"], 3, c["seed"] + 1000)
    else:
        X, Z = W.tanh_manifold(c["n"], c["latent"], c["ambient"], c["seed"])
        M = np.random.default_rng(c["seed"]).random((c["n"], c["m"])).astype(np.float32)
    g = build_graph(gs, ctx, torch.from_numpy(X).to(dev), c["k"], c["node_order"])
    V = torch.from_numpy(M).to(dev)
    Y = torch.empty_like(V)
    for _ in range(2):
        gs.gs_heat_apply(ctx, g, c["t"], c["K"], V, out=Y)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        gs.gs_heat_apply(ctx, g, c["t"], c["K"], V, out=Y)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    gs.gs_sync(ctx)
    s = e0.elapsed_time(e1) / 1e3 / reps
    byts = apply_bytes(c["n"], g.nnz, c["K"], c["m"], last_streams=4)  # gather, T_{K-2}, y, out
    ach = byts / s / 1e9
    out = {"workload": c["name"], "n": c["n"], "nnz": g.nnz, "B": c["m"], "K": c["K"],
           "apply_ms": s * 1e3, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
           "bytes_per_apply": byts, "peak_kind": f"{peak_kind} hbm_gbs",
           "bytes_per_order": byts / c["K"], "order_us": s * 1e6 / c["K"],
           "node_order": c["node_order"],
           "note": "apply time includes the two [n, B] permutations into and out of the locality order",
           "traffic": ncu_traffic(c["tag"]), "traffic_unit": "DRAM bytes per order launch (ncu)"}
    g.close()
    return out


def build_graph(gs, ctx, X, k, node_order=1):
    """Graph build with the node order inside each bisection part set for this graph only: 1 groups
    rows by the part that reads them (the default, best for the one-column loop), 0 orders by degree
    alone (best for the row-group kernel of the many-column filters)."""
    gs.gs_set_option(ctx, gs.GS_OPT_NODE_ORDER, node_order)
    try:
        return gs.gs_build_graph(ctx, X, k)
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_NODE_ORDER, 1)


def _time(stream, fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def batched_case(gs, ctx, dev, stream, count=512, iters=200):
    """The batching workload: `count` ragged problems (n log-uniform in [1e3, 5e4], d 3..20, k in
    {8,10,15}, K in {16,24,32}, t = 5, Dirichlet marginals on 10 % supports, `iters` iterations) in
    one batched call (one persistent launch, replayed from a captured CUDA graph from the second
    call on) against `count` sequential single-problem calls on the same graphs; W^2 agreement."""
    import torch
    probs = W.ragged_batch(count=count, iters=iters)
    graphs = [gs.gs_build_graph(ctx, torch.from_numpy(p.X).to(dev), p.k) for p in probs]
    a = [torch.from_numpy(p.a).to(dev) for p in probs]
    b = [torch.from_numpy(p.b).to(dev) for p in probs]
    ts, Ks = [p.t for p in probs], [p.K for p in probs]
    us = [torch.empty(g.n, dtype=torch.float32, device=dev) for g in graphs]
    vs = [torch.empty(g.n, dtype=torch.float32, device=dev) for g in graphs]
    dist = torch.empty((count, 2), dtype=torch.float64, device=dev)
    run_b = lambda: gs.gs_sinkhorn_batched(ctx, graphs, a, b, ts, Ks, iters, us, vs, dist)  # noqa: E731
    run_b()  # warm (workspace, queue, graph capture)
    run_b()
    l0 = gs.gs_launch_count(ctx)
    ms_b = _time(stream, run_b)
    launches_b = gs.gs_launch_count(ctx) - l0
    db = dist[:, 0].cpu().numpy().copy()
    for i, g in enumerate(graphs):  # warm the per-problem graphs
        gs.gs_sinkhorn(ctx, g, a[i], b[i], ts[i], Ks[i], iters)
    seq = []
    ms_s = _time(stream, lambda: seq.extend(gs.gs_sinkhorn(ctx, g, a[i], b[i], ts[i], Ks[i], iters)[2]
                                            for i, g in enumerate(graphs)))
    gs.gs_sync(ctx)
    ds = np.array([float(d[0]) for d in seq])
    rel = float(np.max(np.abs(db - ds) / np.maximum(np.abs(ds), 1e-30)))
    nodes = sum(g.n for g in graphs)
    nnz = sum(g.nnz for g in graphs)
    for g in graphs:
        g.close()
    return {"workload": f"{count} ragged problems, n log-uniform in [1e3, 5e4], K in {{16, 24, 32}}, t = 5",
            "problems": count, "iters": iters, "total_nodes": nodes, "total_nnz": nnz,
            "batched_ms": ms_b, "batched_launches_per_call": launches_b, "sequential_ms": ms_s,
            "speedup": ms_s / ms_b, "batched_problem_iters_per_s": count * iters / (ms_b / 1e3),
            "max_rel_diff_W2": rel, "rtol_1e-4_met": rel <= 1e-4}


def implicit_case(gs, ctx, dev, stream, t=5.0, K=30, iters=12):
    """The Euler implicit kernel (I + (t/K) L)^{-K} (K conjugate-gradient solves, Sec. 4) against the
    Chebyshev filter of the same degree on the 100k-point manifold graph, one column: time of one
    apply each, and how far each is from a degree-60 Chebyshev apply (error below 1e-12 of the
    exponential at t = 5)."""
    import torch
    p = W.manifold_pair()
    g = gs.gs_build_graph(ctx, torch.from_numpy(p.X).to(dev), p.k)
    V = torch.from_numpy(p.a).to(dev)
    out = {}
    gs.gs_heat_apply_implicit(ctx, g, t, K, V, iters=iters)  # warm
    ms_e = _time(stream, lambda: out.__setitem__("e", gs.gs_heat_apply_implicit(ctx, g, t, K, V, iters=iters)))
    gs.gs_heat_apply(ctx, g, t, K, V)
    ms_c = _time(stream, lambda: out.__setitem__("c", gs.gs_heat_apply(ctx, g, t, K, V)))
    ref = gs.gs_heat_apply(ctx, g, t, 60, V).double()
    gs.gs_sync(ctx)
    scale = float(ref.abs().max())
    err = {k: float((out[k].double() - ref).abs().max()) / scale for k in ("e", "c")}
    g.close()
    return {"workload": "manifold-100k-R50, B = 1", "t": t, "K": K, "cg_iters_per_step": iters,
            "implicit_ms": ms_e, "chebyshev_ms": ms_c, "implicit_over_chebyshev": ms_e / ms_c,
            "implicit_max_rel_err": err["e"], "chebyshev_max_rel_err": err["c"]}


def logdomain_case(gs, ctx, dev, stream, iters_manifold=100):
    """Log-domain Sinkhorn (FP64 potentials, extended-range Chebyshev recurrence): the 2,000-point
    sphere pair at t = 1, K = 20, 200 iterations, where the FP32 scalings overflow; and the
    100k-point manifold pair at t = 5, K = 30 against the FP32 loop over the same iterations (its
    cost over the FP32 loop, and how far the two distances are apart)."""
    import torch
    out = {}
    p = W.sphere_pair()
    g = gs.gs_build_graph(ctx, torch.from_numpy(p.X).to(dev), p.k)
    a, b = torch.from_numpy(p.a).to(dev), torch.from_numpy(p.b).to(dev)
    run = lambda: out.__setitem__("s", gs.gs_sinkhorn_log(ctx, g, a, b, p.t, p.K, p.iters))  # noqa: E731
    run()
    l0 = gs.gs_launch_count(ctx)
    run()
    launches_s = gs.gs_launch_count(ctx) - l0
    ms_s = _time(stream, run)
    gs.gs_sync(ctx)
    w2_s = float(out["s"][2][0])
    g.close()
    q = W.manifold_pair()
    g = gs.gs_build_graph(ctx, torch.from_numpy(q.X).to(dev), q.k)
    a, b = torch.from_numpy(q.a).to(dev), torch.from_numpy(q.b).to(dev)
    it = iters_manifold
    run = lambda: out.__setitem__("m", gs.gs_sinkhorn_log(ctx, g, a, b, q.t, q.K, it))  # noqa: E731
    run()
    ms_m = _time(stream, run)
    run32 = lambda: out.__setitem__("f", gs.gs_sinkhorn(ctx, g, a, b, q.t, q.K, it))  # noqa: E731
    run32()
    ms_f = _time(stream, run32)
    gs.gs_sync(ctx)
    w2_m, w2_f = float(out["m"][2][0]), float(out["f"][2][0])
    g.close()
    orders = 2 * q.K * it
    # one order: CSR values and indices; per row the gathered entry (once), the previous vector,
    # the accumulator read and written, and the output (8 bytes each)
    order_bytes = 8 * g.nnz + 4 * (q.X.shape[0] + 1) + 40 * q.X.shape[0]
    return {"sphere_2k_t1": {"workload": "sphere-2k, t = 1, K = 20 (FP32 scalings overflow here)",
                             "iters": p.iters, "ms": ms_s, "iters_per_s": p.iters / (ms_s / 1e3),
                             "W2": w2_s, "launches": launches_s},
            "manifold_100k_t5": {"workload": "manifold-100k-R50, t = 5, K = 30", "iters": it,
                                 "log_domain_ms": ms_m, "fp32_loop_ms": ms_f,
                                 "log_over_fp32": ms_m / ms_f, "W2_log": w2_m, "W2_fp32": w2_f,
                                 "W2_rel_diff": abs(w2_m - w2_f) / abs(w2_f),
                                 "order_us": ms_m * 1e3 / orders,
                                 "order_GBps": order_bytes / (ms_m / 1e3 / orders) / 1e9}}


def families_case(gs, ctx, dev, stream, bary_iters=100, sink_iters=200):
    """Barycentric distance (Definition 4.3) and expected barycenter effect (Definition 4.4) on the
    200k-point cluster graph: the 32 cluster-union distributions split into two families of 16,
    uniform weights, t = 10, K = 40; one library call each, timed with CUDA events."""
    import torch
    cfg = W.clusters_barycenter()
    g = build_graph(gs, ctx, torch.from_numpy(cfg["X"]).to(dev), cfg["k"], node_order=0)
    M = cfg["M"]
    MT = torch.from_numpy(np.ascontiguousarray(M[:, :16])).to(dev)
    MC = torch.from_numpy(np.ascontiguousarray(M[:, 16:])).to(dev)
    alpha = torch.full((16,), 1.0 / 16, dtype=torch.float64, device=dev)
    Y = torch.from_numpy(cfg["X"]).to(dev)
    t, K = cfg["t"], cfg["K"]
    out = {}
    run = lambda: out.__setitem__("r", gs.gs_barycentric_distance(ctx, g, MT, alpha, MC, alpha, t, K,  # noqa: E731
                                                                  bary_iters, sink_iters))
    run()  # warm (workspace)
    ms = _time(stream, run)
    dist, muT, muC = out["r"]
    ms_e = _time(stream, lambda: out.__setitem__("tau", gs.gs_barycenter_effect(ctx, Y, muT, muC)))
    gs.gs_sync(ctx)
    d = dist.cpu().numpy()
    tau = out["tau"].cpu().numpy()
    n = int(cfg["X"].shape[0])
    g.close()
    return {"workload": "clusters-200k-R30, two families of 16 cluster-union distributions", "n": n,
            "bary_iters": bary_iters, "sink_iters": sink_iters, "K": K, "t": t,
            "barycentric_distance_ms": ms, "gamma_squared": float(d[0]),
            "gamma": float(d[1]) if np.isfinite(d[1]) else None,  # W is undefined where W^2 < 0
            "effect_ms": ms_e, "effect_norm": float(np.linalg.norm(tau)),
            "filter_orders": 2 * (2 * K * bary_iters) + 2 * K * sink_iters}


def adjoint_case(gs, ctx, dev, stream, iters=200, checkpoint=20):
    """The differentiation workload: gradient of J = W^2(src, barycenter(M, alpha)) on the
    500k-point manifold with 64 inputs (K = 40, t = 8), `iters` iterations in each loop, checkpoints
    every `checkpoint`: forward only (barycenter + distance) vs forward + reverse sweep (dJ/dsrc and
    dJ/dalpha)."""
    import torch
    cfg = W.manifold_barycenter_grad(bary_iters=iters, sink_iters=iters, checkpoint=checkpoint)
    g = gs.gs_build_graph(ctx, torch.from_numpy(cfg["X"]).to(dev), cfg["k"])
    M = torch.from_numpy(cfg["M"]).to(dev)
    alpha = torch.tensor(cfg["alpha"], dtype=torch.float64, device=dev)
    src = torch.from_numpy(cfg["src"]).to(dev)
    t, K = cfg["t"], cfg["K"]
    res = {}

    def forward():
        mu = gs.gs_barycenter(ctx, g, M, alpha, t, K, iters)
        res["d"] = gs.gs_distance(ctx, g, src, mu, t, K, iters)

    def gradient():
        mu = gs.gs_barycenter(ctx, g, M, alpha, t, K, iters)
        d, ga, gmu = gs.gs_sinkhorn_grad(ctx, g, src, mu, t, K, iters, checkpoint=checkpoint)
        _, galpha = gs.gs_barycenter_grad(ctx, g, M, alpha, t, K, iters, gmu, checkpoint=checkpoint)
        res["g"] = (d, ga, galpha)

    # the objective is the distance to the barycenter as the iteration leaves it, whose mass is not
    # exactly the source's: the equal-mass argument check is off for this leg
    gs.gs_set_option(ctx, gs.GS_OPT_CHECK_ARGS, 0)
    forward()
    gradient()
    ms_f = _time(stream, forward)
    ms_g = _time(stream, gradient)
    gs.gs_sync(ctx)
    gs.gs_set_option(ctx, gs.GS_OPT_CHECK_ARGS, 1)
    w2_f = float(res["d"][0])
    w2_g = float(res["g"][0][0])
    n = g.n
    g.close()
    return {"workload": "manifold-500k-R40, 64 inputs, K = 40, t = 8", "n": n, "m": int(M.shape[1]), "K": K,
            "iters": iters, "checkpoint": checkpoint, "forward_ms": ms_f, "forward_plus_backward_ms": ms_g,
            "backward_over_forward": ms_g / ms_f - 1.0, "J_forward": w2_f, "J_gradient_pass": w2_g,
            "J_rel_diff": abs(w2_f - w2_g) / abs(w2_f)}


def barycenter_case(gs, ctx, dev, stream, peak, peak_kind, iters=300):
    """The barycenter workload: 32 cluster-union distributions on the 200k-point cluster graph in
    R^30 (k = 10, K = 40, t = 10), uniform weights, `iters` barycenter iterations in one call:
    iterations per second and the counted bytes per Chebyshev order of the two [n, 32] applies."""
    import torch
    cfg = W.clusters_barycenter(iters=iters)
    g = build_graph(gs, ctx, torch.from_numpy(cfg["X"]).to(dev), cfg["k"], node_order=0)
    M = torch.from_numpy(cfg["M"]).to(dev)
    alpha = torch.tensor(cfg["alpha"], dtype=torch.float64, device=dev)
    mu = torch.empty(g.n, dtype=torch.float32, device=dev)
    t, K, m = cfg["t"], cfg["K"], int(M.shape[1])
    run = lambda: gs.gs_barycenter(ctx, g, M, alpha, t, K, iters, mu=mu)  # noqa: E731
    gs.gs_barycenter(ctx, g, M, alpha, t, K, 2, mu=mu)  # warm
    ms = _time(stream, run)
    gs.gs_sync(ctx)
    n, nnz = g.n, g.nnz
    g.close()
    # one iteration: w = M / H(vol v) (last order: gather, T, y, M, and the next input vol w) and
    # d = v H(vol w) with the geometric mean (gather, T, y, v read, v and the next input written,
    # and the [n] barycenter)
    per_iter = apply_bytes(n, nnz, K, m, 5) + apply_bytes(n, nnz, K, m, 6) + 4 * n
    orders = 2 * K * iters
    ach = per_iter * iters / (ms / 1e3) / 1e9
    return {"workload": "clusters-200k-R30, 32 cluster-union distributions, K = 40, t = 10", "n": n, "nnz": nnz,
            "B": m, "K": K, "iters": iters, "ms": ms, "iters_per_s": iters / (ms / 1e3),
            "order_us": ms * 1e3 / orders, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_kind": f"{peak_kind} hbm_gbs", "bytes_per_iter": per_iter,
            "mass": float(mu.double().sum())}


def combinatorial_case(gs, ctx, dev, stream, K=60):
    """The combinatorial-Laplacian filter exp(-t (D - A)) (rescaled by lam = 2 max degree) against
    the normalised-Laplacian filter on the 100k-point manifold graph, one column, the same degree K;
    t chosen so that the expansion's time s = t lam / 2 equals 5 (the normalised filter's t)."""
    import torch
    p = W.manifold_pair()
    g = gs.gs_build_graph(ctx, torch.from_numpy(p.X).to(dev), p.k)
    V = torch.from_numpy(p.a).to(dev)
    _, lam = gs.gs_heat_apply_combinatorial(ctx, g, 1.0, K, V)  # builds the operator, returns lam
    tc = 2.0 * 5.0 / lam
    out = {}
    ms_c = _time(stream, lambda: out.__setitem__("c", gs.gs_heat_apply_combinatorial(ctx, g, tc, K, V)[0]))
    gs.gs_heat_apply(ctx, g, 5.0, K, V)
    ms_n = _time(stream, lambda: out.__setitem__("n", gs.gs_heat_apply(ctx, g, 5.0, K, V)))
    gs.gs_sync(ctx)
    mass_in, mass_out = float(V.double().sum()), float(out["c"].double().sum())
    nnz = g.nnz
    g.close()
    return {"workload": "manifold-100k-R50, B = 1", "K": K, "lam": lam, "t": tc, "s": tc * lam / 2,
            "combinatorial_ms": ms_c, "normalised_ms": ms_n, "order_us": ms_c * 1e3 / K,
            "mass_rel_change": abs(mass_out - mass_in) / mass_in, "nnz_with_diagonal": nnz + p.X.shape[0]}


def matmul_peaks(dev, stream, N=8192, reps=10):
    """Dense-contraction roofs on this GPU: torch (cuBLAS) FP32 matmul with TF32 tensor cores and
    with plain FP32 (CUDA-core FMA), best of `reps` CUDA-event timings, 2 N^3 flops each."""
    import torch
    a = torch.randn(N, N, device=dev)
    b = torch.randn(N, N, device=dev)
    out = {}
    saved = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, tf32 in (("tf32_tflops", True), ("fp32_fma_tflops", False)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            for _ in range(3):
                torch.matmul(a, b)
            best = 1e30
            for _ in range(reps):
                best = min(best, _time(stream, lambda: torch.matmul(a, b)))
            out[name] = 2.0 * N ** 3 / (best / 1e3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = saved
    out["how"] = f"torch.matmul float32 {N}^3, best of {reps}, CUDA events (allow_tf32 on / off)"
    return out


def knn_case(gs, ctx, dev, stream, X, cfg, peaks, reps=3):
    """The kNN graph's distance screen on the headline workload (n = 100k in R^50, k = 15): time of
    the whole gs_knn call (screen, FP64 rerank, ordering of the lists) and the 3xTF32 tensor-core
    flops of the screen (3 MMAs of 128 x 128 x 8 per 8 augmented features, all padded query x
    candidate tiles), as a lower bound on the screen's TF32 rate and its fraction of the measured
    TF32 matmul peak."""
    n, d = X.shape
    gs.gs_knn(ctx, X, cfg["k"])
    ms = min(_time(stream, lambda: gs.gs_knn(ctx, X, cfg["k"])) for _ in range(reps))
    gs.gs_sync(ctx)
    npad = -(-n // 128) * 128
    kaug = -(-(d + 2) // 8) * 8
    flops = 3 * 2.0 * npad * npad * kaug
    tf = flops / (ms / 1e3) / 1e12
    return {"n": n, "d": d, "knn_ms": ms, "screen_tf32_flops": flops, "tflops_lower_bound": tf,
            "tf32_peak_tflops": peaks.get("tf32_tflops"),
            "frac_of_tf32_peak_lower_bound": tf / peaks["tf32_tflops"] if peaks.get("tf32_tflops") else None}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
