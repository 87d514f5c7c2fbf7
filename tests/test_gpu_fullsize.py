"""Parity at the configured full sizes, in the launch configuration bench.py times.

  * 100k-point manifold in R^50, k = 15 (the Sinkhorn workload): kNN lists of 200 sampled rows equal
    the oracle's brute-force lists; sigma is the median of the GPU's own kNN distances; the heat
    filter (K = 30, t = 5) is symmetric; 500 Sinkhorn iterations reach the b-marginal exactly and
    the a-marginal to the FP32 floor; loop modes agree bitwise.  Against the oracle in full: the
    GPU's graph equals the oracle's (edge set, sigma), and after the autotuner has picked the loop
    (as bench.py does) 500 iterations give W^2 within rtol 1e-4 and the scalings within rtol 1e-3
    of the FP64 oracle's on its own graph.
  * 200k-point cluster graph in R^30, k = 10, B = 32 (the barycenter workload): sampled kNN rows
    exact; the barycenter is positive with the invariant sum_i alpha_i ln v_i = 0; against the
    oracle in full, 20 barycenter iterations (K = 40, t = 10) match element by element (rtol 1e-4
    + 1e-6 max).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00805_gb300 import workloads as W
from tests.gpu_common import assert_close, knn_lists_match, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    from paper_2211_00805_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context()


def _sampled_knn_exact(gs, ctx, X, k, rows):
    idx, dist = gs.gs_knn(ctx, to_dev(X), k)
    ri, rd = oracle.knn(X.astype(np.float64), k, rows=rows)
    assert knn_lists_match(to_np(idx)[rows], to_np(dist)[rows], ri, rd, X, rows=rows) == 0
    return idx, dist


def test_manifold_100k_full_size(gs, ctx):
    p = W.manifold_pair()
    rows = np.random.default_rng(1).choice(len(p.X), 200, replace=False)
    idx, dist = _sampled_knn_exact(gs, ctx, p.X, p.k, rows)
    g = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    assert g.sigma == pytest.approx(float(np.median(to_np(dist).astype(np.float64))), rel=1e-6)
    # symmetry of p_K(L, t) at full size
    rng = np.random.default_rng(2)
    x, y = rng.random(g.n).astype(np.float32), rng.random(g.n).astype(np.float32)
    Hx = to_np(gs.gs_heat_apply(ctx, g, p.t, p.K, to_dev(x))).astype(np.float64)
    Hy = to_np(gs.gs_heat_apply(ctx, g, p.t, p.K, to_dev(y))).astype(np.float64)
    assert abs(y @ Hx - x @ Hy) <= 1e-5 * abs(y @ Hx)
    # Algorithm 1 at full size: exact nu-marginal after the w half-step, mu-marginal converged
    a, b = to_dev(p.a), to_dev(p.b)
    u, v, d, it = gs.gs_sinkhorn(ctx, g, a, b, p.t, p.K, p.iters)
    gs.gs_sync(ctx)
    Hu = gs.gs_heat_apply(ctx, g, p.t, p.K, u)
    Hv = gs.gs_heat_apply(ctx, g, p.t, p.K, v)
    marg_b = to_np(v * Hu).astype(np.float64)
    marg_a = to_np(u * Hv).astype(np.float64)
    assert np.abs(marg_b - p.b).sum() < 1e-5
    assert np.abs(marg_a - p.a).sum() < 1e-5  # this pair converges well inside 500 iterations
    assert np.isfinite(to_np(d)[0])
    # both loop modes, in bench's configuration, give identical results with exact exchange
    # words; the default 4-byte words stay within one unit in the last place per exchanged value
    gs.gs_set_option(ctx, gs.GS_OPT_B1_KERNEL, 1)
    outs = []
    for mode, word in ((0, 8), (1, 8), (0, 4)):
        gs.gs_set_option(ctx, gs.GS_OPT_LOOP, mode)
        gs.gs_set_option(ctx, gs.GS_OPT_TAG_WORD, word)
        r = gs.gs_sinkhorn(ctx, g, a, b, p.t, p.K, 50)
        outs.append(np.concatenate([to_np(r[0]), to_np(r[1]), to_np(r[2])]))
    gs.gs_set_option(ctx, gs.GS_OPT_LOOP, 2)
    gs.gs_set_option(ctx, gs.GS_OPT_TAG_WORD, 4)
    gs.gs_set_option(ctx, gs.GS_OPT_B1_KERNEL, 0)
    gs.gs_sync(ctx)
    assert np.array_equal(outs[0], outs[1], equal_nan=True)  # W is NaN where W^2 < 0
    n2 = 2 * g.n
    np.testing.assert_allclose(outs[2][:n2], outs[0][:n2], rtol=1e-4, atol=1e-6 * np.abs(outs[0][:n2]).max())
    assert outs[2][n2] == pytest.approx(outs[0][n2], rel=1e-6)


def test_clusters_200k_full_size(gs, ctx):
    cfg = W.clusters_barycenter()
    X, M = cfg["X"], cfg["M"]
    rows = np.random.default_rng(3).choice(len(X), 100, replace=False)
    _sampled_knn_exact(gs, ctx, X, cfg["k"], rows)
    g = gs.gs_build_graph(ctx, to_dev(X), cfg["k"])
    # the full-size cluster graph is connected (one component)
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    rowptr, col, A, P = gs.gs_graph_export_csr(ctx, g)
    Ah = csr_matrix((to_np(A), to_np(col), to_np(rowptr)), shape=(g.n, g.n))
    assert connected_components(Ah, directed=False)[0] == 1
    V = torch.empty((g.n, M.shape[1]), dtype=torch.float32, device="cuda")
    alpha = to_dev(cfg["alpha"], torch.float64)
    mu = to_np(gs.gs_barycenter(ctx, g, to_dev(M), alpha, cfg["t"], cfg["K"], 20, v_state=V))
    gs.gs_sync(ctx)
    assert np.all(mu >= 0) and np.isfinite(mu).all() and mu.sum() > 0
    # v_i <- v_i mu / d_i with mu = prod_i d_i^alpha_i and sum alpha = 1 keeps sum_i alpha_i ln v_i
    # at its initial value 0 on every row where all scalings stay positive
    Vn = to_np(V).astype(np.float64)
    ok = np.all((Vn > 0) & np.isfinite(Vn), axis=1)
    assert ok.mean() > 0.5
    L = np.log(Vn[ok])
    inv = L @ cfg["alpha"]
    assert np.all(np.abs(inv) <= 1e-4 * (1 + np.abs(L).max(axis=1)))


def _scaling_mask(marg, ref):
    return (marg > 0) & (np.abs(np.log(np.where(ref > 0, ref, 1))) < 80)


def test_manifold_100k_sinkhorn_matches_oracle(gs, ctx):
    # the headline workload in full: n = 100k, k = 15, K = 30, t = 5, 500 iterations
    p = W.manifold_pair()
    X64 = p.X.astype(np.float64)
    Ls, ex = oracle.build_graph(X64, p.k)
    g = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    rowptr, col, A, P = gs.gs_graph_export_csr(ctx, g)
    assert g.sigma == ex["sigma"]
    assert np.array_equal(to_np(rowptr), ex["rowptr"]) and np.array_equal(to_np(col), ex["col"])
    gs.gs_autotune(ctx, g, 1, p.K)  # the loop bench.py runs
    a, b = to_dev(p.a), to_dev(p.b)
    u, v, d, it = gs.gs_sinkhorn(ctx, g, a, b, p.t, p.K, p.iters)
    gs.gs_sync(ctx)
    r = oracle.sinkhorn(Ls, oracle.cheb_coefficients(p.t, p.K), p.a.astype(np.float64),
                        p.b.astype(np.float64), p.t, p.iters)
    assert r["status"] == oracle.OK
    assert to_np(d)[0] == pytest.approx(r["W2"], rel=1e-4)
    assert_close(to_np(u), r["v"], 1e-3, 0, "u", mask=_scaling_mask(p.a, r["v"]))
    assert_close(to_np(v), r["w"], 1e-3, 0, "v", mask=_scaling_mask(p.b, r["w"]))


def test_clusters_200k_barycenter_matches_oracle(gs, ctx):
    # the barycenter workload's graph and block (n = 200k, k = 10, B = 32, K = 40, t = 10) at 20
    # iterations, element by element
    cfg = W.clusters_barycenter()
    X, M = cfg["X"], cfg["M"]
    Ls, ex = oracle.build_graph(X.astype(np.float64), cfg["k"])
    g = gs.gs_build_graph(ctx, to_dev(X), cfg["k"])
    assert g.nnz == len(ex["col"]) and g.sigma == ex["sigma"]
    its = 20
    V = torch.empty((g.n, M.shape[1]), dtype=torch.float32, device="cuda")
    mu = to_np(gs.gs_barycenter(ctx, g, to_dev(M), to_dev(cfg["alpha"], torch.float64), cfg["t"], cfg["K"],
                                its, v_state=V))
    gs.gs_sync(ctx)
    ref, Vref = oracle.barycenter(Ls, oracle.cheb_coefficients(cfg["t"], cfg["K"]), M.astype(np.float64),
                                  cfg["alpha"], its, return_state=True)
    assert_close(mu, ref, 1e-4, 1e-6 * ref.max(), "mu (200k, B = 32)")
    assert_close(to_np(V), Vref, 1e-3, 1e-6 * np.abs(Vref).max(), "v_i (200k, B = 32)")
