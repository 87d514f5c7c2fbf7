"""GPU (FP32 CUDA path, through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances:
  * kNN edge sets: exact, except where the oracle's FP64 distances tie within 1e-6 relative;
    sigma: the same FP64 number (both sides rank bitwise-identical FP64 distances).
  * heat filter: |gpu - ref| <= 1e-4 |ref| + 1e-6 max|ref| per column block (FP32 sum of K terms of
    size up to max|ref|: entries far below the block's maximum carry that absolute floor).
  * distances and barycenters: rtol 1e-4; scalings: rtol 1e-3 where a_i > 0 and |ln u_i| < 80.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2211_00805_gb300 import workloads as W
from tests.gpu_common import assert_close, knn_lists_match, oracle_csr_to_dev, report, to_dev, to_np

pytestmark = pytest.mark.gpu

HEAT_RTOL, HEAT_ATOL_REL = 1e-4, 1e-6


@pytest.fixture(scope="module")
def gs():
    from paper_2211_00805_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context()


def _oracle_graph_fp32(rowptr, col, A):
    """Oracle operator built from the FP32-rounded affinities the GPU receives."""
    A32 = np.asarray(A, np.float32).astype(np.float64)
    deg, L = oracle.laplacian(rowptr, col, A32)
    return oracle.shifted(L), A32


def _random_graph(n, d, k, seed, wide=False):
    X = np.random.default_rng(seed).standard_normal((n, d)).astype(np.float32)
    idx, dist = oracle.knn(X.astype(np.float64), k)
    # wide: sigma = largest kNN distance, so no affinity underflows in FP32 on tiny clouds
    sig = float(dist.max()) if wide else oracle.median_sigma(dist)
    rp, col, A = oracle.affinity_graph(idx, dist, sig)
    return X, rp, col, A


def _cycle(n):
    rp = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    col = np.empty(2 * n, np.int32)
    for i in range(n):
        col[2 * i:2 * i + 2] = sorted([(i - 1) % n, (i + 1) % n])
    return rp, col, np.ones(2 * n)


# ------------------------------------------------------------------------------ coefficients
def test_library_coefficients_match_oracle(gs):
    for t, K in [(1.0, 20), (5.0, 30), (10.0, 40), (8.0, 40)]:
        c = np.array(gs.gs_cheb_coeffs(t, K))
        b = oracle.cheb_coefficients(t, K)
        # T_k(L - Id) = (-1)^k T_k(P): c_k = (-1)^k b_k, with b_0 halved
        ref = b * (-1.0) ** np.arange(K + 1)
        ref[0] *= 0.5
        np.testing.assert_allclose(c, ref, rtol=1e-12)


# ------------------------------------------------------------------------------- heat filter
@pytest.mark.parametrize("B", [1, 2, 3, 4, 5, 8, 12, 16, 32, 64, 100, 128, 132, 260])
def test_heat_apply_matches_oracle(gs, ctx, B):
    X, rp, col, A = _random_graph(1500, 3, 8, seed=B)
    g = gs.gs_graph_from_csr(ctx, *oracle_csr_to_dev(rp, col, A))
    Ls, _ = _oracle_graph_fp32(rp, col, A)
    V = np.random.default_rng(100 + B).random((1500, B)).astype(np.float32)
    for t, K in [(1.0, 20), (5.0, 30), (2.0, 1), (3.0, 2), (4.0, 3)]:
        Y = to_np(gs.gs_heat_apply(ctx, g, t, K, to_dev(V)))
        ref = oracle.heat_apply(Ls, oracle.cheb_coefficients(t, K), V.astype(np.float64))
        assert_close(Y, ref, HEAT_RTOL, HEAT_ATOL_REL * np.abs(ref).max(), f"B={B} t={t} K={K}")
    gs.gs_sync(ctx)


def test_heat_apply_misaligned_input(gs, ctx):
    # a contiguous view starting 4 bytes into its storage: the float4 path must not be used
    X, rp, col, A = _random_graph(900, 3, 8, seed=77)
    g = gs.gs_graph_from_csr(ctx, *oracle_csr_to_dev(rp, col, A))
    Ls, _ = _oracle_graph_fp32(rp, col, A)
    B = 32
    V = np.random.default_rng(7).random((900, B)).astype(np.float32)
    store = torch.empty(900 * B + 1, dtype=torch.float32, device="cuda")
    Vd = store[1:].view(900, B)
    Vd.copy_(to_dev(V))
    Y = to_np(gs.gs_heat_apply(ctx, g, 3.0, 25, Vd))
    ref = oracle.heat_apply(Ls, oracle.cheb_coefficients(3.0, 25), V.astype(np.float64))
    assert_close(Y, ref, HEAT_RTOL, HEAT_ATOL_REL * np.abs(ref).max(), "misaligned")
    with pytest.raises(gs.GeosinkError) as e:
        big = torch.empty(900 * 300 + 1, dtype=torch.float32, device="cuda")[1:].view(900, 300)
        gs.gs_heat_apply(ctx, g, 3.0, 5, big)
    assert e.value.status == gs.GS_ERR_UNSUPPORTED


def test_heat_apply_cycle_closed_form(gs, ctx):
    n = 97
    rp, col, A = _cycle(n)
    g = gs.gs_graph_from_csr(ctx, *oracle_csr_to_dev(rp, col, A))
    e0 = np.zeros(n, np.float32)
    e0[5] = 1.0
    t, K = 3.0, 30
    y = to_np(gs.gs_heat_apply(ctx, g, t, K, to_dev(e0)))
    m = np.arange(n)
    closed = (np.exp(-t * (1 - np.cos(2 * np.pi * m / n)))[None, :]
              * np.cos(2 * np.pi * np.outer(np.arange(n) - 5, m) / n)).sum(1) / n
    assert_close(y, closed, HEAT_RTOL, HEAT_ATOL_REL * closed.max(), "cycle")


def test_heat_apply_symmetric(gs, ctx):
    X, rp, col, A = _random_graph(3000, 4, 10, seed=9)
    g = gs.gs_graph_from_csr(ctx, *oracle_csr_to_dev(rp, col, A))
    rng = np.random.default_rng(3)
    x, y = rng.random(3000).astype(np.float32), rng.random(3000).astype(np.float32)
    Hx = to_np(gs.gs_heat_apply(ctx, g, 5.0, 30, to_dev(x))).astype(np.float64)
    Hy = to_np(gs.gs_heat_apply(ctx, g, 5.0, 30, to_dev(y))).astype(np.float64)
    assert abs(y @ Hx - x @ Hy) <= 1e-5 * abs(y @ Hx)


def test_heat_apply_ragged_small_graphs(gs, ctx):
    # sizes that leave partial row groups in the last block of every mapping
    for n in (3, 17, 33, 255, 257, 1029):
        X, rp, col, A = _random_graph(n, 2, 2, seed=n, wide=True)
        g = gs.gs_graph_from_csr(ctx, *oracle_csr_to_dev(rp, col, A))
        Ls, _ = _oracle_graph_fp32(rp, col, A)
        for B in (1, 4, 7):
            V = np.random.default_rng(n + B).random((n, B)).astype(np.float32)
            Y = to_np(gs.gs_heat_apply(ctx, g, 2.0, 12, to_dev(V)))
            ref = oracle.heat_apply(Ls, oracle.cheb_coefficients(2.0, 12), V.astype(np.float64))
            assert_close(Y, ref, HEAT_RTOL, HEAT_ATOL_REL * np.abs(ref).max(), f"n={n} B={B}")


# ------------------------------------------------------------------------------------- graph
def test_knn_sphere_exact(gs, ctx):
    p = W.sphere_pair()
    idx, dist = gs.gs_knn(ctx, to_dev(p.X), p.k)
    ri, rd = oracle.knn(p.X.astype(np.float64), p.k)
    assert knn_lists_match(to_np(idx), to_np(dist), ri, rd, p.X) == 0
    np.testing.assert_allclose(to_np(dist), rd, rtol=1e-7)


def test_knn_manifold_sampled_rows(gs, ctx):
    X, Z = W.tanh_manifold(20_000, 10, 50, seed=2)
    idx, dist = gs.gs_knn(ctx, to_dev(X), 15)
    rows = np.random.default_rng(0).choice(len(X), 300, replace=False)
    ri, rd = oracle.knn(X.astype(np.float64), 15, rows=rows)
    # the rerank uses the oracle's FP64 operation order, so even near-ties come out the same
    assert knn_lists_match(to_np(idx)[rows], to_np(dist)[rows], ri, rd, X, rows=rows) == 0


def test_knn_screen_in_caller_order_above_the_bisection_limit(gs, ctx):
    # With more points than the persistent loop's partition can bisect (152 parts of at most 4,096
    # points on this GPU) the tensor-memory screen sweeps the candidates in the caller's order
    # instead of the bisection order; lists and ties follow the same (distance, index) order.
    X, _ = W.tanh_manifold(700_000, 4, 8, seed=9)
    idx, dist = gs.gs_knn(ctx, to_dev(X), 10)
    rows = np.random.default_rng(1).choice(len(X), 200, replace=False)
    ri, rd = oracle.knn(X.astype(np.float64), 10, rows=rows)
    assert knn_lists_match(to_np(idx)[rows], to_np(dist)[rows], ri, rd, X, rows=rows) == 0


def test_build_graph_matches_oracle(gs, ctx):
    p = W.sphere_pair()
    g = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    rowptr, col, A, P = gs.gs_graph_export_csr(ctx, g)
    Ls, ex = oracle.build_graph(p.X.astype(np.float64), p.k)
    assert g.sigma == ex["sigma"]
    assert np.array_equal(to_np(rowptr), ex["rowptr"])
    assert np.array_equal(to_np(col), ex["col"])
    assert_close(to_np(A), ex["A"], 1e-7, 0, "A")
    # P_ij = -(Ls)_ij on the same pattern (Ls = L - Id has no diagonal)
    assert np.array_equal(Ls[1], ex["col"])
    assert_close(to_np(P), -Ls[2], 1e-6, 0, "P")


def test_build_graph_with_given_sigma_and_duplicates(gs, ctx):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((700, 5)).astype(np.float32)
    X[100:110] = X[3]  # exact duplicates: distance ties at 0, resolved by index
    g = gs.gs_build_graph(ctx, to_dev(X), 6, sigma=0.7)
    rowptr, col, A, P = gs.gs_graph_export_csr(ctx, g)
    Ls, ex = oracle.build_graph(X.astype(np.float64), 6, sigma=0.7)
    assert g.sigma == pytest.approx(0.7, rel=1e-7)
    assert np.array_equal(to_np(col), ex["col"])
    assert_close(to_np(A), ex["A"], 1e-6, 0, "A")


def test_point_graph_order_gives_compact_blocks(gs, ctx):
    # a graph built from points is ordered by recursive coordinate bisection into the persistent
    # loop's blocks; the same graph given as CSR gets the breadth-first order.  The bisection
    # leaves each block fewer distinct neighbour columns, and both orders give the same operator.
    X, Z = W.tanh_manifold(30_000, 10, 50, seed=2)
    g = gs.gs_build_graph(ctx, to_dev(X), 15)
    rowptr, col, A, _ = gs.gs_graph_export_csr(ctx, g)
    g2 = gs.gs_graph_from_csr(ctx, rowptr, col, A)
    lay, lay2 = gs.gs_graph_layout(g), gs.gs_graph_layout(g2)
    assert lay["blocks"] == lay2["blocks"]
    assert lay["sum_block_distinct"] < 0.9 * lay2["sum_block_distinct"]
    a = W.softmax_bump(Z, np.zeros(Z.shape[1]))
    b = W.softmax_bump(Z, np.full(Z.shape[1], 0.5))
    out = []
    for graph in (g, g2):
        u, v, d, _ = gs.gs_sinkhorn(ctx, graph, to_dev(a), to_dev(b), 5.0, 30, 100)
        gs.gs_sync(ctx)
        out.append((to_np(u), to_np(d)[0]))
    assert out[0][1] == pytest.approx(out[1][1], rel=1e-5)
    m = out[1][0] > 0
    np.testing.assert_allclose(out[0][0][m], out[1][0][m], rtol=1e-3)


# ---------------------------------------------------------------------------------- Sinkhorn
@pytest.fixture(scope="module")
def sphere_graph(gs, ctx):
    p = W.sphere_pair()
    g = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    Ls, ex = oracle.build_graph(p.X.astype(np.float64), p.k)
    return p, g, Ls


def _check_sinkhorn(gs, ctx, g, Ls, a, b, t, K, iters, vol=None):
    u, v, dist, it = gs.gs_sinkhorn(ctx, g, to_dev(a), to_dev(b), t, K, iters,
                                    vol=None if vol is None else to_dev(vol))
    gs.gs_sync(ctx)
    r = oracle.sinkhorn(Ls, oracle.cheb_coefficients(t, K), a.astype(np.float64),
                        b.astype(np.float64), t, iters, a=None if vol is None else vol.astype(np.float64))
    assert r["status"] == oracle.OK
    d = to_np(dist)
    assert d[0] == pytest.approx(r["W2"], rel=1e-4)
    if r["W2"] >= 0:  # W = sqrt(W^2) is real only then (W^2 = 4t (1 + KL) can be negative)
        assert d[1] == pytest.approx(r["W"], rel=1e-4)
    else:
        assert math.isnan(d[1])
    uu, vv = to_np(u), to_np(v)
    mu = (a > 0) & (np.abs(np.log(np.where(r["v"] > 0, r["v"], 1))) < 80)
    mv = (b > 0) & (np.abs(np.log(np.where(r["w"] > 0, r["w"], 1))) < 80)
    assert_close(uu, r["v"], 1e-3, 0, "u", mask=mu)
    assert_close(vv, r["w"], 1e-3, 0, "v", mask=mv)
    assert int(to_np(it)[0]) == iters
    return d


def test_sinkhorn_sphere_t5(gs, ctx, sphere_graph):
    p, g, Ls = sphere_graph
    _check_sinkhorn(gs, ctx, g, Ls, p.a, p.b, 5.0, 30, 200)


def test_sinkhorn_sphere_t1_reports_nonfinite(gs, ctx, sphere_graph):
    # t = 1, K = 20 as configured: the FP32 scalings overflow (recorded deviation); the library
    # must say so instead of returning garbage.
    p, g, Ls = sphere_graph
    gs.gs_sinkhorn(ctx, g, to_dev(p.a), to_dev(p.b), 1.0, 20, 200)
    with pytest.raises(gs.GeosinkError) as e:
        gs.gs_sync(ctx)
    assert e.value.status == gs.GS_ERR_NONFINITE


def test_sinkhorn_vertex_weights_zero_mass_odd_K(gs, ctx, sphere_graph):
    p, g, Ls = sphere_graph
    vol = np.random.default_rng(1).uniform(0.5, 1.5, len(p.a)).astype(np.float32)
    a = np.where(p.X[:, 2] > -0.2, p.a, 0).astype(np.float32)
    a = (a / np.sum(a * vol)).astype(np.float32)
    b = (p.b / np.sum(p.b * vol)).astype(np.float32)
    _check_sinkhorn(gs, ctx, g, Ls, a, b, 5.0, 31, 120, vol=vol)


def test_distance_equals_sinkhorn(gs, ctx, sphere_graph):
    p, g, Ls = sphere_graph
    d = to_np(gs.gs_distance(ctx, g, to_dev(p.a), to_dev(p.b), 5.0, 30, 100))
    _, _, d2, _ = gs.gs_sinkhorn(ctx, g, to_dev(p.a), to_dev(p.b), 5.0, 30, 100)
    assert np.array_equal(d, to_np(d2))


def test_sinkhorn_eps_stop_matches_oracle(gs, ctx, sphere_graph):
    p, g, Ls = sphere_graph
    t, K = 5.0, 30
    r = oracle.sinkhorn(Ls, oracle.cheb_coefficients(t, K), p.a.astype(np.float64),
                        p.b.astype(np.float64), t, 400, eps=1e-5)
    u, v, dist, it = gs.gs_sinkhorn(ctx, g, to_dev(p.a), to_dev(p.b), t, K, 400, eps=1e-5)
    gs.gs_sync(ctx)
    assert r["status"] == oracle.OK
    assert abs(int(to_np(it)[0]) - r["iters"]) <= 10
    assert to_np(dist)[0] == pytest.approx(r["W2"], rel=1e-4)
    gs.gs_sinkhorn(ctx, g, to_dev(p.a), to_dev(p.b), t, K, 20, eps=1e-30)
    with pytest.raises(gs.GeosinkError) as e:
        gs.gs_sync(ctx)
    assert e.value.status == gs.GS_ERR_NOT_CONVERGED


def test_sinkhorn_manifold_small(gs, ctx):
    p = W.manifold_pair(n=6000, iters=150)
    g = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    Ls, ex = oracle.build_graph(p.X.astype(np.float64), p.k)
    assert g.nnz == len(ex["col"])
    _check_sinkhorn(gs, ctx, g, Ls, p.a, p.b, p.t, p.K, p.iters)


# -------------------------------------------------------------------------------- barycenter
@pytest.mark.parametrize("m", [1, 3, 32, 64])
def test_barycenter_matches_oracle(gs, ctx, m):
    cfg = W.clusters_barycenter(n=4000, m=max(m, 1), iters=30)
    X = cfg["X"]
    M = cfg["M"][:, :m]
    alpha = np.random.default_rng(m).dirichlet(np.ones(m))
    g = gs.gs_build_graph(ctx, to_dev(X), cfg["k"])
    Ls, ex = oracle.build_graph(X.astype(np.float64), cfg["k"])
    t, K = 10.0, 40
    V = torch.empty((len(X), m), dtype=torch.float32, device="cuda")
    mu = to_np(gs.gs_barycenter(ctx, g, to_dev(M), to_dev(alpha, torch.float64), t, K, cfg["iters"],
                                v_state=V))
    gs.gs_sync(ctx)
    ref, Vref = oracle.barycenter(Ls, oracle.cheb_coefficients(t, K), M.astype(np.float64), alpha,
                                  cfg["iters"], return_state=True)
    assert_close(mu, ref, 1e-4, 1e-6 * ref.max(), f"mu m={m}")
    assert_close(to_np(V), Vref, 1e-3, 1e-6 * np.abs(Vref).max(), f"v_i m={m}")


@pytest.mark.parametrize("m", [3, 32])
def test_barycenter_with_vertex_weights_matches_oracle(gs, ctx, m):
    # vertex weights enter both filter inputs of every iteration (vol v_i, vol w_i); the inputs
    # are densities of equal weighted mass sum(vol mu_i); one-column-per-lane (m = 3) and float4
    # row-group (m = 32) kernels
    cfg = W.clusters_barycenter(n=4000, m=m, iters=30)
    X = cfg["X"]
    vol = np.random.default_rng(40 + m).uniform(0.7, 1.3, len(X)).astype(np.float32)
    M = cfg["M"][:, :m].astype(np.float64)
    M = (M / (vol.astype(np.float64) @ M)).astype(np.float32)
    alpha = np.random.default_rng(m).dirichlet(np.ones(m))
    g = gs.gs_build_graph(ctx, to_dev(X), cfg["k"])
    Ls, ex = oracle.build_graph(X.astype(np.float64), cfg["k"])
    t, K = 10.0, 40
    mu = to_np(gs.gs_barycenter(ctx, g, to_dev(M), to_dev(alpha, torch.float64), t, K, cfg["iters"],
                                vol=to_dev(vol)))
    gs.gs_sync(ctx)
    ref = oracle.barycenter(Ls, oracle.cheb_coefficients(t, K), M.astype(np.float64), alpha, cfg["iters"],
                            a=vol.astype(np.float64))
    assert_close(mu, ref, 1e-4, 1e-6 * ref.max(), f"mu m={m}, vertex weights")


# ------------------------------------------------------------------------- loop modes, faults
def _broad_pair(p):
    # a broad bump (vMF, kappa = 1) and a mild tilt of it: with the one- and two-hop kernels of
    # K = 1, 2 (zero between farther nodes) the scalings stay within e^{+-40}, inside FP32's range
    ez = np.array([0.0, 0.0, 1.0])
    a = W.vmf_bump(p.X, ez, 1.0)
    b = a * (1.0 + 0.3 * p.X[:, 0])
    return a, (b / b.sum()).astype(np.float32)


@pytest.mark.parametrize("t,K", [(5.0, 30), (0.5, 1), (1.0, 2)])
def test_persistent_and_graph_loops_agree(gs, ctx, sphere_graph, t, K):
    # every persistent form (graph from global memory, slices in shared memory, gather cache with a
    # grid barrier, neighbour flags or tagged values re-read in groups or one at a time) and graph
    # replay of the thread-per-row sliced-ELL kernel
    # sum in the same order; K = 1 (the only order is first and last) and K = 2 are the edge cases
    p, g, Ls = sphere_graph
    a, b = (p.a, p.b) if K > 2 else _broad_pair(p)
    out = {}
    gs.gs_set_option(ctx, gs.GS_OPT_B1_KERNEL, 1)
    gs.gs_set_option(ctx, gs.GS_OPT_TAG_WORD, 8)  # exact exchange words: bitwise comparable
    for cfg in ((0, 1, 1), (0, 0, 1), (0, 2, 0), (0, 2, 1), (0, 2, 2), (0, 2, 4), (1, 1, 1)):
        mode, smem, sync = cfg
        gs.gs_set_option(ctx, gs.GS_OPT_LOOP, mode)
        gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SMEM_GRAPH, smem)
        gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SYNC, sync)
        u, v, d, _ = gs.gs_sinkhorn(ctx, g, to_dev(a), to_dev(b), t, K, 120)
        gs.gs_sync(ctx)
        out[cfg] = (to_np(u), to_np(v), to_np(d))
    # the same points partitioned into two 512-thread blocks per SM (tagged values, neighbour flags);
    # the node order follows the partition (coordinate bisection), so this graph sums each row in
    # its own order: its two forms agree bitwise with each other, and with the first graph to rounding
    gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_BLOCKS, 2)
    try:
        g2 = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_BLOCKS, 1)
    assert gs.gs_graph_layout(g2)["blocks"] == 2 * gs.gs_graph_layout(g)["blocks"]
    gs.gs_set_option(ctx, gs.GS_OPT_LOOP, 0)
    gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SMEM_GRAPH, 2)
    out2 = {}
    for sync in (2, 4, 1):
        gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SYNC, sync)
        u, v, d, _ = gs.gs_sinkhorn(ctx, g2, to_dev(a), to_dev(b), t, K, 120)
        gs.gs_sync(ctx)
        out2[sync] = (to_np(u), to_np(v), to_np(d))
    # default 4-byte exchange words (values read across blocks within one unit in the last place)
    gs.gs_set_option(ctx, gs.GS_OPT_TAG_WORD, 4)
    gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SYNC, 2)
    u4, v4, d4, _ = gs.gs_sinkhorn(ctx, g, to_dev(a), to_dev(b), t, K, 120)
    gs.gs_sync(ctx)
    gs.gs_set_option(ctx, gs.GS_OPT_LOOP, 2)
    gs.gs_set_option(ctx, gs.GS_OPT_B1_KERNEL, 0)
    gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SMEM_GRAPH, 2)
    gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SYNC, 3)
    for key in out:
        for i in range(3):
            np.testing.assert_array_equal(out[(0, 1, 1)][i], out[key][i], err_msg=str(key))
    ref = out[(0, 1, 1)]
    for i in range(3):
        np.testing.assert_array_equal(out2[2][i], out2[1][i], err_msg="two blocks per SM")
        np.testing.assert_array_equal(out2[4][i], out2[1][i], err_msg="two blocks per SM, one at a time")
    assert out2[2][2][0] == pytest.approx(ref[2][0], rel=1e-6)
    for got, want in ((out2[2][0], ref[0]), (out2[2][1], ref[1])):
        m = want > 0
        np.testing.assert_allclose(got[m], want[m], rtol=1e-4)
    assert to_np(d4)[0] == pytest.approx(ref[2][0], rel=1e-6)
    for got, want in ((to_np(u4), ref[0]), (to_np(v4), ref[1])):
        m = want > 0
        np.testing.assert_allclose(got[m], want[m], rtol=1e-4)


def test_node_order_option_gives_the_oracle_results(gs, ctx, sphere_graph):
    # GS_OPT_NODE_ORDER 0 (decreasing degree inside each bisection part) and 1 (degree classes, then
    # the reading block, the default) lay the same graph out differently; both give the oracle's
    # filter and Sinkhorn results (up to summation order)
    p, g1, Ls = sphere_graph
    assert gs.gs_get_option(ctx, gs.GS_OPT_NODE_ORDER) == 1
    gs.gs_set_option(ctx, gs.GS_OPT_NODE_ORDER, 0)
    try:
        g0 = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_NODE_ORDER, 1)
    V = np.random.default_rng(3).random((len(p.X), 32)).astype(np.float32)
    ref = oracle.heat_apply(Ls, oracle.cheb_coefficients(5.0, 30), V.astype(np.float64))
    for g in (g0, g1):
        Y = to_np(gs.gs_heat_apply(ctx, g, 5.0, 30, to_dev(V)))
        assert_close(Y, ref, HEAT_RTOL, HEAT_ATOL_REL * np.abs(ref).max(), "node order")
        _check_sinkhorn(gs, ctx, g, Ls, p.a, p.b, 5.0, 30, 60)
    with pytest.raises(gs.GeosinkError):
        gs.gs_set_option(ctx, gs.GS_OPT_NODE_ORDER, 2)


def test_register_rows_loop_matches_shared_memory_form_and_oracle(gs, ctx):
    # GS_OPT_LOOP_REGS: the tagged 4-byte loop with each row's first 16 entries in registers sums
    # in the shared-memory form's order, so both give bitwise the same u, v and distance (both
    # staging forms); rows here run from under 8 to over 40 entries, odd and even widths, so the
    # register blocks, the register tail and the shared-memory continuation all take part
    p = W.manifold_pair(n=6000, iters=80)
    g = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    Ls, ex = oracle.build_graph(p.X.astype(np.float64), p.k)
    deg = np.diff(ex["rowptr"])
    assert deg.max() > 32 and deg.min() < 16 and (deg % 2 == 1).any()
    assert gs.gs_get_option(ctx, gs.GS_OPT_LOOP_REGS) == 1
    gs.gs_set_option(ctx, gs.GS_OPT_LOOP, 0)
    gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SMEM_GRAPH, 2)
    gs.gs_set_option(ctx, gs.GS_OPT_TAG_WORD, 4)
    out = {}
    try:
        for sync in (2, 4):
            gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SYNC, sync)
            for regs in (1, 0):
                gs.gs_set_option(ctx, gs.GS_OPT_LOOP_REGS, regs)
                u, v, d, _ = gs.gs_sinkhorn(ctx, g, to_dev(p.a), to_dev(p.b), p.t, p.K, p.iters)
                gs.gs_sync(ctx)
                out[(sync, regs)] = (to_np(u), to_np(v), to_np(d))
        gs.gs_set_option(ctx, gs.GS_OPT_LOOP_REGS, 1)
        gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SYNC, 2)
        _check_sinkhorn(gs, ctx, g, Ls, p.a, p.b, p.t, p.K, p.iters)
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_LOOP_REGS, 1)
        gs.gs_set_option(ctx, gs.GS_OPT_LOOP, 2)
        gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SYNC, 3)
    for sync in (2, 4):
        for i in range(3):
            np.testing.assert_array_equal(out[(sync, 1)][i], out[(sync, 0)][i], err_msg=f"sync {sync}")
    with pytest.raises(gs.GeosinkError):
        gs.gs_set_option(ctx, gs.GS_OPT_LOOP_REGS, 2)


def test_sinkhorn_single_order_filter_matches_oracle(gs, ctx, sphere_graph):
    # K = 1: H = c_0 I + c_1 P, positive for t = 0.5 (I_0(t) > 2 I_1(t)); persistent default path
    p, g, Ls = sphere_graph
    a, b = _broad_pair(p)
    _check_sinkhorn(gs, ctx, g, Ls, a, b, 0.5, 1, 60)


@pytest.mark.parametrize("sync,word", [(0, 4), (1, 4), (2, 4), (2, 8), (4, 4), (4, 8)])
def test_persistent_barrier_timeout_is_reported_and_context_survives(gs, ctx, sphere_graph, sync, word):
    # the self-test makes every block wait for an arrival (or a stage) that never comes; the
    # bounded wait runs out, the launch ends, gs_sync reports the timeout, and the next call works
    p, g, Ls = sphere_graph
    gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SYNC, sync)
    gs.gs_set_option(ctx, gs.GS_OPT_TAG_WORD, word)
    gs.gs_set_option(ctx, gs.GS_OPT_BARRIER_SELFTEST, 1)
    gs.gs_sinkhorn(ctx, g, to_dev(p.a), to_dev(p.b), 5.0, 30, 10)
    with pytest.raises(gs.GeosinkError) as e:
        gs.gs_sync(ctx)
    assert e.value.status == gs.GS_ERR_TIMEOUT
    _check_sinkhorn(gs, ctx, g, Ls, p.a, p.b, 5.0, 30, 50)
    gs.gs_set_option(ctx, gs.GS_OPT_PERSIST_SYNC, 3)
    gs.gs_set_option(ctx, gs.GS_OPT_TAG_WORD, 4)


@pytest.mark.parametrize("B,option,variant", [(1, 3, 1), (1, 3, 2), (1, 3, 3), (1, 3, 5), (1, 3, 6), (1, 3, 7), (32, 4, 2),
                                              (32, 4, 3), (32, 4, 4), (32, 4, 5), (64, 4, 3),
                                              (8, 4, 3), (128, 4, 3), (12, 4, 5), (3, 4, 5),
                                              (32, 4, 8), (32, 4, 9), (64, 4, 8), (64, 4, 9),
                                              (128, 4, 8), (128, 4, 9), (12, 4, 8), (96, 4, 9)])
def test_kernel_variants_match_oracle(gs, ctx, B, option, variant):
    # every order-kernel variant (sliced ELL, lane-split CSR, chunked async gathers, staged lists)
    X, rp, col, A = _random_graph(2500, 4, 9, seed=31 + B)
    g = gs.gs_graph_from_csr(ctx, *oracle_csr_to_dev(rp, col, A))
    Ls, _ = _oracle_graph_fp32(rp, col, A)
    V = np.random.default_rng(B).random((2500, B)).astype(np.float32)
    gs.gs_set_option(ctx, option, variant)
    try:
        for t, K in [(5.0, 30), (2.0, 1), (3.0, 2)]:
            Y = to_np(gs.gs_heat_apply(ctx, g, t, K, to_dev(V)))
            ref = oracle.heat_apply(Ls, oracle.cheb_coefficients(t, K), V.astype(np.float64))
            assert_close(Y, ref, HEAT_RTOL, HEAT_ATOL_REL * np.abs(ref).max(), f"B={B} v={variant} K={K}")
        gs.gs_sync(ctx)
    finally:
        gs.gs_set_option(ctx, option, 0)


def _hub_graph(n, seed):
    """A kNN graph with hub rows added (degrees 40 to 400, far above the split threshold of the
    B > 1 kernel), as high-dimensional kNN graphs have; symmetric, weights in (0, 1]."""
    import scipy.sparse as sp
    X, rp, col, A = _random_graph(n, 4, 9, seed)
    rows = np.repeat(np.arange(n), np.diff(rp))
    Msp = sp.csr_matrix((A, (rows, col)), shape=(n, n))
    rng = np.random.default_rng(seed)
    hubs = rng.choice(n, 8, replace=False)
    hr, hc = [], []
    for h, deg in zip(hubs, [40, 60, 97, 150, 233, 300, 333, 400]):
        nb = rng.choice(np.setdiff1d(np.arange(n), [h]), deg, replace=False)
        hr += [h] * deg
        hc += list(nb)
    H = sp.csr_matrix((rng.uniform(0.05, 1.0, len(hr)), (hr, hc)), shape=(n, n))
    G = Msp.maximum(Msp.T).maximum(H).maximum(H.T).tocsr()
    G.sort_indices()
    return G.indptr.astype(np.int64), G.indices.astype(np.int32), G.data.astype(np.float64)


@pytest.mark.parametrize("B,variant", [(2, 0), (3, 0), (8, 0), (12, 0), (32, 0), (64, 0), (128, 0), (200, 0),
                                       (32, 8), (32, 9), (64, 8), (64, 9), (128, 8), (128, 9)])
def test_long_rows_split_across_a_warp_match_oracle(gs, ctx, B, variant):
    # rows longer than the split threshold are summed by a whole warp in segments
    rp, col, A = _hub_graph(3000, 71)
    assert np.diff(rp).max() >= 400
    g = gs.gs_graph_from_csr(ctx, *oracle_csr_to_dev(rp, col, A))
    Ls, _ = _oracle_graph_fp32(rp, col, A)
    V = np.random.default_rng(B).random((3000, B)).astype(np.float32)
    gs.gs_set_option(ctx, gs.GS_OPT_BLK_KERNEL, variant)
    try:
        for t, K in [(5.0, 30), (2.0, 1), (3.0, 2)]:
            Y = to_np(gs.gs_heat_apply(ctx, g, t, K, to_dev(V)))
            ref = oracle.heat_apply(Ls, oracle.cheb_coefficients(t, K), V.astype(np.float64))
            assert_close(Y, ref, HEAT_RTOL, HEAT_ATOL_REL * np.abs(ref).max(), f"B={B} v={variant} K={K}")
        Y1 = to_np(gs.gs_heat_apply(ctx, g, 5.0, 30, to_dev(V)))
        Y2 = to_np(gs.gs_heat_apply(ctx, g, 5.0, 30, to_dev(V)))
        assert np.array_equal(Y1, Y2)  # the segment order is fixed: repeatable bit for bit
        gs.gs_sync(ctx)
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_BLK_KERNEL, 0)


@pytest.mark.parametrize("m,variant", [(1, 0), (32, 0), (32, 8), (32, 9), (64, 8), (64, 9)])
def test_barycenter_on_hub_graph_matches_oracle(gs, ctx, m, variant):
    # the barycenter epilogue (geometric mean across the row's lanes) on split rows
    rp, col, A = _hub_graph(3000, 72)
    g = gs.gs_graph_from_csr(ctx, *oracle_csr_to_dev(rp, col, A))
    Ls, _ = _oracle_graph_fp32(rp, col, A)
    rng = np.random.default_rng(m)
    M = rng.random((3000, m)) + 0.1
    M = (M / M.sum(0)).astype(np.float32)
    alpha = rng.dirichlet(np.ones(m))
    t, K, iters = 5.0, 20, 10
    gs.gs_set_option(ctx, gs.GS_OPT_BLK_KERNEL, variant)
    try:
        mu = to_np(gs.gs_barycenter(ctx, g, to_dev(M), to_dev(alpha, torch.float64), t, K, iters))
        gs.gs_sync(ctx)
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_BLK_KERNEL, 0)
    ref = oracle.barycenter(Ls, oracle.cheb_coefficients(t, K), M.astype(np.float64), alpha, iters)
    assert_close(mu, ref, 1e-4, 1e-6 * ref.max(), f"mu m={m} v={variant}")


@pytest.mark.parametrize("tensor", [2, 1, 0])
def test_knn_tensor_core_and_cuda_core_screens_exact(gs, ctx, tensor):
    # 2: tcgen05 screen, 1: warp-level TF32 MMA, 0: CUDA cores; all must give the oracle's lists
    X, Z = W.tanh_manifold(3000, 8, 24, seed=9)
    saved = gs.gs_get_option(ctx, gs.GS_OPT_KNN_TENSOR)
    gs.gs_set_option(ctx, gs.GS_OPT_KNN_TENSOR, tensor)
    try:
        idx, dist = gs.gs_knn(ctx, to_dev(X), 12)
        gs.gs_sync(ctx)
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_KNN_TENSOR, saved)
    ri, rd = oracle.knn(X.astype(np.float64), 12)
    assert knn_lists_match(to_np(idx), to_np(dist), ri, rd, X) == 0
    np.testing.assert_allclose(to_np(dist), rd, rtol=1e-7)


@pytest.mark.parametrize("n,d,k", [(2999, 50, 15), (1000, 62, 10), (777, 3, 10), (40, 30, 24), (30, 12, 20),
                                   (130, 5, 8), (600, 70, 10)])
def test_knn_tcgen05_screen_shapes_exact(gs, ctx, n, d, k):
    # augmented width d + 2 in one or two 32-feature blocks, ragged last query / candidate tiles,
    # fewer points than screened candidates, and d = 70 (beyond the kernel: falls back)
    X = np.random.default_rng(n + d).standard_normal((n, d)).astype(np.float32)
    saved = gs.gs_get_option(ctx, gs.GS_OPT_KNN_TENSOR)
    gs.gs_set_option(ctx, gs.GS_OPT_KNN_TENSOR, 2)
    try:
        idx, dist = gs.gs_knn(ctx, to_dev(X), k)
        gs.gs_sync(ctx)
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_KNN_TENSOR, saved)
    ri, rd = oracle.knn(X.astype(np.float64), k)
    assert knn_lists_match(to_np(idx), to_np(dist), ri, rd, X) == 0
    np.testing.assert_allclose(to_np(dist), rd, rtol=1e-7)



def test_knn_tcgen05_screen_exact_ties(gs, ctx):
    # duplicated points give exactly tied distances, broken by index on both sides
    base = np.random.default_rng(11).standard_normal((400, 20)).astype(np.float32)
    X = np.concatenate([base, base, base[:150]])
    saved = gs.gs_get_option(ctx, gs.GS_OPT_KNN_TENSOR)
    gs.gs_set_option(ctx, gs.GS_OPT_KNN_TENSOR, 2)
    try:
        idx, dist = gs.gs_knn(ctx, to_dev(X), 10)
        gs.gs_sync(ctx)
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_KNN_TENSOR, saved)
    ri, rd = oracle.knn(X.astype(np.float64), 10)
    assert np.array_equal(to_np(idx), ri)
    np.testing.assert_allclose(to_np(dist), rd, rtol=1e-7, atol=1e-30)
