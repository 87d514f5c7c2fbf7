"""GPU reverse mode (gs_sinkhorn_grad / gs_barycenter_grad, the autograd wrappers) and the batched
persistent solver (gs_sinkhorn_batched) against the FP64 oracle and the single-problem path.

Gradient tolerance: |gpu - ref| <= 2e-4 |ref| + 1e-4 max|ref|.  The reverse sweep is 2 * iters
FP32 filter applies deep, each adding ~K eps_32 relative error to values whose sizes span the
whole vector, so entries far below the maximum carry an absolute floor.  Measured against the
oracle's reverse mode on the 1,500-point sphere pair (30 and 200 iterations): the largest error of
dW^2/da is 9.4e-5 of max|ref| (5.6e-5 at 200 iterations), of dW^2/db 4.7e-5; of the barycenter's
weight gradient 1.7e-6.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00805_gb300 import workloads as W
from tests.gpu_common import assert_close, to_dev, to_np

pytestmark = pytest.mark.gpu

GRTOL, GATOL_REL = 2e-4, 1e-4


@pytest.fixture(scope="module")
def gs():
    from paper_2211_00805_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context()


@pytest.fixture(scope="module")
def sphere(gs, ctx):
    p = W.sphere_pair(n=1500, kappa=8.0)
    g = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    Ls, ex = oracle.build_graph(p.X.astype(np.float64), p.k)
    return p, g, Ls


@pytest.mark.parametrize("ck", [1, 7, 30])
def test_sinkhorn_grad_matches_oracle(gs, ctx, sphere, ck):
    p, g, Ls = sphere
    t, K, it = 5.0, 30, 30
    vol = np.random.default_rng(3).uniform(0.7, 1.3, len(p.a)).astype(np.float32)
    # marginals of equal mass with respect to the vertex weights (Algorithm 1's plan has marginals
    # vol * a and vol * b)
    a = (p.a / np.sum(p.a * vol)).astype(np.float32)
    b = (p.b / np.sum(p.b * vol)).astype(np.float32)
    dist, ga, gb = gs.gs_sinkhorn_grad(ctx, g, to_dev(a), to_dev(b), t, K, it, checkpoint=ck,
                                       vol=to_dev(vol))
    gs.gs_sync(ctx)
    W2, rga, rgb = oracle.sinkhorn_grad(Ls, oracle.cheb_coefficients(t, K), a.astype(np.float64),
                                        b.astype(np.float64), t, it, a=vol.astype(np.float64))
    assert to_np(dist)[0] == pytest.approx(W2, rel=1e-4)
    assert_close(to_np(ga), rga, GRTOL, GATOL_REL * np.abs(rga).max(), f"dW2/da ck={ck}")
    assert_close(to_np(gb), rgb, GRTOL, GATOL_REL * np.abs(rgb).max(), f"dW2/db ck={ck}")


def test_sinkhorn_grad_checkpoint_invariant(gs, ctx, sphere):
    p, g, Ls = sphere
    outs = [gs.gs_sinkhorn_grad(ctx, g, to_dev(p.a), to_dev(p.b), 5.0, 30, 25, checkpoint=c)
            for c in (1, 4, 25)]
    for d, ga, gb in outs[1:]:
        assert torch.equal(ga, outs[0][1]) and torch.equal(gb, outs[0][2])


def test_sinkhorn_grad_vs_oracle_finite_differences(gs, ctx, sphere):
    # GPU gradient against FP64 central differences of the oracle's forward map (relative step
    # 1e-4 a_i, as the differentiation workload prescribes), on the largest-mass coordinates
    p, g, Ls = sphere
    t, K, it = 5.0, 30, 20
    a64, b64 = p.a.astype(np.float64), p.b.astype(np.float64)
    bk = oracle.cheb_coefficients(t, K)
    _, ga, _ = gs.gs_sinkhorn_grad(ctx, g, to_dev(p.a), to_dev(p.b), t, K, it)
    ga = to_np(ga)
    for i in np.argsort(-a64)[:3]:
        h = 1e-4 * a64[i]
        ap, am = a64.copy(), a64.copy()
        ap[i] += h
        am[i] -= h
        fd = (oracle.sinkhorn(Ls, bk, ap, b64, t, it)["W2"]
              - oracle.sinkhorn(Ls, bk, am, b64, t, it)["W2"]) / (2 * h)
        assert ga[i] == pytest.approx(fd, rel=GRTOL, abs=GATOL_REL * np.abs(ga).max())


def test_barycenter_grad_matches_oracle(gs, ctx):
    cfg = W.clusters_barycenter(n=3000, m=8, iters=12)
    X, M = cfg["X"], cfg["M"]
    alpha = np.random.default_rng(2).dirichlet(np.ones(8))
    g = gs.gs_build_graph(ctx, to_dev(X), cfg["k"])
    Ls, _ = oracle.build_graph(X.astype(np.float64), cfg["k"])
    t, K, it = 10.0, 40, 12
    mubar = np.random.default_rng(5).standard_normal(len(X)).astype(np.float32)
    mu, galpha = gs.gs_barycenter_grad(ctx, g, to_dev(M), to_dev(alpha, torch.float64), t, K, it,
                                       to_dev(mubar), checkpoint=5)
    gs.gs_sync(ctx)
    rmu, ralpha = oracle.barycenter_grad(Ls, oracle.cheb_coefficients(t, K), M.astype(np.float64),
                                         alpha, it, mubar.astype(np.float64))
    assert_close(to_np(mu), rmu, 1e-4, 1e-6 * rmu.max(), "mu")
    assert_close(to_np(galpha), ralpha, GRTOL, GATOL_REL * np.abs(ralpha).max(), "dalpha")
    # the checkpoint interval changes what is recomputed, never the values: bit for bit, including
    # one segment (every state taped by the forward pass) and one iteration per segment
    for ck in (1, 12):
        mu2, ga2 = gs.gs_barycenter_grad(ctx, g, to_dev(M), to_dev(alpha, torch.float64), t, K, it,
                                         to_dev(mubar), checkpoint=ck)
        assert torch.equal(mu2, mu) and torch.equal(ga2, galpha), f"checkpoint {ck}"


def test_autograd_distance_to_barycenter(gs, ctx):
    from paper_2211_00805_gb300.autograd import geodesic_barycenter, geodesic_sinkhorn_distance
    cfg = W.manifold_barycenter_grad(n=2500, m=6, bary_iters=10, sink_iters=12)
    X, M, src = cfg["X"], cfg["M"], cfg["src"]
    g = gs.gs_build_graph(ctx, to_dev(X), cfg["k"])
    Ls, _ = oracle.build_graph(X.astype(np.float64), cfg["k"])
    t, K = cfg["t"], cfg["K"]
    alpha = torch.tensor(cfg["alpha"], dtype=torch.float64, device="cuda", requires_grad=True)
    a = to_dev(src).requires_grad_(True)
    # the objective is the unrolled map to the barycenter as it comes out of 10 iterations, whose
    # mass is not exactly the source's: the equal-mass check is switched off for it
    gs.gs_set_option(ctx, gs.GS_OPT_CHECK_ARGS, 0)
    try:
        mu = geodesic_barycenter(ctx, g, to_dev(M), alpha, t, K, cfg["bary_iters"], checkpoint=4)
        J = geodesic_sinkhorn_distance(ctx, g, a, mu, t, K, cfg["sink_iters"], checkpoint=5)
        J.backward()
        gs.gs_sync(ctx)
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_CHECK_ARGS, 1)
    rJ, rgs, rga = oracle.barycenter_distance_grad(Ls, oracle.cheb_coefficients(t, K),
                                                   src.astype(np.float64), M.astype(np.float64),
                                                   cfg["alpha"], t, cfg["bary_iters"], cfg["sink_iters"])
    assert float(J) == pytest.approx(rJ, rel=1e-4)
    assert_close(to_np(a.grad), rgs, GRTOL, GATOL_REL * np.abs(rgs).max(), "dJ/dsrc")
    assert_close(to_np(alpha.grad), rga, GRTOL, GATOL_REL * np.abs(rga).max(), "dJ/dalpha")


# ----------------------------------------------------------------------------------- batched
def test_batched_matches_single_and_oracle(gs, ctx):
    probs = W.ragged_batch(count=10, n_min=600, n_max=6000, iters=40)
    graphs = [gs.gs_build_graph(ctx, to_dev(p.X), p.k) for p in probs]
    a = [to_dev(p.a) for p in probs]
    b = [to_dev(p.b) for p in probs]
    u, v, dist = gs.gs_sinkhorn_batched(ctx, graphs, a, b, [p.t for p in probs], [p.K for p in probs], 40)
    gs.gs_sync(ctx)
    d = to_np(dist)
    # the same call again replays its captured graph (tables kept on the device): same results
    u2, v2 = [torch.empty_like(x) for x in u], [torch.empty_like(x) for x in v]
    dist2 = torch.empty_like(dist)
    for _ in range(2):
        gs.gs_sinkhorn_batched(ctx, graphs, a, b, [p.t for p in probs], [p.K for p in probs], 40, u2, v2, dist2)
    l0 = gs.gs_launch_count(ctx)
    gs.gs_sinkhorn_batched(ctx, graphs, a, b, [p.t for p in probs], [p.K for p in probs], 40, u2, v2, dist2)
    assert gs.gs_launch_count(ctx) - l0 == 3  # argument checks, the persistent kernel, the scatter
    gs.gs_sync(ctx)
    assert torch.allclose(dist2, dist, rtol=0, atol=0, equal_nan=True)  # W is NaN where W^2 < 0
    assert all(torch.equal(x, y) for x, y in zip(u2, u))
    for i, (p, g) in enumerate(zip(probs, graphs)):
        us, vs, ds, _ = gs.gs_sinkhorn(ctx, g, a[i], b[i], p.t, p.K, 40)
        gs.gs_sync(ctx)
        assert d[i, 0] == pytest.approx(to_np(ds)[0], rel=1e-5)
        m = p.a > 0
        assert_close(to_np(u[i]), to_np(us), 1e-4, 0, f"u[{i}]", mask=m)
    for i in (0, 7):
        p = probs[i]
        Ls, _ = oracle.build_graph(p.X.astype(np.float64), p.k)
        r = oracle.sinkhorn(Ls, oracle.cheb_coefficients(p.t, p.K), p.a.astype(np.float64),
                            p.b.astype(np.float64), p.t, 40)
        assert d[i, 0] == pytest.approx(r["W2"], rel=1e-4)


def test_batched_single_order_filter(gs, ctx):
    # K = 1 (the only order is first and last) and mixed K across the batch
    probs = W.ragged_batch(count=3, n_min=500, n_max=1500, iters=20)
    graphs = [gs.gs_build_graph(ctx, to_dev(p.X), p.k) for p in probs]
    Ks = [1, 2, 5]
    ts = [0.5, 1.0, 2.0]
    # broad full-support marginals (one- and two-hop kernels keep the scalings in FP32 range)
    ab = []
    for p in probs:
        a = np.full(len(p.X), 1.0 / len(p.X), np.float32)
        b = (a * (1.0 + 0.3 * np.tanh(p.X[:, 0]))).astype(np.float32)
        ab.append((a, b / b.sum()))
    u, v, dist = gs.gs_sinkhorn_batched(ctx, graphs, [to_dev(a) for a, _ in ab], [to_dev(b) for _, b in ab],
                                         ts, Ks, 20)
    gs.gs_sync(ctx)
    d = to_np(dist)
    for i, (p, g) in enumerate(zip(probs, graphs)):
        Ls, _ = oracle.build_graph(p.X.astype(np.float64), p.k)
        r = oracle.sinkhorn(Ls, oracle.cheb_coefficients(ts[i], Ks[i]), ab[i][0].astype(np.float64),
                            ab[i][1].astype(np.float64), ts[i], 20)
        assert r["status"] == oracle.OK
        assert d[i, 0] == pytest.approx(r["W2"], rel=1e-4)


def test_autotune_choice_is_used_and_exact(gs, ctx, sphere):
    # the autotuner picks an order variant and, for B > 1, the RHS tile width (lanes per row) and,
    # for B = 1, the row-split width; the record serves a rebuilt graph of the same points too
    p, g, Ls = sphere
    g2 = gs.gs_build_graph(ctx, to_dev(p.X), p.k)  # same size: untuned, finds the record
    for B in (1, 32, 64):
        choice = gs.gs_autotune(ctx, g, B, 30)
        assert choice in (1, 2, 3, 4, 5, 6, 7, 8, 9)
        ch = gs.gs_autotune_choices(ctx, g, B, 30)
        assert ch["recorded"] == 1 and ch["kernel"] == choice
        if B == 1:
            assert ch["loop_mode"] in (1, 2) and ch["persist_sync"] in (0, 1, 2, 4)
        else:
            assert ch["lanes"] in (1, 2, 4, 8, 16, 32) and ch["columns_per_pass"] in (4 * ch["lanes"], ch["lanes"])
        assert gs.gs_autotune_choices(ctx, g2, B, 30) == ch
        V = np.random.default_rng(B).random((g.n, B)).astype(np.float32)
        for graph in (g, g2):
            Y = to_np(gs.gs_heat_apply(ctx, graph, 5.0, 30, to_dev(V)))
            ref = oracle.heat_apply(Ls, oracle.cheb_coefficients(5.0, 30), V.astype(np.float64))
            assert_close(Y, ref, 1e-4, 1e-6 * np.abs(ref).max(), f"autotuned B={B}")
    gs.gs_sync(ctx)


@pytest.mark.parametrize("B,lanes", [(32, 4), (64, 8), (64, 16), (12, 1), (128, 16)])
def test_rhs_tile_widths_match_oracle(gs, ctx, sphere, B, lanes):
    # every RHS tile width the autotuner may pick (lanes per row, each lane walking several
    # chunks), through a record for the graph's size: results equal the oracle's
    p, g, Ls = sphere
    V = np.random.default_rng(B + lanes).random((g.n, B)).astype(np.float32)
    gs.gs_autotune(ctx, g, B, 30)
    Y0 = to_np(gs.gs_heat_apply(ctx, g, 5.0, 30, to_dev(V)))
    ref = oracle.heat_apply(Ls, oracle.cheb_coefficients(5.0, 30), V.astype(np.float64))
    assert_close(Y0, ref, 1e-4, 1e-6 * np.abs(ref).max(), f"tuned B={B}")
    gs.gs_set_option(ctx, gs.GS_OPT_BLK_KERNEL, 2)
    try:
        gs.gs_set_option(ctx, gs.GS_OPT_TILE_LANES, lanes)
        Y = to_np(gs.gs_heat_apply(ctx, g, 5.0, 30, to_dev(V)))
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_TILE_LANES, 0)
        gs.gs_set_option(ctx, gs.GS_OPT_BLK_KERNEL, 0)
    assert_close(Y, ref, 1e-4, 1e-6 * np.abs(ref).max(), f"B={B} lanes={lanes}")
    gs.gs_sync(ctx)


def test_differentiation_workload_vs_oracle_finite_differences(gs, ctx):
    # The differentiation workload's objective J(a, alpha) = W^2(a, barycenter(M, alpha)) with its
    # recipe (6-d latent tanh manifold in R^40, k = 10, K = 40, t = 8, 64 inputs, checkpoints every
    # 20) at a size the FP64 oracle can difference: n = 800 points and 100 iterations per loop
    # instead of 500k and 200.  GPU gradient through the autograd adjoint against central
    # differences of the oracle's forward map on 50 random coordinates: 25 of a (step 1e-4 a_i)
    # and 25 of alpha (step 1e-4); perturbed inputs are not renormalised.
    from paper_2211_00805_gb300.autograd import geodesic_barycenter, geodesic_sinkhorn_distance
    its = 100
    cfg = W.manifold_barycenter_grad(n=800, bary_iters=its, sink_iters=its, checkpoint=20)
    X, M, src = cfg["X"], cfg["M"], cfg["src"]
    t, K = cfg["t"], cfg["K"]
    g = gs.gs_build_graph(ctx, to_dev(X), cfg["k"])
    Ls, _ = oracle.build_graph(X.astype(np.float64), cfg["k"])
    bk = oracle.cheb_coefficients(t, K)
    alpha = torch.tensor(cfg["alpha"], dtype=torch.float64, device="cuda", requires_grad=True)
    a = to_dev(src).requires_grad_(True)
    gs.gs_set_option(ctx, gs.GS_OPT_CHECK_ARGS, 0)  # the barycenter's mass is not exactly a's
    try:
        mu = geodesic_barycenter(ctx, g, to_dev(M), alpha, t, K, its, checkpoint=20)
        J = geodesic_sinkhorn_distance(ctx, g, a, mu, t, K, its, checkpoint=20)
        J.backward()
        gs.gs_sync(ctx)
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_CHECK_ARGS, 1)
    ga, gal = to_np(a.grad).astype(np.float64), to_np(alpha.grad)
    M64, a64, al64 = M.astype(np.float64), src.astype(np.float64), np.asarray(cfg["alpha"], np.float64)
    mu0 = oracle.barycenter(Ls, bk, M64, al64, its)
    J0 = oracle.sinkhorn(Ls, bk, a64, mu0, t, its)["W2"]
    assert float(J.detach()) == pytest.approx(J0, rel=1e-4)
    rng = np.random.default_rng(7)
    for i in rng.choice(len(a64), 25, replace=False):
        h = 1e-4 * a64[i]
        ap, am = a64.copy(), a64.copy()
        ap[i] += h
        am[i] -= h
        fd = (oracle.sinkhorn(Ls, bk, ap, mu0, t, its)["W2"] - oracle.sinkhorn(Ls, bk, am, mu0, t, its)["W2"]) / (2 * h)
        assert ga[i] == pytest.approx(fd, rel=GRTOL, abs=GATOL_REL * np.abs(ga).max()), f"dJ/da[{i}]"
    for j in rng.choice(len(al64), 25, replace=False):
        h = 1e-4
        Jpm = []
        for sgn in (1.0, -1.0):
            alj = al64.copy()
            alj[j] += sgn * h
            Jpm.append(oracle.sinkhorn(Ls, bk, a64, oracle.barycenter(Ls, bk, M64, alj, its), t, its)["W2"])
        fd = (Jpm[0] - Jpm[1]) / (2 * h)
        assert gal[j] == pytest.approx(fd, rel=GRTOL, abs=GATOL_REL * np.abs(gal).max()), f"dJ/dalpha[{j}]"
