"""GPU families of distributions (gs_barycentric_distance, Definition 4.3; gs_barycenter_effect,
Definition 4.4) against the FP64 oracle, and the expected-barycenter-effect experiment of Table 2.

Tolerances: the barycenters and the distance inherit the FP32 filter's ~1e-4 relative error (as
the barycenter and Sinkhorn parity tests); the effect kernel itself sums FP32 inputs in FP64, so
on identical measures it agrees with the oracle to ~1e-12.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2211_00805_gb300 import workloads as W
from tests.gpu_common import assert_close, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    from paper_2211_00805_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context()


@pytest.fixture(scope="module")
def sphere(gs, ctx):
    p = W.sphere_pair(n=2000)
    g = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    Ls, _ = oracle.build_graph(p.X.astype(np.float64), p.k)
    return p, g, Ls


def _families(X):
    rng = np.random.default_rng(12)
    north, south = np.array([0.0, 0.0, 1.0]), np.array([0.3, 0.0, -1.0])
    def bumps(c, m):
        cs = [c + 0.4 * rng.standard_normal(3) for _ in range(m)]
        return np.stack([W.vmf_bump(X, x / np.linalg.norm(x), 4.0) for x in cs], 1).astype(np.float32)
    MT, MC = bumps(north, 3), bumps(south, 4)
    aT = rng.dirichlet(np.ones(3))
    aC = rng.dirichlet(np.ones(4))
    return MT, aT, MC, aC


def test_barycentric_distance_matches_oracle(gs, ctx, sphere):
    p, g, Ls = sphere
    MT, aT, MC, aC = _families(p.X)
    t, K, bi, si = 5.0, 30, 20, 200
    dist, muT, muC = gs.gs_barycentric_distance(ctx, g, to_dev(MT), to_dev(aT, torch.float64), to_dev(MC),
                                                to_dev(aC, torch.float64), t, K, bi, si)
    gs.gs_sync(ctx)
    ref = oracle.barycentric_distance(Ls, oracle.cheb_coefficients(t, K), MT.astype(np.float64), aT,
                                      MC.astype(np.float64), aC, t, bi, si)
    assert ref["status"] == oracle.OK
    assert_close(to_np(muT), ref["muT"], 1e-4, 1e-6 * ref["muT"].max(), "muT")
    assert_close(to_np(muC), ref["muC"], 1e-4, 1e-6 * ref["muC"].max(), "muC")
    assert to_np(muT).sum() == pytest.approx(1.0, rel=1e-5)
    d = to_np(dist)
    assert d[0] == pytest.approx(ref["W2"], rel=1e-4)
    assert d[1] == pytest.approx(ref["W"], rel=1e-4)
    # the effect of Definition 4.4 on the sphere coordinates, same measures: FP64 sums only
    tau = to_np(gs.gs_barycenter_effect(ctx, to_dev(p.X), muT, muC))
    gs.gs_sync(ctx)
    np.testing.assert_allclose(tau, oracle.barycenter_effect(p.X, to_np(muT), to_np(muC)), rtol=1e-10,
                               atol=1e-12)
    # against the oracle's barycenters: the filter's error
    np.testing.assert_allclose(tau, oracle.barycenter_effect(p.X, ref["muT"], ref["muC"]), rtol=1e-3,
                               atol=1e-4)


def test_barycenter_effect_kernel_and_arguments(gs, ctx):
    rng = np.random.default_rng(3)
    n, d = 5003, 7
    Y = rng.standard_normal((n, d)).astype(np.float32)
    muT, muC = rng.random(n).astype(np.float32), (3.0 * rng.random(n)).astype(np.float32)
    tau = to_np(gs.gs_barycenter_effect(ctx, to_dev(Y), to_dev(muT), to_dev(muC)))
    gs.gs_sync(ctx)
    np.testing.assert_allclose(tau, oracle.barycenter_effect(Y, muT, muC), rtol=1e-10, atol=1e-13)
    # a measure without mass is reported at the next synchronisation
    gs.gs_barycenter_effect(ctx, to_dev(Y), to_dev(np.zeros(n, np.float32)), to_dev(muC))
    with pytest.raises(gs.GeosinkError) as e:
        gs.gs_sync(ctx)
    assert e.value.status == gs.GS_ERR_NONFINITE


def test_barycentric_distance_rejects_bad_arguments(gs, ctx, sphere):
    p, g, Ls = sphere
    MT, aT, MC, aC = _families(p.X)
    n = len(p.X)
    mu = torch.empty(n, dtype=torch.float32, device="cuda")
    dist = torch.empty(2, dtype=torch.float64, device="cuda")
    lib = gs.lib()
    args = [ctx.handle, g.handle, to_dev(MT).data_ptr(), 3, to_dev(aT, torch.float64).data_ptr(),
            to_dev(MC).data_ptr(), 4, to_dev(aC, torch.float64).data_ptr(), None, 5.0, 30, 10, 10,
            mu.data_ptr(), mu.data_ptr(), dist.data_ptr()]
    assert lib.gs_barycentric_distance(*args) == gs.GS_ERR_ARG  # muT and muC the same buffer
    args[14] = torch.empty(n, dtype=torch.float32, device="cuda").data_ptr()
    args[3] = 0
    assert lib.gs_barycentric_distance(*args) == gs.GS_ERR_ARG  # empty family


def _golden_table2():
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_expected_barycenter_effect.txt")
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            name, m, s, _, _ = line.split()
            rows[name] = (float(m), float(s))
    return rows


@pytest.mark.parametrize("outlier,row", [(None, "none"), (0.0, "0")])
def test_expected_barycenter_effect_table2_on_gpu(gs, ctx, outlier, row):
    # Table 2's experiment through the library: the barycentric pair, then the effect on the shifted
    # coordinate; against the oracle on the same inputs and against the printed value
    mean, std = _golden_table2()[row]
    X, MC, MT = W.treatment_families(outlier, seed=0)
    g = gs.gs_build_graph(ctx, to_dev(X), 10)
    alpha = to_dev(np.full(10, 0.1), torch.float64)
    dist, muT, muC = gs.gs_barycentric_distance(ctx, g, to_dev(MT), alpha, to_dev(MC), alpha, 5.0, 30, 50, 100)
    tau = to_np(gs.gs_barycenter_effect(ctx, to_dev(np.ascontiguousarray(X[:, :1])), muT, muC))[0]
    gs.gs_sync(ctx)
    Ls, _ = oracle.build_graph(X.astype(np.float64), 10)
    b = oracle.cheb_coefficients(5.0, 30)
    ref = oracle.barycenter_effect(X[:, :1], oracle.barycenter(Ls, b, MT, np.full(10, 0.1), 50),
                                   oracle.barycenter(Ls, b, MC, np.full(10, 0.1), 50))[0]
    assert tau == pytest.approx(ref, rel=2e-3)
    assert abs(tau - mean) < 3 * std
    assert np.isfinite(to_np(dist)[0])


# ------------------------------------------------------------- Euler implicit kernel (Sec. 4)
@pytest.mark.parametrize("B,t,K", [(1, 5.0, 30), (3, 2.0, 8), (32, 10.0, 40)])
def test_heat_apply_implicit_matches_oracle(gs, ctx, sphere, B, t, K):
    p, g, Ls = sphere
    V = np.random.default_rng(B).random((len(p.X), B)).astype(np.float32)
    Y = to_np(gs.gs_heat_apply_implicit(ctx, g, t, K, to_dev(V), tol=1e-7, iters=40))
    gs.gs_sync(ctx)
    ref = oracle.heat_apply_implicit(Ls, t, K, V.astype(np.float64))
    assert_close(Y, ref, 1e-4, 1e-6 * np.abs(ref).max(), f"implicit B={B}")
    Y2 = to_np(gs.gs_heat_apply_implicit(ctx, g, t, K, to_dev(V), tol=1e-7, iters=40))
    gs.gs_sync(ctx)
    assert np.array_equal(Y, Y2)  # fixed-order reductions: repeatable bit for bit
