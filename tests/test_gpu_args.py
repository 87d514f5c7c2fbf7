"""Device-side argument checks of the C ABI (raised as GS_ERR_ARG by gs_sync).

Algorithm 1 needs marginals that are non-negative and carry the same mass with respect to the
vertex weights, sum(vol a) = sum(vol b) (tolerance 1e-6 relative); the barycenter of Sec. 3.3
needs weights alpha >= 0 with sum 1 (tolerance 1e-6).  Each check is triggered here once, and
the option GS_OPT_CHECK_ARGS = 0 switches them off.
"""
import numpy as np
import pytest
import torch

from paper_2211_00805_gb300 import workloads as W
from tests.gpu_common import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    from paper_2211_00805_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def setup(gs):
    ctx = gs.Context()
    p = W.sphere_pair(n=800, t=5.0, K=30)
    g = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    return ctx, g, p


def _expect_arg(gs, ctx):
    with pytest.raises(gs.GeosinkError) as e:
        gs.gs_sync(ctx)
    assert e.value.status == gs.GS_ERR_ARG


def _bad_marginals(p):
    neg = p.a.copy()
    neg[3] = -neg[3]  # a negative entry (mass moved so that the sums still agree)
    neg[4] += 2 * p.a[3]
    heavy = (p.b * (1 + 1e-4)).astype(np.float32)  # masses 1e-4 apart
    return [(neg, p.b), (p.a, heavy)]


def test_sinkhorn_family_rejects_bad_marginals(gs, setup):
    ctx, g, p = setup
    for a, b in _bad_marginals(p):
        A, Bm = to_dev(a), to_dev(b)
        gs.gs_sinkhorn(ctx, g, A, Bm, 5.0, 30, 5)
        _expect_arg(gs, ctx)
        gs.gs_distance(ctx, g, A, Bm, 5.0, 30, 5)
        _expect_arg(gs, ctx)
        gs.gs_sinkhorn_log(ctx, g, A, Bm, 5.0, 30, 2)
        _expect_arg(gs, ctx)
        gs.gs_sinkhorn_grad(ctx, g, A, Bm, 5.0, 30, 4, checkpoint=2)
        _expect_arg(gs, ctx)
        gs.gs_sinkhorn_batched(ctx, [g, g], [to_dev(p.a), A], [to_dev(p.b), Bm], [5.0, 5.0], [30, 30], 5)
        _expect_arg(gs, ctx)
    # balanced marginals pass, and so do equal masses with respect to vertex weights
    gs.gs_sinkhorn(ctx, g, to_dev(p.a), to_dev(p.b), 5.0, 30, 5)
    gs.gs_sync(ctx)
    vol = np.random.default_rng(2).uniform(0.5, 1.5, len(p.a)).astype(np.float32)
    a = (p.a / np.sum(p.a * vol)).astype(np.float32)
    b = (p.b / np.sum(p.b * vol)).astype(np.float32)
    gs.gs_sinkhorn(ctx, g, to_dev(a), to_dev(b), 5.0, 30, 5, vol=to_dev(vol))
    gs.gs_sync(ctx)
    # ... but plain-normalised marginals under uneven vertex weights do not
    gs.gs_sinkhorn(ctx, g, to_dev(p.a), to_dev(p.b), 5.0, 30, 5, vol=to_dev(vol))
    _expect_arg(gs, ctx)


def test_barycenter_family_rejects_bad_weights(gs, setup):
    ctx, g, p = setup
    M = to_dev(np.stack([p.a, p.b], 1))
    mubar = to_dev(np.ones(len(p.a), np.float32))
    for alpha in ([0.7, 0.4], [1.2, -0.2], [0.5, 0.5 - 1e-4]):
        al = to_dev(np.array(alpha), torch.float64)
        gs.gs_barycenter(ctx, g, M, al, 5.0, 30, 3)
        _expect_arg(gs, ctx)
        gs.gs_barycenter_grad(ctx, g, M, al, 5.0, 30, 3, mubar, checkpoint=1)
        _expect_arg(gs, ctx)
        good = to_dev(np.array([0.5, 0.5]), torch.float64)
        gs.gs_barycentric_distance(ctx, g, M, al, M, good, 5.0, 30, 3, 3)
        _expect_arg(gs, ctx)
    gs.gs_barycenter(ctx, g, M, to_dev(np.array([0.25, 0.75]), torch.float64), 5.0, 30, 3)
    gs.gs_sync(ctx)


def test_checks_can_be_switched_off(gs, setup):
    ctx, g, p = setup
    a, b = _bad_marginals(p)[1]
    gs.gs_set_option(ctx, gs.GS_OPT_CHECK_ARGS, 0)
    try:
        assert gs.gs_get_option(ctx, gs.GS_OPT_CHECK_ARGS) == 0
        gs.gs_sinkhorn(ctx, g, to_dev(a), to_dev(b), 5.0, 30, 5)
        gs.gs_sync(ctx)
    finally:
        gs.gs_set_option(ctx, gs.GS_OPT_CHECK_ARGS, 1)
    gs.gs_sinkhorn(ctx, g, to_dev(a), to_dev(b), 5.0, 30, 5)
    _expect_arg(gs, ctx)
