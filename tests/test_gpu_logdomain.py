"""GPU log-domain Sinkhorn (gs_sinkhorn_log: Algorithm 1 with FP64 potentials and the
extended-range Chebyshev recurrence) against the FP64 oracle's Sinkhorn loop.

Tolerances: the recurrence adds FP32 mantissas (rounding ~6e-8 per operation, K orders of ~k
terms per half-step); the loop does not expand errors in the potentials, so after 200 iterations
they stay within ~1e-4 of the oracle's (the numpy model of the same arithmetic in
test_logdomain_model.py: 1.4e-5 on the case below).  Bounds: 5e-4 absolute on ln u, ln v; 1e-5
relative on W^2, whose constant-shift error cancels between the two equal-mass marginals.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00805_gb300 import workloads as W
from tests.gpu_common import oracle_csr_to_dev, to_dev, to_np

pytestmark = pytest.mark.gpu

LOG_ATOL, W2_RTOL = 5e-4, 1e-5


@pytest.fixture(scope="module")
def gs():
    from paper_2211_00805_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context()


@pytest.fixture(params=[2, 1], ids=["persistent", "per-order"])
def mode(request, gs, ctx):
    # GS_OPT_LOOP 2: the whole loop as one persistent launch where the graph allows it;
    # 1: one launch per Chebyshev order, replayed as a CUDA graph
    gs.gs_set_option(ctx, gs.GS_OPT_LOOP, request.param)
    yield request.param
    gs.gs_set_option(ctx, gs.GS_OPT_LOOP, 2)


@pytest.fixture(scope="module")
def sphere(gs, ctx):
    p = W.sphere_pair()
    g = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    Ls, _ = oracle.build_graph(p.X.astype(np.float64), p.k)
    return p, g, Ls


def _check(gs, ctx, g, Ls, a, b, t, K, iters, vol=None):
    lu, lv, dist, it = gs.gs_sinkhorn_log(ctx, g, to_dev(a), to_dev(b), t, K, iters,
                                          vol=None if vol is None else to_dev(vol))
    gs.gs_sync(ctx)
    r = oracle.sinkhorn(Ls, oracle.cheb_coefficients(t, K), a.astype(np.float64), b.astype(np.float64), t,
                        iters, a=None if vol is None else vol.astype(np.float64))
    assert r["status"] == oracle.OK
    lu, lv, d = to_np(lu), to_np(lv), to_np(dist)
    assert int(to_np(it)[0]) == iters
    for got, ref, marg, name in ((lu, r["v"], a, "ln u"), (lv, r["w"], b, "ln v")):
        zero = marg == 0
        assert np.all(np.isneginf(got[zero])), name  # no mass: u_i = 0
        err = np.abs(got[~zero] - np.log(ref[~zero]))
        assert err.max() < LOG_ATOL, f"{name}: max |error| {err.max():.3g}"
    assert d[0] == pytest.approx(r["W2"], rel=W2_RTOL)
    if r["W2"] >= 0:
        assert d[1] == pytest.approx(r["W"], rel=W2_RTOL)
    else:  # W^2 = 4t (1 + KL) can be negative: no real square root
        assert np.isnan(d[1])
    return lu, lv, d, r


def test_log_sinkhorn_small_t_where_fp32_overflows(gs, ctx, mode, sphere):
    # the 2,000-point sphere pair at t = 1, K = 20, 200 iterations: the scalings reach e^{+-170}
    p, g, Ls = sphere
    lu, lv, d, r = _check(gs, ctx, g, Ls, p.a, p.b, 1.0, 20, 200)
    assert max(np.abs(lu).max(), np.abs(lv).max()) > 150.0  # far outside FP32
    # the FP32 loop cannot represent this case and says so
    gs.gs_sinkhorn(ctx, g, to_dev(p.a), to_dev(p.b), 1.0, 20, 200)
    with pytest.raises(gs.GeosinkError) as e:
        gs.gs_sync(ctx)
    assert e.value.status == gs.GS_ERR_NONFINITE


def test_log_sinkhorn_agrees_with_the_fp32_loop_where_both_fit(gs, ctx, mode, sphere):
    p, g, Ls = sphere
    lu, lv, d, r = _check(gs, ctx, g, Ls, p.a, p.b, 5.0, 30, 200)
    u, v, dist, _ = gs.gs_sinkhorn(ctx, g, to_dev(p.a), to_dev(p.b), 5.0, 30, 200)
    gs.gs_sync(ctx)
    u, v = to_np(u).astype(np.float64), to_np(v).astype(np.float64)
    m = (u > 0) & (np.abs(lu) < 80)
    np.testing.assert_allclose(np.exp(lu[m]), u[m], rtol=1e-3)
    m = (v > 0) & (np.abs(lv) < 80)
    np.testing.assert_allclose(np.exp(lv[m]), v[m], rtol=1e-3)
    assert d[0] == pytest.approx(to_np(dist)[0], rel=1e-4)


def test_log_sinkhorn_vertex_weights_zero_mass_odd_K(gs, ctx, mode, sphere):
    p, g, Ls = sphere
    vol = np.random.default_rng(1).uniform(0.5, 1.5, len(p.a)).astype(np.float32)
    a = np.where(p.X[:, 2] > -0.2, p.a, 0).astype(np.float32)
    a = (a / np.sum(a * vol)).astype(np.float32)
    b = (p.b / np.sum(p.b * vol)).astype(np.float32)
    _check(gs, ctx, g, Ls, a, b, 1.0, 21, 100, vol=vol)


@pytest.mark.parametrize("t,K", [(2.0, 1), (3.0, 2), (0.5, 3), (0.5, 12)])
def test_log_sinkhorn_low_degrees(gs, ctx, mode, sphere, t, K):
    # p_K reaches K hops only, so pole-to-pole marginals have no plan for K below the graph's
    # diameter (the FP64 oracle's scalings diverge too); b = a times a random +-30% factor needs
    # only local moves
    p, g, Ls = sphere
    b = p.a * (1 + 0.3 * np.random.default_rng(5).uniform(-1, 1, len(p.a)))
    b = (b / b.sum()).astype(np.float32)
    _check(gs, ctx, g, Ls, p.a, b, t, K, 60)


def test_log_sinkhorn_tiny_graph_one_block_plus_a_row(gs, ctx, mode):
    # 33 rows: one full block of 32 lane groups and a ragged tail of one row
    p = W.sphere_pair(n=33)
    idx, dist = oracle.knn(p.X.astype(np.float64), 6)
    rp, col, A = oracle.affinity_graph(idx, dist, oracle.median_sigma(dist))
    g = gs.gs_graph_from_csr(ctx, *oracle_csr_to_dev(rp, col, A))
    A32 = np.asarray(A, np.float32).astype(np.float64)  # the affinities the GPU holds
    Ls = oracle.shifted(oracle.laplacian(rp, col, A32)[1])
    _check(gs, ctx, g, Ls, p.a, p.b, 1.0, 20, 50)


def test_log_sinkhorn_repeats_bit_for_bit(gs, ctx, mode, sphere):
    p, g, Ls = sphere
    a, b = to_dev(p.a), to_dev(p.b)
    r1 = [to_np(x) for x in gs.gs_sinkhorn_log(ctx, g, a, b, 1.0, 20, 40)]
    r2 = [to_np(x) for x in gs.gs_sinkhorn_log(ctx, g, a, b, 1.0, 20, 40)]
    gs.gs_sync(ctx)
    for x, y in zip(r1, r2):
        assert np.array_equal(x, y)


def test_log_sinkhorn_persistent_and_per_order_forms_agree(gs, ctx, sphere):
    # the persistent loop sums each row by one thread in the sliced-ELL entry order and exchanges
    # mantissas with a parity bit in their last place; the per-order launches sum by four lanes:
    # the same iteration to FP32 rounding
    p, g, Ls = sphere
    a, b = to_dev(p.a), to_dev(p.b)
    out = {}
    for m in (2, 1):
        gs.gs_set_option(ctx, gs.GS_OPT_LOOP, m)
        out[m] = [to_np(x) for x in gs.gs_sinkhorn_log(ctx, g, a, b, 1.0, 20, 100)]
    gs.gs_set_option(ctx, gs.GS_OPT_LOOP, 2)
    gs.gs_sync(ctx)
    for x, y in zip(out[2][:2], out[1][:2]):
        fin = np.isfinite(y)
        assert np.array_equal(np.isfinite(x), fin)
        assert np.abs(x[fin] - y[fin]).max() < 2e-4
    assert out[2][2][0] == pytest.approx(out[1][2][0], rel=1e-6)


def test_log_sinkhorn_two_rows_per_thread_at_scale(gs, ctx):
    # 160k points: more rows per partition block than threads (two rows per thread in the
    # persistent form); against the per-order form and the FP32 loop (t = 5, where both fit)
    # (a broad bump and a local tilt of it: K = 30 hops cover the transport on this large sphere)
    p = W.sphere_pair(n=160_000, t=5.0, K=30)
    g = gs.gs_build_graph(ctx, to_dev(p.X), p.k)
    assert gs.gs_graph_layout(g)["rows_per_block"] > 1024
    a0 = W.vmf_bump(p.X, np.array([0.0, 0.0, 1.0]), 1.0)
    b0 = a0 * (1.0 + 0.3 * np.tanh(p.X[:, 0]))
    a, b = to_dev(a0), to_dev((b0 / b0.sum()).astype(np.float32))
    out = {}
    for m in (2, 1):
        gs.gs_set_option(ctx, gs.GS_OPT_LOOP, m)
        out[m] = [to_np(x) for x in gs.gs_sinkhorn_log(ctx, g, a, b, 5.0, 30, 30)]
    gs.gs_set_option(ctx, gs.GS_OPT_LOOP, 2)
    u, v, dist, _ = gs.gs_sinkhorn(ctx, g, a, b, 5.0, 30, 30)
    gs.gs_sync(ctx)
    for x, y in zip(out[2][:2], out[1][:2]):
        fin = np.isfinite(y)
        assert np.array_equal(np.isfinite(x), fin)
        assert np.abs(x[fin] - y[fin]).max() < 2e-4
    lu, uu = out[2][0], to_np(u).astype(np.float64)
    msk = (uu > 0) & (np.abs(lu) < 80)
    np.testing.assert_allclose(np.exp(lu[msk]), uu[msk], rtol=1e-3)
    assert out[2][2][0] == pytest.approx(float(to_np(dist)[0]), rel=1e-4)


def test_log_sinkhorn_bounded_wait_timeout_is_reported_and_context_survives(gs, ctx, sphere):
    # the self-test makes every staging wait of the persistent log-domain loop look for a parity no
    # exchanged word carries: the waits run out, gs_sync reports the timeout, the next call works
    p, g, Ls = sphere
    gs.gs_set_option(ctx, gs.GS_OPT_BARRIER_SELFTEST, 1)
    gs.gs_sinkhorn_log(ctx, g, to_dev(p.a), to_dev(p.b), 5.0, 30, 5)
    with pytest.raises(gs.GeosinkError) as e:
        gs.gs_sync(ctx)
    assert e.value.status == gs.GS_ERR_TIMEOUT
    assert gs.gs_get_option(ctx, gs.GS_OPT_BARRIER_SELFTEST) == 0
    _check(gs, ctx, g, Ls, p.a, p.b, 5.0, 30, 40)


def test_log_sinkhorn_rejects_bad_arguments(gs, ctx, sphere):
    p, g, Ls = sphere
    n = len(p.a)
    lib = gs.lib()
    a, b = to_dev(p.a), to_dev(p.b)
    lu = torch.empty(n, dtype=torch.float64, device="cuda")
    lv = torch.empty(n, dtype=torch.float64, device="cuda")
    # ctx, g, a, b, vol, t, K, eps, iters, log_u, log_v, dist, iters_done
    args = [ctx.handle, g.handle, a.data_ptr(), b.data_ptr(), None, 1.0, 20, 0.0, 10, lu.data_ptr(), lv.data_ptr(),
            None, None]
    assert lib.gs_sinkhorn_log(*args[:9], lu.data_ptr(), lu.data_ptr(), None, None) == gs.GS_ERR_ARG
    assert lib.gs_sinkhorn_log(*args[:8], 0, *args[9:]) == gs.GS_ERR_ARG  # iters
    assert lib.gs_sinkhorn_log(*args[:7], float("nan"), *args[8:]) == gs.GS_ERR_ARG  # eps
    assert lib.gs_sinkhorn_log(*args[:6], 0, *args[7:]) == gs.GS_ERR_ARG  # K
    assert lib.gs_sinkhorn_log(*args[:5], -1.0, *args[6:]) == gs.GS_ERR_ARG  # t
    assert lib.gs_sinkhorn_log(*args[:2], None, *args[3:]) == gs.GS_ERR_ARG  # a
    gs.gs_sync(ctx)  # the context stays usable


def _oracle_marginal_errors(Ls, t, K, a, b, upto):
    """sum_i |u_i p_K(w)_i - a_i| after iterations 10, 20, ..., upto (the eps stop's measure)."""
    c = oracle.cheb_coefficients(t, K)
    w = np.ones(len(a))
    errs = []
    for j in range(1, upto + 1):
        u = oracle._div0(a, oracle.heat_apply(Ls, c, w))
        w = oracle._div0(b, oracle.heat_apply(Ls, c, u))
        if j % 10 == 0:
            errs.append(np.abs(u * oracle.heat_apply(Ls, c, w) - a).sum())
    return errs


def test_log_sinkhorn_eps_stop_matches_oracle(gs, ctx, sphere):
    # t = 1 (FP32 scalings overflow): eps between the oracle's marginal errors after 30 and 40
    # iterations, so the oracle and the GPU both stop after iteration 40, whether the stop is
    # found at the start of iteration 41 or by the check after the last iteration
    p, g, Ls = sphere
    t, K = 1.0, 20
    a64, b64 = p.a.astype(np.float64), p.b.astype(np.float64)
    e30, e40 = _oracle_marginal_errors(Ls, t, K, a64, b64, 40)[2:4]
    assert e40 < 0.99 * e30  # a clear gap: the GPU's errors are within ~1e-3 of these
    eps = float(np.sqrt(e30 * e40))
    r = oracle.sinkhorn(Ls, oracle.cheb_coefficients(t, K), a64, b64, t, 60, eps=eps)
    assert r["status"] == oracle.OK and r["iters"] == 40
    a, b = to_dev(p.a), to_dev(p.b)
    res = {}
    for iters in (60, 40):
        lu, lv, dist, it = gs.gs_sinkhorn_log(ctx, g, a, b, t, K, iters, eps=eps)
        gs.gs_sync(ctx)
        assert int(to_np(it)[0]) == 40
        res[iters] = (to_np(lu), to_np(lv), to_np(dist))
        for got, ref in ((res[iters][0], r["v"]), (res[iters][1], r["w"])):
            err = np.abs(got - np.log(ref))
            assert err.max() < LOG_ATOL
        assert res[iters][2][0] == pytest.approx(r["W2"], rel=W2_RTOL)
    for x, y in zip(res[60], res[40]):  # the same 40 iterations either way
        assert np.array_equal(x, y)


def test_log_sinkhorn_eps_not_reached_is_reported(gs, ctx, sphere):
    p, g, Ls = sphere
    lu, lv, dist, it = gs.gs_sinkhorn_log(ctx, g, to_dev(p.a), to_dev(p.b), 1.0, 20, 20, eps=1e-30)
    with pytest.raises(gs.GeosinkError) as e:
        gs.gs_sync(ctx)
    assert e.value.status == gs.GS_ERR_NOT_CONVERGED
    assert int(to_np(it)[0]) == 20
    _, _, _, r = _check(gs, ctx, g, Ls, p.a, p.b, 1.0, 20, 20)  # the oracle's 20 iterations
    for got, ref in ((to_np(lu), r["v"]), (to_np(lv), r["w"])):
        assert np.abs(got - np.log(ref)).max() < LOG_ATOL
