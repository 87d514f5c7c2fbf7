"""Pins for the oracle's Sinkhorn loop (Algorithm 1), distance (Definition 4.1 / eq. 4),
barycenter (Sec. 3.3) and reverse modes, against definitions and invariants (CPU only)."""
import math

import numpy as np
import pytest

import oracle
from paper_2211_00805_gb300 import workloads as W
from tests.oracle_helpers import dense_knn_laplacian, heat_expm


@pytest.fixture(scope="module")
def sphere_small():
    X = W.sphere(240, seed=3).astype(np.float64)
    Ls, ex = oracle.build_graph(X, 8)
    Ld, *_ = dense_knn_laplacian(X, 8)
    ez = np.array([0.0, 0.0, 1.0])
    mu = W.vmf_bump(X, ez, 4.0).astype(np.float64)
    nu = W.vmf_bump(X, -ez, 4.0).astype(np.float64)
    return X, Ls, Ld, mu / mu.sum(), nu / nu.sum()


def _dense_filter(Ls, b, n):
    return oracle.heat_apply(Ls, b, np.eye(n))


def test_sinkhorn_marginals_at_convergence(sphere_small):
    X, Ls, Ld, mu, nu = sphere_small
    t, K = 2.0, 30
    b = oracle.cheb_coefficients(t, K)
    r = oracle.sinkhorn(Ls, b, mu, nu, t, 400)
    Hd = _dense_filter(Ls, b, len(X))
    v, w = r["v"], r["w"]
    pi = v[:, None] * Hd * w[None, :]
    assert np.max(np.abs(pi.sum(1) - mu)) < 1e-10
    assert np.max(np.abs(pi.sum(0) - nu)) < 1e-14
    assert r["status"] == oracle.OK and r["iters"] == 400


def test_distance_primal_equals_dual(sphere_small):
    # Algorithm 1 returns 4t sum(mu ln v + nu ln w); eq. (4) / Definition 4.1 state the same
    # quantity as 4t (1 + KL(pi | H_t)) for the optimal plan pi = diag(v) H diag(w).
    X, Ls, Ld, mu, nu = sphere_small
    t, K = 2.0, 30
    b = oracle.cheb_coefficients(t, K)
    r = oracle.sinkhorn(Ls, b, mu, nu, t, 400)
    Hd = _dense_filter(Ls, b, len(X))
    pi = r["v"][:, None] * Hd * r["w"][None, :]
    nz = pi > 0
    kl = np.sum(pi[nz] * (np.log(pi[nz] / Hd[nz]) - 1.0))
    assert r["W2"] == pytest.approx(4 * t * (1 + kl), rel=1e-9)
    assert r["W"] == pytest.approx(math.sqrt(r["W2"]), rel=1e-15)


def test_sinkhorn_matches_exact_heat_kernel(sphere_small):
    # the same alternating scaling with the exact kernel exp(-tL): the Chebyshev truncation error
    # (below 1e-20 here) must not show
    X, Ls, Ld, mu, nu = sphere_small
    t, K = 2.0, 30
    r = oracle.sinkhorn(Ls, oracle.cheb_coefficients(t, K), mu, nu, t, 300)
    H = heat_expm(Ld, t)
    w = np.ones(len(X))
    for _ in range(300):
        v = mu / (H @ w)
        w = nu / (H @ v)
    W2 = 4 * t * np.sum(mu * np.log(v) + nu * np.log(w))
    assert r["W2"] == pytest.approx(W2, rel=1e-10)
    np.testing.assert_allclose(r["v"], v, rtol=1e-9)


def test_sinkhorn_vertex_weights_marginals(sphere_small):
    X, Ls, Ld, mu, nu = sphere_small
    n = len(X)
    a = np.random.default_rng(9).uniform(0.5, 1.5, n)
    mu_a, nu_a = mu / np.sum(a * mu), nu / np.sum(a * nu)  # densities w.r.t. the weights a
    t, K = 2.0, 30
    b = oracle.cheb_coefficients(t, K)
    r = oracle.sinkhorn(Ls, b, mu_a, nu_a, t, 400, a=a)
    Hd = _dense_filter(Ls, b, n)
    pi = r["v"][:, None] * Hd * r["w"][None, :]
    # marginals measured against the vertex weights: sum_j pi_ij a_j = mu_i, sum_i a_i pi_ij = nu_j
    assert np.max(np.abs(pi @ a - mu_a)) < 1e-9
    assert np.max(np.abs(a @ pi - nu_a)) < 1e-12
    kl = np.sum((a[:, None] * a[None, :] * pi)[pi > 0] * (np.log(pi[pi > 0] / Hd[pi > 0]) - 1))
    assert r["W2"] == pytest.approx(4 * t * (1 + kl), rel=1e-9)


def test_sinkhorn_zero_mass(sphere_small):
    X, Ls, Ld, mu, nu = sphere_small
    mu0 = np.where(X[:, 2] > 0.2, mu, 0.0)
    mu0 /= mu0.sum()
    r = oracle.sinkhorn(Ls, oracle.cheb_coefficients(2.0, 30), mu0, nu, 2.0, 200)
    assert r["status"] == oracle.OK and np.isfinite(r["W2"])
    assert np.all(r["v"][mu0 == 0] == 0) and np.all(r["v"][mu0 > 0] > 0)


def test_sinkhorn_eps_stop(sphere_small):
    X, Ls, Ld, mu, nu = sphere_small
    b = oracle.cheb_coefficients(2.0, 30)
    r = oracle.sinkhorn(Ls, b, mu, nu, 2.0, 1000, eps=1e-9)
    assert r["status"] == oracle.OK and r["iters"] % 10 == 0 and r["iters"] < 1000
    err = np.abs(r["v"] * oracle.heat_apply(Ls, b, r["w"]) - mu).sum()
    assert err < 1e-9
    r2 = oracle.sinkhorn(Ls, b, mu, nu, 2.0, 20, eps=1e-30)
    assert r2["status"] == oracle.NOT_CONVERGED and r2["iters"] == 20


# ------------------------------------------------------------------------------- barycenter
@pytest.fixture(scope="module")
def bary_setup():
    rng = np.random.default_rng(31)
    X = W.sphere(200, seed=5).astype(np.float64)
    Ls, ex = oracle.build_graph(X, 8)
    Ld, *_ = dense_knn_laplacian(X, 8)
    cs = rng.standard_normal((3, 3))
    M = np.stack([W.vmf_bump(X, c / np.linalg.norm(c), 6.0) for c in cs], 1).astype(np.float64)
    M /= M.sum(0)
    return X, Ls, Ld, M


def test_barycenter_one_hot_weights_closed_form(bary_setup):
    # alpha = e_j leaves v_j = 1, so mu* = H(mu_j / H(1)) after any number of iterations
    X, Ls, Ld, M = bary_setup
    t, K = 2.0, 30
    H = heat_expm(Ld, t)
    for j in range(3):
        alpha = np.eye(3)[j]
        mu = oracle.barycenter(Ls, oracle.cheb_coefficients(t, K), M, alpha, 7)
        ref = H @ (M[:, j] / (H @ np.ones(len(X))))
        np.testing.assert_allclose(mu, ref, rtol=1e-10)


def test_barycenter_identical_inputs(bary_setup):
    X, Ls, Ld, M = bary_setup
    t, K = 2.0, 30
    H = heat_expm(Ld, t)
    Mi = np.repeat(M[:, :1], 3, axis=1)
    mu = oracle.barycenter(Ls, oracle.cheb_coefficients(t, K), Mi, np.array([0.2, 0.3, 0.5]), 5)
    np.testing.assert_allclose(mu, H @ (M[:, 0] / (H @ np.ones(len(X)))), rtol=1e-10)


def test_barycenter_log_scaling_invariant(bary_setup):
    # v_i <- v_i mu / d_i with mu = prod d_i^alpha_i keeps sum_i alpha_i ln v_i = 0 (start v_i = 1)
    X, Ls, Ld, M = bary_setup
    alpha = np.array([0.5, 0.3, 0.2])
    for iters in (1, 4, 9):
        mu, Vs = oracle.barycenter(Ls, oracle.cheb_coefficients(2.0, 30), M, alpha, iters,
                                   return_state=True)
        assert np.max(np.abs(np.log(Vs) @ alpha)) < 1e-12


def test_barycenter_fixed_point_marginals(bary_setup):
    # at convergence every plan pi_i = diag(w_i) H diag(v_i) has marginals mu_i and mu*
    X, Ls, Ld, M = bary_setup
    t, K = 2.0, 30
    b = oracle.cheb_coefficients(t, K)
    alpha = np.array([0.5, 0.3, 0.2])
    mu, Vs = oracle.barycenter(Ls, b, M, alpha, 600, return_state=True)
    H = lambda x: oracle.heat_apply(Ls, b, x)  # noqa: E731
    Ws = M / H(Vs)
    assert np.max(np.abs(Ws * H(Vs) - M)) < 1e-15
    assert np.max(np.abs(Vs * H(Ws) - mu[:, None])) < 1e-8 * mu.max()


def test_barycenter_fixed_point_marginals_with_vertex_weights(bary_setup):
    # with vertex weights a the inputs are densities of equal weighted mass sum(a mu_i); at
    # convergence w_i (H(a v_i)) = mu_i and v_i (H(a w_i)) = mu* for every i, with a inside both
    # filter inputs, and mu* keeps that weighted mass
    X, Ls, Ld, M = bary_setup
    t, K = 2.0, 30
    b = oracle.cheb_coefficients(t, K)
    a = np.random.default_rng(12).uniform(0.7, 1.3, len(X))
    Mw = M / (a @ M)
    alpha = np.array([0.5, 0.3, 0.2])
    mu, Vs = oracle.barycenter(Ls, b, Mw, alpha, 600, a=a, return_state=True)
    H = lambda x: oracle.heat_apply(Ls, b, x)  # noqa: E731
    Ws = Mw / H(a[:, None] * Vs)
    assert np.max(np.abs(Ws * H(a[:, None] * Vs) - Mw)) < 1e-14 * Mw.max()
    assert np.max(np.abs(Vs * H(a[:, None] * Ws) - mu[:, None])) < 1e-8 * mu.max()
    assert a @ mu == pytest.approx(1.0, rel=1e-10)
    # and the weights matter: the unweighted fixed point of the same columns is another measure
    mu1 = oracle.barycenter(Ls, b, Mw, alpha, 600)
    assert np.max(np.abs(mu1 - mu)) > 1e-3 * mu.max()


# ------------------------------------------------------------------------------ reverse mode
def _central_fd(f, x, i, h):
    xp, xm = x.copy(), x.copy()
    xp[i] += h
    xm[i] -= h
    return (f(xp) - f(xm)) / (2 * h)


def test_sinkhorn_grad_matches_finite_differences(sphere_small):
    X, Ls, Ld, mu, nu = sphere_small
    t, K, it = 2.0, 20, 30
    b = oracle.cheb_coefficients(t, K)
    a = np.random.default_rng(4).uniform(0.8, 1.2, len(X))
    W2, gmu, gnu = oracle.sinkhorn_grad(Ls, b, mu, nu, t, it, a=a)
    assert W2 == pytest.approx(oracle.sinkhorn(Ls, b, mu, nu, t, it, a=a)["W2"], rel=1e-14)
    rng = np.random.default_rng(8)
    for i in rng.choice(len(X), 6, replace=False):
        h = 1e-4 * mu[i]
        fd = _central_fd(lambda m: oracle.sinkhorn(Ls, b, m, nu, t, it, a=a)["W2"], mu, i, h)
        assert gmu[i] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(gmu).max())
        h = 1e-4 * nu[i]
        fd = _central_fd(lambda m: oracle.sinkhorn(Ls, b, mu, m, t, it, a=a)["W2"], nu, i, h)
        assert gnu[i] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(gnu).max())


def test_sinkhorn_grad_envelope_at_convergence(sphere_small):
    # at the optimum, tangential derivatives of the dual value are the potentials 4t ln v
    X, Ls, Ld, mu, nu = sphere_small
    t = 2.0
    b = oracle.cheb_coefficients(t, 30)
    W2, gmu, _ = oracle.sinkhorn_grad(Ls, b, mu, nu, t, 300)
    r = oracle.sinkhorn(Ls, b, mu, nu, t, 300)
    pot = 4 * t * np.log(r["v"])
    np.testing.assert_allclose(gmu - gmu.mean(), pot - pot.mean(), atol=1e-6 * np.abs(pot).max())


def test_barycenter_grad_matches_finite_differences(bary_setup):
    X, Ls, Ld, M = bary_setup
    t, K = 2.0, 20
    b = oracle.cheb_coefficients(t, K)
    alpha = np.array([0.5, 0.3, 0.2])
    src = W.vmf_bump(X, np.array([1.0, 0, 0]), 3.0).astype(np.float64)
    src /= src.sum()
    J, gsrc, galpha = oracle.barycenter_distance_grad(Ls, b, src, M, alpha, t, 12, 15)

    def J_of(al, s=src):
        mu = oracle.barycenter(Ls, b, M, al, 12)
        return oracle.sinkhorn(Ls, b, s, mu, t, 15)["W2"]

    assert J == pytest.approx(J_of(alpha), rel=1e-13)
    for i in range(3):
        fd = _central_fd(J_of, alpha, i, 1e-5)
        assert galpha[i] == pytest.approx(fd, rel=1e-5)
    for i in (0, 77, 150):
        fd = _central_fd(lambda s: J_of(alpha, s), src, i, 1e-4 * src[i])
        assert gsrc[i] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(gsrc).max())


def test_barycenter_grad_with_vertex_weights_matches_finite_differences(bary_setup):
    # the same composition with vertex weights a in every filter input (barycenter and Algorithm 1)
    X, Ls, Ld, M = bary_setup
    t, K = 2.0, 20
    b = oracle.cheb_coefficients(t, K)
    a = np.random.default_rng(13).uniform(0.7, 1.3, len(X))
    alpha = np.array([0.2, 0.5, 0.3])
    src = W.vmf_bump(X, np.array([0.0, 1.0, 0.0]), 3.0).astype(np.float64)
    src /= src.sum()
    J, gsrc, galpha = oracle.barycenter_distance_grad(Ls, b, src, M, alpha, t, 12, 15, a=a)

    def J_of(al, s=src):
        mu = oracle.barycenter(Ls, b, M, al, 12, a=a)
        return oracle.sinkhorn(Ls, b, s, mu, t, 15, a=a)["W2"]

    assert J == pytest.approx(J_of(alpha), rel=1e-13)
    for i in range(3):  # the central difference's O(h^2) error is 1.4e-5 at h = 1e-5 for alpha_3
        fd = _central_fd(J_of, alpha, i, 1e-6)
        assert galpha[i] == pytest.approx(fd, rel=2e-6)
    for i in (3, 90, 171):
        fd = _central_fd(lambda s: J_of(alpha, s), src, i, 1e-4 * src[i])
        assert gsrc[i] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(gsrc).max())


# --------------------------------------------------------------- families (Definitions 4.3, 4.4)
def _dense_sinkhorn_w2(H, mu, nu, t, iters):
    # Algorithm 1 with the exact kernel matrix H = expm(-t L) (not the Chebyshev series)
    v, w = np.zeros_like(mu), np.ones_like(nu)
    for _ in range(iters):
        v = mu / (H @ w)
        w = nu / (H @ v)
    return 4.0 * t * float(np.sum(mu * np.log(v) + nu * np.log(w)))


def test_barycentric_distance_one_hot_families_match_the_exact_kernel(bary_setup):
    # alpha = e_j: mu* = H(mu_j / H(1)) (closed form above); gamma is then Algorithm 1 between the
    # two normalised closed-form barycenters, here run with the dense matrix exponential
    X, Ls, Ld, M = bary_setup
    t, K = 2.0, 30
    H = heat_expm(Ld, t)
    one = np.ones(len(X))
    r = oracle.barycentric_distance(Ls, oracle.cheb_coefficients(t, K), M[:, :2], np.array([1.0, 0.0]),
                                    M[:, 1:], np.array([0.0, 1.0]), t, 6, 300)
    bT = H @ (M[:, 0] / (H @ one))
    bC = H @ (M[:, 2] / (H @ one))
    bT, bC = bT / bT.sum(), bC / bC.sum()
    np.testing.assert_allclose(r["muT"], bT, rtol=1e-9)
    np.testing.assert_allclose(r["muC"], bC, rtol=1e-9)
    assert r["W2"] == pytest.approx(_dense_sinkhorn_w2(H, bT, bC, t, 300), rel=1e-8)
    assert r["W"] == pytest.approx(math.sqrt(r["W2"]), rel=1e-15)


def test_barycentric_distance_symmetric_and_mass_invariant(bary_setup):
    X, Ls, Ld, M = bary_setup
    b = oracle.cheb_coefficients(2.0, 30)
    aT, aC = np.array([0.7, 0.3]), np.array([0.4, 0.6])
    r = oracle.barycentric_distance(Ls, b, M[:, :2], aT, M[:, 1:], aC, 2.0, 200, 400)
    r_swapped = oracle.barycentric_distance(Ls, b, M[:, 1:], aC, M[:, :2], aT, 2.0, 200, 400)
    assert r["W2"] == pytest.approx(r_swapped["W2"], rel=1e-9)
    # the barycenter scales with its inputs, and gamma compares the normalised barycenters
    r_scaled = oracle.barycentric_distance(Ls, b, 3.0 * M[:, :2], aT, 0.25 * M[:, 1:], aC, 2.0, 200, 400)
    assert r_scaled["W2"] == pytest.approx(r["W2"], rel=1e-9)
    # the pairing of members and weights matters, not their order
    r_perm = oracle.barycentric_distance(Ls, b, M[:, 1::-1], aT[::-1], M[:, 1:], aC, 2.0, 200, 400)
    assert r_perm["W2"] == pytest.approx(r["W2"], rel=1e-9)


def test_barycenter_effect_closed_forms():
    rng = np.random.default_rng(8)
    n, d = 50, 3
    Y = rng.standard_normal((n, d))
    # Dirac barycenters: the difference of the two nodes' features
    eT, eC = np.eye(n)[4] * 2.5, np.eye(n)[17]
    np.testing.assert_allclose(oracle.barycenter_effect(Y, eT, eC), Y[4] - Y[17], rtol=1e-14)
    # equal measures: no effect; a shift of all features: no change; a linear map acts linearly
    muT, muC = rng.random(n), rng.random(n)
    assert np.abs(oracle.barycenter_effect(Y, muT, 3 * muT)).max() < 1e-14
    tau = oracle.barycenter_effect(Y, muT, muC)
    np.testing.assert_allclose(oracle.barycenter_effect(Y + 7.0, muT, muC), tau, atol=1e-12)
    A = rng.standard_normal((d, 2))
    np.testing.assert_allclose(oracle.barycenter_effect(Y @ A, muT, muC), tau @ A, rtol=1e-12)
    # with the arithmetic mean of each family as its barycenter (the total-variation barycenter)
    # the effect is the difference of the families' mean features (Sec. 4, after Definition 4.4):
    # nine members centred at 5 and one at -60 against ten at 0 give (9 * 5 - 60) / 10 = -1.5
    y = np.concatenate([np.full(10, 5.0), [-60.0], np.zeros(10)])[:, None]
    T = np.zeros((21, 10))
    T[np.arange(9), np.arange(9)] = 1.0          # nine members, one node at 5 each
    T[10, 9] = 1.0                               # the outlier at -60
    C = np.zeros((21, 10))
    C[11 + np.arange(10), np.arange(10)] = 1.0   # ten members at 0
    assert oracle.barycenter_effect(y, T.mean(1), C.mean(1))[0] == pytest.approx(-1.5, rel=1e-14)


def _table2_rows():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table2_expected_barycenter_effect.txt")
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            name, m, s, mtv, stv = line.split()
            rows[name] = (float(m), float(s), float(mtv), float(stv))
    return rows


@pytest.mark.parametrize("outlier,row", [(None, "none"), (0.0, "0")])
def test_expected_barycenter_effect_reproduces_table2(outlier, row):
    # Table 2: the effect of the Geodesic Sinkhorn barycenters stays near the true shift of 5, and
    # the total-variation effect is the difference of empirical means; one seed against the
    # printed mean within three printed standard deviations
    mean, std, mean_tv, std_tv = _table2_rows()[row]
    X, MC, MT = W.treatment_families(outlier, seed=0)
    Ls, _ = oracle.build_graph(X.astype(np.float64), 10)
    b = oracle.cheb_coefficients(5.0, 30)
    muC = oracle.barycenter(Ls, b, MC, np.full(10, 0.1), 50)
    muT = oracle.barycenter(Ls, b, MT, np.full(10, 0.1), 50)
    tau = oracle.barycenter_effect(X[:, :1], muT, muC)[0]
    tau_tv = oracle.barycenter_effect(X[:, :1], MT.mean(1), MC.mean(1))[0]
    assert abs(tau - mean) < 3 * std
    assert abs(tau_tv - mean_tv) < 3 * std_tv


def test_sinkhorn_small_t_beyond_fp32_matches_dense_log_sum_exp():
    # The regime of the log-domain GPU loop: on the 2,000-point sphere pair at t = 1 the scalings
    # leave the FP32 range (|ln u| > ln FLT_MAX = 88.72) within 30 iterations.  The oracle's FP64
    # loop must still be exact there: compare it with the textbook log-domain form of the same
    # iteration on the dense kernel, f <- ln mu - LSE_j(ln H_ij + g_j), g <- ln nu - LSE_i(ln H_ij + f_i),
    # which never forms a scaling.
    from scipy.special import logsumexp
    p = W.sphere_pair()
    Ls, _ = oracle.build_graph(p.X.astype(np.float64), p.k)
    mu, nu = p.a.astype(np.float64), p.b.astype(np.float64)
    t, K, iters = 1.0, 20, 30
    b = oracle.cheb_coefficients(t, K)
    r = oracle.sinkhorn(Ls, b, mu, nu, t, iters)
    assert r["status"] == oracle.OK
    H = _dense_filter(Ls, b, len(mu))
    assert H.min() >= 0.0  # the truncated series stays non-negative on this graph
    with np.errstate(divide="ignore"):
        lH = np.log(H)
    f, g = np.zeros(len(mu)), np.zeros(len(mu))
    for _ in range(iters):
        f = np.log(mu) - logsumexp(lH + g[None, :], axis=1)
        g = np.log(nu) - logsumexp(lH.T + f[None, :], axis=1)
    assert max(np.abs(f).max(), np.abs(g).max()) > 88.73
    np.testing.assert_allclose(np.log(r["v"]), f, rtol=0, atol=1e-10)
    np.testing.assert_allclose(np.log(r["w"]), g, rtol=0, atol=1e-10)
    assert r["W2"] == pytest.approx(4 * t * (mu @ f + nu @ g), rel=1e-12)
