"""Pins for the FP64 oracle against things other than itself (CPU only).

Coefficients   -> scipy's exponentially scaled Bessel routine, Chebyshev-Gauss quadrature,
                  the closed-form values of the series at y = +-1, the Bessel-tail bound.
Heat filter    -> dense expm / eigh of the Laplacian built from coordinates, the cycle-graph
                  Fourier closed form, symmetry of p_K(L, t).
Graph          -> scipy's k-d tree, pure-Python brute force with the tie rule, the null vector
                  sqrt(deg) of the normalised Laplacian, its spectrum inside [0, 2].
"""
import math

import numpy as np
import pytest
import scipy.special as ss
from scipy.spatial import cKDTree

import oracle
from paper_2211_00805_gb300 import workloads as W
from tests.oracle_helpers import (bessel_tail_bound, csr_to_dense, dense_knn_laplacian, heat_eigh,
                                  heat_expm)


# ------------------------------------------------------------------------------ coefficients
@pytest.mark.parametrize("t,K", [(0.5, 12), (1.0, 20), (5.0, 30), (8.0, 40), (10.0, 40), (20.0, 60)])
def test_coefficients_match_scipy_ive(t, K):
    b = oracle.cheb_coefficients(t, K)
    k = np.arange(K + 1)
    ref = 2.0 * (-1.0) ** k * ss.ive(k, t)
    np.testing.assert_allclose(b, ref, rtol=1e-12, atol=1e-300)


@pytest.mark.parametrize("t,K", [(1.0, 20), (5.0, 30), (10.0, 40)])
def test_coefficients_match_quadrature(t, K):
    assert np.max(np.abs(oracle.cheb_coefficients(t, K)
                         - oracle.cheb_coefficients_quadrature(t, K))) < 1e-14


@pytest.mark.parametrize("t", [0.5, 1.0, 5.0, 10.0])
def test_coefficients_endpoint_values(t):
    # T_k(1) = 1 and T_k(-1) = (-1)^k: the series must give exp(-2t) at y = 1 and 1 at y = -1.
    b = oracle.cheb_coefficients(t, 120)
    k = np.arange(len(b))
    at_p1 = 0.5 * b[0] + math.fsum(b[1:])
    at_m1 = 0.5 * b[0] + math.fsum((b * (-1.0) ** k)[1:])
    assert abs(at_p1 - math.exp(-2 * t)) < 1e-15
    assert abs(at_m1 - 1.0) < 1e-14


@pytest.mark.parametrize("t,K", [(1.0, 20), (5.0, 30), (10.0, 40), (8.0, 40), (5.0, 16)])
def test_coefficient_tail_below_bound(t, K):
    b = oracle.cheb_coefficients(t, K + 80)
    assert np.sum(np.abs(b[K + 1:])) <= bessel_tail_bound(t, K) * (1 + 1e-12)


# ------------------------------------------------------------------------------- heat filter
def _small_graph(n=120, d=2, k=6, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d))
    Ls, ex = oracle.build_graph(X, k)
    return X, Ls, ex


@pytest.mark.parametrize("t,K", [(1.0, 20), (5.0, 30), (0.3, 8)])
def test_filter_matches_dense_expm_and_eigh(t, K):
    X, Ls, ex = _small_graph()
    n = len(X)
    Ld, _, _, _ = dense_knn_laplacian(X, 6)
    b = oracle.cheb_coefficients(t, K)
    V = np.random.default_rng(2).standard_normal((n, 3))
    Y = oracle.heat_apply(Ls, b, V)
    tail = bessel_tail_bound(t, K)
    # |p_K(L) - exp(-tL)|_2 <= sum_{k>K} |b_k| because |T_k| <= 1 on the spectrum of L - Id
    bound = tail * np.linalg.norm(V, axis=0).max() + 1e-12
    assert np.max(np.abs(Y - heat_expm(Ld, t) @ V)) <= bound
    assert np.max(np.abs(Y - heat_eigh(Ld, t) @ V)) <= bound


def test_filter_truncation_error_decays_with_K():
    X, Ls, ex = _small_graph(n=80)
    Ld, *_ = dense_knn_laplacian(X, 6)
    e0 = np.zeros(len(X)); e0[0] = 1.0
    exact = heat_expm(Ld, 2.0)[:, 0]
    errs = [np.max(np.abs(oracle.heat_apply(Ls, oracle.cheb_coefficients(2.0, K), e0) - exact))
            for K in (2, 4, 6, 8, 10)]
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    for K, e in zip((2, 4, 6, 8, 10), errs):
        assert e <= bessel_tail_bound(2.0, K) + 1e-14


@pytest.mark.parametrize("n,t,K", [(50, 1.0, 20), (64, 3.0, 30), (31, 5.0, 40)])
def test_cycle_graph_closed_form(n, t, K):
    # cycle C_n with unit weights: deg = 2, L = I - A/2, eigenpairs 1 - cos(2 pi m / n) with
    # Fourier modes, so H_t(i, 0) = (1/n) sum_m exp(-t (1 - cos(2 pi m/n))) cos(2 pi m i / n).
    rowptr = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    col = np.empty(2 * n, np.int32)
    for i in range(n):
        col[2 * i:2 * i + 2] = sorted([(i - 1) % n, (i + 1) % n])
    deg, L = oracle.laplacian(rowptr, col, np.ones(2 * n))
    assert np.all(deg == 2.0)
    Ls = oracle.shifted(L)
    e0 = np.zeros(n); e0[0] = 1.0
    y = oracle.heat_apply(Ls, oracle.cheb_coefficients(t, K), e0)
    m = np.arange(n)
    i = np.arange(n)
    closed = (np.exp(-t * (1 - np.cos(2 * np.pi * m / n)))[None, :]
              * np.cos(2 * np.pi * np.outer(i, m) / n)).sum(1) / n
    assert np.max(np.abs(y - closed)) <= bessel_tail_bound(t, K) + 1e-14


def test_filter_is_symmetric():
    X, Ls, ex = _small_graph(n=150, d=3, k=8, seed=7)
    b = oracle.cheb_coefficients(3.0, 25)
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal(150), rng.standard_normal(150)
    lhs = x @ oracle.heat_apply(Ls, b, y)
    rhs = y @ oracle.heat_apply(Ls, b, x)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


def test_filter_block_equals_columns():
    X, Ls, ex = _small_graph(n=90, d=2, k=5, seed=4)
    b = oracle.cheb_coefficients(2.0, 15)
    V = np.random.default_rng(5).standard_normal((90, 4))
    Y = oracle.heat_apply(Ls, b, V)
    for c in range(4):
        assert np.array_equal(Y[:, c], oracle.heat_apply(Ls, b, V[:, c]))


# ------------------------------------------------------------------------------------ graph
def test_knn_matches_kdtree():
    rng = np.random.default_rng(11)
    X = rng.standard_normal((500, 5))
    idx, dist = oracle.knn(X, 7)
    dref, iref = cKDTree(X).query(X, 8)
    assert np.array_equal(idx, iref[:, 1:])
    np.testing.assert_allclose(dist, dref[:, 1:], rtol=1e-12)


def test_knn_ties_and_self_exclusion_brute_force():
    # duplicated and lattice points produce exact ties; the rule is (distance, index) ascending
    X = np.array([[0, 0], [1, 0], [0, 1], [1, 1], [0, 0], [2, 0], [1, 0], [0, 2]], float)
    k = 4
    idx, dist = oracle.knn(X, k)
    for q in range(len(X)):
        cand = sorted((sum((X[q][c] - X[j][c]) ** 2 for c in range(2)), j)
                      for j in range(len(X)) if j != q)[:k]
        assert [j for _, j in cand] == list(idx[q])
        assert np.allclose([math.sqrt(s) for s, _ in cand], dist[q])


def test_knn_sampled_rows_equal_full():
    rng = np.random.default_rng(12)
    X = rng.standard_normal((300, 4))
    idx, dist = oracle.knn(X, 5)
    rows = np.array([0, 17, 299, 150])
    i2, d2 = oracle.knn(X, 5, rows=rows)
    assert np.array_equal(i2, idx[rows]) and np.array_equal(d2, dist[rows])


def test_median_sigma_definition():
    d = np.random.default_rng(0).random((7, 3))
    s = sorted(d.ravel().tolist())
    assert oracle.median_sigma(d) == s[10]
    d2 = np.random.default_rng(1).random((4, 3))
    s2 = sorted(d2.ravel().tolist())
    assert oracle.median_sigma(d2) == pytest.approx(0.5 * (s2[5] + s2[6]), rel=0, abs=1e-16)


def test_graph_matches_dense_construction():
    rng = np.random.default_rng(21)
    X = rng.standard_normal((140, 3))
    Ls, ex = oracle.build_graph(X, 6)
    Ld, Ad, degd, sig = dense_knn_laplacian(X, 6)
    assert ex["sigma"] == pytest.approx(sig, rel=1e-14)
    n = len(X)
    A = csr_to_dense(ex["rowptr"], ex["col"], ex["A"], n)
    assert np.array_equal(A != 0, Ad != 0)
    np.testing.assert_allclose(A, Ad, rtol=1e-12, atol=0)
    np.testing.assert_allclose(A, A.T, rtol=0, atol=0)
    L = csr_to_dense(*ex["L"], n)
    np.testing.assert_allclose(L, Ld, atol=1e-14)
    np.testing.assert_allclose(csr_to_dense(*Ls, n), Ld - np.eye(n), atol=1e-14)


def test_laplacian_null_vector_and_spectrum():
    rng = np.random.default_rng(22)
    X = rng.standard_normal((200, 2))
    Ls, ex = oracle.build_graph(X, 5)
    n = len(X)
    L = csr_to_dense(*ex["L"], n)
    # D^{1/2} 1 spans the kernel of the symmetric-normalised Laplacian
    assert np.max(np.abs(L @ np.sqrt(ex["deg"]))) < 1e-13
    lam = np.linalg.eigvalsh(L)
    assert lam.min() > -1e-12 and lam.max() < 2 + 1e-12
    assert np.all(np.diag(L) == 1.0)


def test_benchmark_graphs_are_connected():
    # the cluster-curve workload is built so that consecutive clusters overlap: its kNN graph (and
    # the manifold workload's) must have one connected component, or Sinkhorn has no transport
    # between components and the barycenter is ill-posed
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import connected_components
    for X in (W.cluster_curves(4000, 30, seed=3)[0], W.tanh_manifold(4000, 10, 50, 2)[0]):
        Ls, ex = oracle.build_graph(X.astype(np.float64), 10)
        n = len(X)
        A = csr_matrix((ex["A"], ex["col"], ex["rowptr"]), shape=(n, n))
        assert connected_components(A, directed=False)[0] == 1


# ------------------------------------------------------------- Euler implicit kernel (Sec. 4)
def test_euler_implicit_kernel_matches_its_spectral_form_and_tends_to_the_exponential():
    # (I + (t/K) L)^{-K} = U diag((1 + t lambda / K)^{-K}) U^T, and -> exp(-t L) as K grows
    from tests.oracle_helpers import dense_knn_laplacian, heat_eigh
    X = W.sphere(300, seed=4).astype(np.float64)
    Ls, _ = oracle.build_graph(X, 8)
    Ld, *_ = dense_knn_laplacian(X, 8)
    lam, U = np.linalg.eigh(Ld)
    V = np.random.default_rng(2).random((300, 3))
    t = 2.0
    errs = []
    for K in (5, 20, 80):
        Y = oracle.heat_apply_implicit(Ls, t, K, V)
        ref = (U * (1.0 + t * lam / K) ** (-K)) @ (U.T @ V)
        np.testing.assert_allclose(Y, ref, rtol=1e-9, atol=1e-12)
        errs.append(np.abs(Y - heat_eigh(Ld, t) @ V).max())
    # first-order method: the error falls about fourfold per fourfold K
    assert errs[0] > 3 * errs[1] > 9 * errs[2]


# ----------------------------------------------- combinatorial Laplacian D - A (Sec. 3.4 / 3.5)
@pytest.mark.parametrize("t,K", [(0.2, 20), (0.5, 30)])
def test_combinatorial_filter_matches_dense_expm(t, K):
    X, Ls, ex = _small_graph()
    n = len(X)
    _, A, deg, _ = dense_knn_laplacian(X, 6)
    Lc = np.diag(deg) - A  # straight from the coordinates
    V = np.random.default_rng(4).standard_normal((n, 3))
    Y = oracle.heat_apply_combinatorial(ex["rowptr"], ex["col"], ex["A"], t, K, V)
    lam = 2.0 * deg.max()
    # |T_k| <= 1 on the spectrum of L' - Id, so the error is at most the tail at time t lam / 2
    bound = bessel_tail_bound(t * lam / 2, K) * np.linalg.norm(V, axis=0).max() + 1e-12
    assert np.max(np.abs(Y - heat_expm(Lc, t) @ V)) <= bound


def test_combinatorial_rescaling_bounds_the_spectrum():
    X, Ls, ex = _small_graph()
    n = len(X)
    (rp, col, val), lam = oracle.combinatorial_shifted(ex["rowptr"], ex["col"], ex["A"])
    M = csr_to_dense(rp, col, val, n)
    ev = np.linalg.eigvalsh(M)
    assert ev.min() >= -1 - 1e-12 and ev.max() <= 1 + 1e-12
    np.testing.assert_allclose(M @ np.ones(n), -np.ones(n), atol=1e-13)  # L 1 = 0
    _, A, deg, _ = dense_knn_laplacian(X, 6)
    assert np.linalg.eigvalsh(np.diag(deg) - A).max() <= lam
    assert lam == pytest.approx(2.0 * deg.max(), rel=1e-13)


def test_combinatorial_heat_preserves_constants_and_mass():
    # exp(-t (D - A)) fixes constants and, being symmetric, the total mass sum_i f_i
    X, Ls, ex = _small_graph()
    n = len(X)
    t, K = 0.5, 30
    (_, _, _), lam = oracle.combinatorial_shifted(ex["rowptr"], ex["col"], ex["A"])
    tail = bessel_tail_bound(t * lam / 2, K)
    y = oracle.heat_apply_combinatorial(ex["rowptr"], ex["col"], ex["A"], t, K, np.ones(n))
    assert np.max(np.abs(y - 1.0)) <= tail + 1e-13
    f = np.random.default_rng(6).random(n)
    g = oracle.heat_apply_combinatorial(ex["rowptr"], ex["col"], ex["A"], t, K, f)
    assert abs(g.sum() - f.sum()) <= tail * f.sum() + 1e-12
    assert np.max(np.abs(g - f)) > 1e-3  # and it does diffuse


@pytest.mark.parametrize("n,t,K", [(50, 0.5, 30), (64, 1.5, 40)])
def test_combinatorial_cycle_closed_form(n, t, K):
    # cycle C_n, unit weights: D - A = 2 I - A has eigenvalues 2 - 2 cos(2 pi m / n) on the Fourier
    # modes (twice the normalised Laplacian's), so H_t(i, 0) is the Fourier sum below
    rowptr = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    col = np.empty(2 * n, np.int32)
    for i in range(n):
        col[2 * i:2 * i + 2] = sorted([(i - 1) % n, (i + 1) % n])
    e0 = np.zeros(n); e0[0] = 1.0
    y = oracle.heat_apply_combinatorial(rowptr, col, np.ones(2 * n), t, K, e0)
    m = np.arange(n)
    closed = (np.exp(-t * (2 - 2 * np.cos(2 * np.pi * m / n)))[None, :]
              * np.cos(2 * np.pi * np.outer(m, m) / n)).sum(1) / n
    assert np.max(np.abs(y - closed)) <= bessel_tail_bound(2 * t, K) + 1e-14
