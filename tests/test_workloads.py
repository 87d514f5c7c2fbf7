"""The seeded input generators do what their recipes state (CPU only): shapes, types,
determinism, and the distributional facts the recipes claim."""
import math

import numpy as np
import pytest

from paper_2211_00805_gb300 import workloads as W


def test_generators_are_deterministic_per_seed():
    assert np.array_equal(W.sphere(500, 3), W.sphere(500, 3))
    assert not np.array_equal(W.sphere(500, 3), W.sphere(500, 4))
    X1, Z1 = W.tanh_manifold(300, 4, 12, seed=7)
    X2, Z2 = W.tanh_manifold(300, 4, 12, seed=7)
    assert np.array_equal(X1, X2) and np.array_equal(Z1, Z2)
    assert np.array_equal(W.cluster_curves(400, 8, seed=1)[0], W.cluster_curves(400, 8, seed=1)[0])


def test_sphere_points_are_unit_vectors_spread_over_the_sphere():
    X = W.sphere(20_000, 0)
    assert X.dtype == np.float32 and X.shape == (20_000, 3)
    np.testing.assert_allclose(np.linalg.norm(X.astype(np.float64), axis=1), 1.0, atol=1e-6)
    assert np.abs(X.mean(0)).max() < 0.03  # uniform: mean at the centre
    np.testing.assert_allclose((X.astype(np.float64) ** 2).mean(0), 1 / 3, atol=0.02)


def test_tanh_manifold_shapes_and_latents():
    X, Z = W.tanh_manifold(5000, 10, 50, seed=2)
    assert X.dtype == np.float32 and X.shape == (5000, 50) and Z.shape == (5000, 10)
    assert np.isfinite(X).all()
    assert abs(Z.mean()) < 0.05 and abs(Z.std() - 1.0) < 0.05  # z ~ N(0, I)


def test_cluster_spread_is_a_fixed_fraction_of_the_gap_between_centres():
    clusters, curves, spread = 20, 4, 0.35
    X, labels = W.cluster_curves(60_000, 30, clusters=clusters, curves=curves, seed=3, spread=spread)
    assert X.shape == (60_000, 30) and labels.min() == 0 and labels.max() == clusters - 1
    per = clusters // curves
    means = np.stack([X[labels == j].astype(np.float64).mean(0) for j in range(clusters)])
    sds = np.array([X[labels == j].astype(np.float64).std(0).mean() for j in range(clusters)])
    for c in range(curves):
        prev = np.zeros(30)  # every curve starts at the shared origin
        for q in range(per):
            j = c * per + q
            gap = np.linalg.norm(means[j] - prev)
            assert sds[j] / gap == pytest.approx(spread, rel=0.08), (c, q)
            prev = means[j]


def test_bump_distributions_sum_to_one_with_their_stated_ratios():
    X = W.sphere(3000, 1).astype(np.float64)
    c = np.array([0.0, 0.0, 1.0])
    a = W.vmf_bump(X, c, 20.0).astype(np.float64)
    assert a.sum() == pytest.approx(1.0, rel=1e-6)
    i, j = 10, 20
    assert a[i] / a[j] == pytest.approx(math.exp(20.0 * (X[i] @ c - X[j] @ c)), rel=1e-4)
    Z = np.random.default_rng(0).standard_normal((3000, 5))
    cz = np.random.default_rng(1).standard_normal(5)
    s = W.softmax_bump(Z, cz).astype(np.float64)
    assert s.sum() == pytest.approx(1.0, rel=1e-6)
    d2 = ((Z - cz) ** 2).sum(1)
    assert s[i] / s[j] == pytest.approx(math.exp(-0.5 * (d2[i] - d2[j])), rel=1e-4)


def test_cluster_unions_are_uniform_on_three_clusters():
    _, labels = W.cluster_curves(5000, 8, seed=3)
    M = W.cluster_unions(labels, 12, 3, seed=9)
    assert M.shape == (5000, 12) and M.dtype == np.float32
    for i in range(12):
        col = M[:, i].astype(np.float64)
        assert col.sum() == pytest.approx(1.0, rel=1e-5)
        assert len(np.unique(labels[col > 0])) == 3
        assert np.ptp(col[col > 0]) == 0.0  # uniform on its support


def test_dirichlet_support_size_and_mass():
    w = W.dirichlet_support(10_000, 0.1, np.random.default_rng(2))
    assert (w > 0).sum() == 1000 and w.astype(np.float64).sum() == pytest.approx(1.0, rel=1e-5)


@pytest.mark.parametrize("outlier", [None, 0.0, -30.0])
def test_treatment_families_members_and_centres(outlier):
    X, MC, MT = W.treatment_families(outlier, seed=0, per=400)
    assert X.shape == (8000, 5) and MC.shape == (8000, 10) and MT.shape == (8000, 10)
    np.testing.assert_allclose(MC.sum(0), 1.0, rtol=1e-5)
    np.testing.assert_allclose(MT.sum(0), 1.0, rtol=1e-5)
    first = X[:, 0].astype(np.float64)
    centres = [0.0] * 10 + [5.0] * 9 + [5.0 if outlier is None else outlier]
    for i, c in enumerate(centres):
        member = first[i * 400:(i + 1) * 400]
        assert abs(member.mean() - c) < 0.2
        assert (MC if i < 10 else MT)[i * 400, i % 10] == pytest.approx(1 / 400)


def test_ragged_batch_ranges():
    probs = W.ragged_batch(count=40, n_min=200, n_max=2000, iters=7)
    assert len(probs) == 40
    for p in probs:
        n, D = p.X.shape
        assert 200 <= n <= 2000 and 3 <= D <= 20
        assert p.k in (8, 10, 15) and p.K in (16, 24, 32) and p.t == 5.0 and p.iters == 7
        for m in (p.a, p.b):
            assert (m > 0).sum() == round(0.1 * n) and m.astype(np.float64).sum() == pytest.approx(1.0, rel=1e-5)
    ns = np.log([p.X.shape[0] for p in probs])
    assert ns.min() < math.log(400) and ns.max() > math.log(1000)  # spread over the log range


def test_named_workload_defaults():
    p = W.sphere_pair(n=300)
    assert (p.k, p.K, p.t, p.iters) == (10, 20, 1.0, 200)
    q = W.manifold_pair(n=500)
    assert q.X.shape == (500, 50) and (q.k, q.K, q.t, q.iters) == (15, 30, 5.0, 500)
