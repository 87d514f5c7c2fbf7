"""GPU heat filter of the combinatorial Laplacian D - A (Sec. 3.4), rescaled to the spectrum [0, 2]
that Sec. 3.5 assumes (lam = 2 max degree, time s = t lam / 2), against the FP64 oracle
(oracle.heat_apply_combinatorial) on the same FP32 affinities, and against the cycle's closed form.

Tolerance (the heat-filter tolerance): |gpu - ref| <= 1e-4 |ref| + 1e-6 max|ref|.
"""
import numpy as np
import pytest

import oracle
from tests.gpu_common import assert_close, oracle_csr_to_dev, to_dev, to_np

pytestmark = pytest.mark.gpu

RTOL, ATOL_REL = 1e-4, 1e-6


@pytest.fixture(scope="module")
def gs():
    from paper_2211_00805_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(gs):
    return gs.Context()


def _knn_graph(n, d, k, seed):
    X = np.random.default_rng(seed).standard_normal((n, d))
    idx, dist = oracle.knn(X, k)
    rp, col, A = oracle.affinity_graph(idx, dist, oracle.median_sigma(dist))
    return rp, col, A.astype(np.float32).astype(np.float64)  # the values the GPU receives


@pytest.mark.parametrize("B", [1, 5, 32])
def test_combinatorial_filter_matches_oracle_knn(gs, ctx, B):
    rp, col, A = _knn_graph(1800, 3, 9, seed=B)
    g = gs.gs_graph_from_csr(ctx, *oracle_csr_to_dev(rp, col, A))
    V = np.random.default_rng(50 + B).random((1800, B)).astype(np.float32)
    deg = np.bincount(np.repeat(np.arange(1800), np.diff(rp)), weights=A, minlength=1800)
    for t, K in [(0.05, 20), (0.3, 40), (1.0, 3)]:
        Y, lam = gs.gs_heat_apply_combinatorial(ctx, g, t, K, to_dev(V))
        assert lam == pytest.approx(2 * deg.max(), rel=1e-12)
        ref = oracle.heat_apply_combinatorial(rp, col, A, t, K, V.astype(np.float64))
        assert_close(to_np(Y), ref, RTOL, ATOL_REL * np.abs(ref).max(), f"B={B} t={t} K={K}")
    gs.gs_sync(ctx)


def test_combinatorial_filter_cycle_closed_form(gs, ctx):
    # unit-weight cycle: D - A has eigenvalues 2 - 2 cos(2 pi m / n); lam = 4
    n = 64
    rp = np.arange(0, 2 * n + 1, 2, dtype=np.int64)
    col = np.empty(2 * n, np.int32)
    for i in range(n):
        col[2 * i:2 * i + 2] = sorted([(i - 1) % n, (i + 1) % n])
    A = np.ones(2 * n)
    g = gs.gs_graph_from_csr(ctx, *oracle_csr_to_dev(rp, col, A))
    e0 = np.zeros(n, np.float32)
    e0[7] = 1.0
    t, K = 0.8, 40
    y, lam = gs.gs_heat_apply_combinatorial(ctx, g, t, K, to_dev(e0))
    assert lam == 4.0
    m = np.arange(n)
    closed = (np.exp(-t * (2 - 2 * np.cos(2 * np.pi * m / n)))[None, :]
              * np.cos(2 * np.pi * np.outer(np.arange(n) - 7, m) / n)).sum(1) / n
    assert_close(to_np(y), closed, RTOL, ATOL_REL * closed.max(), "cycle")
    ref = oracle.heat_apply_combinatorial(rp, col, A, t, K, e0.astype(np.float64))
    assert_close(to_np(y), ref, RTOL, ATOL_REL * np.abs(ref).max(), "cycle vs oracle")


def test_combinatorial_filter_on_a_point_graph_preserves_mass(gs, ctx):
    # on a graph built from points (locality order, caller-order results): exp(-t(D - A)) keeps
    # constants and the total mass (columns of D - A sum to zero), to the FP32 floor
    X = np.random.default_rng(3).standard_normal((5000, 4)).astype(np.float32)
    g = gs.gs_build_graph(ctx, to_dev(X), 10)
    rp, col, A, _ = gs.gs_graph_export_csr(ctx, g)
    V = np.random.default_rng(4).random((5000, 4)).astype(np.float32)
    Y, lam = gs.gs_heat_apply_combinatorial(ctx, g, 0.2, 30, to_dev(V))
    ref = oracle.heat_apply_combinatorial(to_np(rp), to_np(col), to_np(A).astype(np.float64), 0.2, 30,
                                          V.astype(np.float64))
    assert_close(to_np(Y), ref, RTOL, ATOL_REL * np.abs(ref).max(), "point graph")
    np.testing.assert_allclose(to_np(Y).astype(np.float64).sum(0), V.astype(np.float64).sum(0), rtol=1e-5)
