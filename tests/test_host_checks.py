"""CPU tests of the test harness's own checks: the kNN list comparison must reject a wrong
neighbour on either side of the symmetric difference (mistakes planted in a copy of the oracle's
lists), and accept swaps between exact ties."""
import numpy as np
import pytest

import oracle
from tests.gpu_common import knn_lists_match


@pytest.fixture(scope="module")
def knn_case():
    X = np.random.default_rng(4).standard_normal((300, 6))
    idx, dist = oracle.knn(X, 8)
    return X, idx, dist


def test_identical_lists_pass(knn_case):
    X, idx, dist = knn_case
    assert knn_lists_match(idx, dist.astype(np.float32), idx, dist, X) == 0


def test_wrong_kth_neighbour_is_caught(knn_case):
    X, idx, dist = knn_case
    bad = idx.copy()
    q = 17
    far = int(np.argmax(((X - X[q]) ** 2).sum(1)))
    bad[q, -1] = far  # the k-th neighbour replaced by the farthest point
    with pytest.raises(AssertionError):
        knn_lists_match(bad, None, idx, dist, X)


def test_wrong_distance_is_caught(knn_case):
    X, idx, dist = knn_case
    gd = dist.astype(np.float32).copy()
    gd[5, 2] *= 1.001
    with pytest.raises(AssertionError):
        knn_lists_match(idx, gd, idx, dist, X)


def test_self_or_repeat_is_caught(knn_case):
    X, idx, dist = knn_case
    bad = idx.copy()
    bad[9, 3] = 9
    with pytest.raises(AssertionError):
        knn_lists_match(bad, None, idx, dist, X)
    bad = idx.copy()
    bad[9, 3] = bad[9, 2]
    with pytest.raises(AssertionError):
        knn_lists_match(bad, None, idx, dist, X)


def test_exact_tie_swap_is_accepted():
    # a query with two equidistant candidates for the last place: either may be listed
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0], [0.0, -2.0], [5.0, 5.0]])
    idx, dist = oracle.knn(X, 2, rows=np.array([0]))
    assert idx[0, 1] == 2  # ties broken by lower index in the oracle
    swapped = idx.copy()
    swapped[0, 1] = 3
    assert knn_lists_match(swapped, None, idx, dist, X, rows=np.array([0])) == 1
