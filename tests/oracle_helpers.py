"""Dense, textbook helpers used only as independent pins for the oracle (tiny graphs).

Nothing here is shared with the oracle's arithmetic: the dense matrices are built from the
point coordinates directly and the heat kernel comes from scipy's matrix exponential or numpy's
symmetric eigendecomposition.
"""
import numpy as np
import scipy.linalg


def dense_knn_laplacian(X, k, sigma=None):
    """Dense kNN affinity + symmetric-normalised Laplacian straight from the coordinates."""
    X = np.asarray(X, np.float64)
    n = len(X)
    D2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(D2, np.inf)
    order = np.argsort(D2, axis=1, kind="stable")[:, :k]
    dists = np.sqrt(np.take_along_axis(D2, order, axis=1))
    if sigma is None:
        sigma = float(np.median(dists))
    E = np.zeros((n, n), bool)
    E[np.repeat(np.arange(n), k), order.ravel()] = True
    E = E | E.T
    D = np.sqrt(np.where(np.isinf(D2), 0.0, D2))
    A = np.where(E, np.exp(-(D ** 2) / sigma ** 2), 0.0)
    deg = A.sum(1)
    L = np.eye(n) - A / np.sqrt(np.outer(deg, deg))
    return L, A, deg, sigma


def heat_expm(L, t):
    return scipy.linalg.expm(-t * L)


def heat_eigh(L, t):
    lam, psi = np.linalg.eigh(L)
    return (psi * np.exp(-t * lam)) @ psi.T


def csr_to_dense(rp, col, val, n):
    M = np.zeros((n, n))
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            M[i, col[e]] += val[e]
    return M


def bessel_tail_bound(t, K, terms=200):
    """Upper bound on sum_{k>K} |b_k| from I_k(t) <= (t/2)^k / k! * exp(t^2 / (4 (k + 1)))."""
    from math import exp, lgamma, log
    s = 0.0
    for k in range(K + 1, K + 1 + terms):
        s += 2.0 * exp(-t) * exp(k * log(t / 2) - lgamma(k + 1) + t * t / (4 * (k + 1)))
    return s
