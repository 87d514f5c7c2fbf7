"""Geodesic Sinkhorn oracle: a plain, slow, FP64 CPU statement of the method.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this package.  It shares no code with the CUDA library (no kernel,
header, helper, table or constant generator), and the CUDA library never imports it.

Notation follows the paper (arXiv 2211.00805):

* ``L``      the symmetric-normalised graph Laplacian I - D^{-1/2} A D^{-1/2} (Sec. 3.4 defines the
             combinatorial one but assumes its spectrum lies in [0, 2], Sec. 3.5; the normalised one
             is the reading taken here, since it satisfies that assumption by construction);
* ``Ls``     the shifted operator L - Id on which the Chebyshev polynomials act (Sec. 3.5);
* ``b``      the Chebyshev coefficients b_0..b_K of the expansion of H_t = exp(-t L) (Sec. 3.5);
* ``mu, nu`` the two distributions, ``v, w`` their scalings and ``a`` the vertex weights of
             Algorithm 1 (Sec. 4);
* barycenter: distributions mu_i, weights alpha_i, scalings v_i, w_i (Sec. 3.3, with the
             iterative-Bregman-projection algorithm of the convolutional-Wasserstein paper it cites).
* the combinatorial Laplacian D - A itself (Sec. 3.4), as a filter variant:
             ``combinatorial_shifted`` rescales it by 2 / lam, lam = 2 max D_ii >= lambda_n, and
             ``heat_apply_combinatorial`` runs the same expansion at time t lam / 2.

Two heavy loops (brute-force kNN and the CSR recurrence) live in ``oracle_core.c``, compiled with
plain ``gcc -O2 -fopenmp``; everything else is numpy, one step per line of the method.

Parity status: every function here is pinned by ``tests/test_oracle_*.py`` against something other
than itself (dense eigendecomposition / matrix exponential, the cycle-graph closed form, scipy's
Bessel routine and k-d tree, the Bessel-tail bound, invariants, finite differences).  None is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle_core.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_core.so")

OK, NONFINITE, NOT_CONVERGED = 0, 4, 5


def build(force: bool = False) -> str:
    """Compile ``oracle_core.c`` into ``oracle/_build/liboracle_core.so`` (host gcc, no GPU)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


_lib = None


def _core():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        p = ctypes.c_void_p
        lib.or_knn_rows.argtypes = [p, i64, i32, i32, p, i64, p, p]
        lib.or_knn_rows.restype = i32
        lib.or_cheb_filter.argtypes = [i64, p, p, p, i32, p, i32, p, p]
        lib.or_cheb_filter.restype = i32
        lib.or_num_threads.argtypes = []
        lib.or_num_threads.restype = i32
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def num_threads() -> int:
    """Host threads the C core uses (OpenMP's maximum)."""
    return int(_core().or_num_threads())


# --------------------------------------------------------------------------------------------
# Graph (Sec. 4: a common graph built with an affinity kernel; Sec. 3.4: A, D, L)
# --------------------------------------------------------------------------------------------
def knn(X, k: int, rows=None):
    """k nearest neighbours by brute force, FP64 direct differences, self excluded, ties -> lower index.

    Returns ``(idx int32 [r, k], dist float64 [r, k])`` for the query ``rows`` (default: all).
    """
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, d = X.shape
    rows = np.arange(n, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, np.int64)
    idx = np.empty((len(rows), k), np.int32)
    dist = np.empty((len(rows), k), np.float64)
    rc = _core().or_knn_rows(_ptr(X), n, d, k, _ptr(rows), len(rows), _ptr(idx), _ptr(dist))
    if rc != 0:
        raise ValueError("knn: bad arguments")
    return idx, dist


def median_sigma(dist) -> float:
    """Kernel bandwidth sigma = median of all n*k kNN distances (mean of the two middle values
    when the count is even)."""
    return float(np.median(np.asarray(dist, np.float64)))


def affinity_graph(idx, dist, sigma: float):
    """Symmetric kNN affinity graph: edge set = union of the directed kNN edges, weight
    A_ij = exp(-d_ij^2 / sigma^2), no self-loops (Sec. 3.4's weighted adjacency A).

    Returns CSR ``(rowptr int64 [n+1], col int32 [nnz], A float64 [nnz])``, columns ascending.
    """
    idx = np.asarray(idx)
    dist = np.asarray(dist, np.float64)
    n, k = idx.shape
    src = np.repeat(np.arange(n, dtype=np.int64), k)
    dst = idx.reshape(-1).astype(np.int64)
    d = dist.reshape(-1)
    # both directions of every kNN edge; the distance of (i, j) and (j, i) is the same number
    rows = np.concatenate([src, dst])
    cols = np.concatenate([dst, src])
    dd = np.concatenate([d, d])
    order = np.lexsort((cols, rows))
    rows, cols, dd = rows[order], cols[order], dd[order]
    keep = np.ones(len(rows), bool)
    keep[1:] = (rows[1:] != rows[:-1]) | (cols[1:] != cols[:-1])
    rows, cols, dd = rows[keep], cols[keep], dd[keep]
    A = np.exp(-(dd * dd) / (sigma * sigma))
    rowptr = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rowptr[1:])
    return rowptr, cols.astype(np.int32), A


def laplacian(rowptr, col, A):
    """Symmetric-normalised Laplacian L = I - D^{-1/2} A D^{-1/2}, D_ii = sum_k A_ik (Sec. 3.4).

    Returns ``(deg, (rowptr, col, val))`` with the diagonal stored, columns ascending.
    """
    rowptr = np.asarray(rowptr, np.int64)
    col = np.asarray(col, np.int32)
    A = np.asarray(A, np.float64)
    n = len(rowptr) - 1
    row = np.repeat(np.arange(n), np.diff(rowptr))
    deg = np.bincount(row, weights=A, minlength=n)
    offdiag = -A / np.sqrt(deg[row] * deg[col])
    # insert the unit diagonal (there are no self-loops in A)
    rows = np.concatenate([row, np.arange(n)])
    cols = np.concatenate([col.astype(np.int64), np.arange(n)])
    vals = np.concatenate([offdiag, np.ones(n)])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    return deg, (rp, cols.astype(np.int32), vals)


def shifted(L):
    """Ls = L - Id, the argument of the Chebyshev polynomials (Sec. 3.5), with its (exactly zero)
    diagonal removed."""
    rp, col, val = L
    n = len(rp) - 1
    row = np.repeat(np.arange(n), np.diff(rp))
    val = val - (row == col).astype(np.float64)
    keep = val != 0.0
    rp2 = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(row[keep], minlength=n), out=rp2[1:])
    return rp2, np.ascontiguousarray(col[keep]), np.ascontiguousarray(val[keep])


def combinatorial_shifted(rowptr, col, A):
    """The combinatorial Laplacian L = D - A of Sec. 3.4 brought to the spectrum [0, 2] that Sec. 3.5
    assumes: L' = (2 / lam) L with lam = 2 max_i D_ii, an upper bound on the largest eigenvalue
    (Gershgorin: every disc of D - A lies in [0, 2 D_ii]).  Since exp(-t L) = exp(-s L') with
    s = t lam / 2, the expansion of Sec. 3.5 at time s in T_k(L' - Id) approximates the heat kernel
    of the combinatorial Laplacian.

    Returns ``((rowptr, col, val), lam)``: the shifted operator L' - Id as CSR with its diagonal
    2 D_ii / lam - 1 stored (columns ascending), and lam.
    """
    rowptr = np.asarray(rowptr, np.int64)
    col = np.asarray(col, np.int32)
    A = np.asarray(A, np.float64)
    n = len(rowptr) - 1
    row = np.repeat(np.arange(n), np.diff(rowptr))
    deg = np.bincount(row, weights=A, minlength=n)
    lam = 2.0 * float(deg.max())
    rows = np.concatenate([row, np.arange(n)])
    cols = np.concatenate([col.astype(np.int64), np.arange(n)])
    vals = np.concatenate([-(2.0 / lam) * A, (2.0 / lam) * deg - 1.0])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    return (rp, cols.astype(np.int32), vals), lam


def heat_apply_combinatorial(rowptr, col, A, t: float, K: int, V):
    """p_K of exp(-t (D - A)) applied to V: the recurrence of Sec. 3.5 on L' - Id at time t lam / 2
    (see ``combinatorial_shifted``)."""
    Ls, lam = combinatorial_shifted(rowptr, col, A)
    return heat_apply(Ls, cheb_coefficients(t * lam / 2.0, K), V)


def build_graph(X, k: int, sigma: float = 0.0):
    """Point cloud -> (Ls, extras): kNN, sigma (median rule when sigma <= 0), A, L, Ls."""
    idx, dist = knn(X, k)
    s = median_sigma(dist) if sigma <= 0 else float(sigma)
    rowptr, col, A = affinity_graph(idx, dist, s)
    deg, L = laplacian(rowptr, col, A)
    return shifted(L), dict(idx=idx, dist=dist, sigma=s, rowptr=rowptr, col=col, A=A, deg=deg, L=L)


# --------------------------------------------------------------------------------------------
# Chebyshev coefficients (Sec. 3.5: "evaluated with the Bessel function")
# --------------------------------------------------------------------------------------------
def cheb_coefficients(t: float, K: int):
    """b_0..b_K of exp(-t L) = b_0/2 + sum_k b_k T_k(L - Id), for spectra in [0, 2].

    With y = L - 1 in [-1, 1], exp(-t (1 + y)) = e^{-t} [I_0(t) + 2 sum_{k>=1} (-1)^k I_k(t) T_k(y)]
    (generating function of the modified Bessel functions I_k), so b_k = 2 (-1)^k e^{-t} I_k(t).
    I_k(t) = sum_m (t/2)^{2m+k} / (m! (m+k)!), summed term by term in log space with the e^{-t}
    factor folded in so that nothing overflows.
    """
    if not (t > 0) or K < 0:
        raise ValueError("cheb_coefficients: need t > 0 and K >= 0")
    lt = math.log(t / 2.0)
    b = np.empty(K + 1)
    for k in range(K + 1):
        terms = []
        m = 0
        peak = -math.inf
        while True:
            lg = (2 * m + k) * lt - math.lgamma(m + 1) - math.lgamma(m + k + 1) - t
            peak = max(peak, lg)
            terms.append(math.exp(lg))
            if m > t and lg < peak - 80.0:
                break
            m += 1
        b[k] = 2.0 * (-1) ** k * math.fsum(terms)
    return b


def cheb_coefficients_quadrature(t: float, K: int, N: int = 256):
    """The same coefficients by Chebyshev-Gauss quadrature of f(y) = exp(-t (1 + y)) on [-1, 1]:
    b_k = (2/N) sum_j f(cos th_j) cos(k th_j), th_j = pi (j + 1/2) / N."""
    th = math.pi * (np.arange(N) + 0.5) / N
    f = np.exp(-t * (1.0 + np.cos(th)))
    return np.array([2.0 / N * math.fsum(f * np.cos(k * th)) for k in range(K + 1)])


# --------------------------------------------------------------------------------------------
# Heat filter p_K(L, t) (Sec. 3.5)
# --------------------------------------------------------------------------------------------
def heat_apply(Ls, b, V):
    """p_K(L, t) V through the three-term recurrence (Sec. 3.5), FP64; V is [n] or [n, B]."""
    rp, col, val = Ls
    V = np.asarray(V, np.float64)
    squeeze = V.ndim == 1
    V2 = np.ascontiguousarray(V.reshape(V.shape[0], -1))
    n, B = V2.shape
    K = len(b) - 1
    b = np.ascontiguousarray(b, np.float64)
    Y = np.empty_like(V2)
    rc = _core().or_cheb_filter(n, _ptr(np.ascontiguousarray(rp, np.int64)),
                                _ptr(np.ascontiguousarray(col, np.int32)),
                                _ptr(np.ascontiguousarray(val, np.float64)), K, _ptr(b), B,
                                _ptr(V2), _ptr(Y))
    if rc != 0:
        raise ValueError("heat_apply: bad arguments")
    return Y[:, 0] if squeeze else Y


def heat_apply_implicit(Ls, t: float, K: int, V):
    """The Euler implicit approximation of H_t (Sec. 4, the remark after the proposition on K): K
    backward Euler steps of the heat equation, (I + (t/K) L)^{-K} V with L = Ls + I, as the dense
    inverse of I + (t/K) L applied K times (small graphs only)."""
    rp, col, val = Ls
    n = len(rp) - 1
    L = np.eye(n)
    row = np.repeat(np.arange(n), np.diff(rp))
    np.add.at(L, (row, np.asarray(col, np.int64)), np.asarray(val, np.float64))
    Minv = np.linalg.inv(np.eye(n) + (t / K) * L)
    Y = np.asarray(V, np.float64)
    for _ in range(K):
        Y = Minv @ Y
    return Y


# --------------------------------------------------------------------------------------------
# Geodesic Sinkhorn (Algorithm 1, Definition 4.1)
# --------------------------------------------------------------------------------------------
def _div0(num, den):
    """num / den elementwise with 0 / anything := 0 (zero mass stays zero)."""
    out = np.zeros(np.broadcast(num, den).shape)
    nz = num != 0
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        out[nz] = (num / den)[nz] if np.ndim(den) else num[nz] / den
    return out


def _xlogy0(x, y):
    """x ln y with 0 ln(anything) := 0."""
    out = np.zeros(np.shape(x))
    nz = x != 0
    with np.errstate(divide="ignore", invalid="ignore"):
        out[nz] = x[nz] * np.log(y[nz])
    return out


def sinkhorn(Ls, b, mu, nu, t: float, iters: int, a=None, eps: float = 0.0):
    """Algorithm 1: w <- 1; repeat { v <- mu / p_K(a * w); w <- nu / p_K(a * v) };
    return 4t sum a * (mu ln v + nu ln w).

    ``a`` are the vertex weights (default 1).  With ``eps > 0`` the loop stops after the first
    iteration j (j a multiple of 10) whose mu-marginal error sum |v * p_K(a * w) - mu| is below
    eps; otherwise exactly ``iters`` iterations run.  Zero mass: mu_i = 0 gives v_i = 0 and
    contributes 0 to the sum.  Returns a dict with v, w, W2 (Algorithm 1's return value, the
    squared distance), W (its square root, Definition 4.1 read as (4t)^{1/2} (...)^{1/2}),
    iters (iterations done) and status (0 ok, 4 non-finite scalings, 5 not converged).
    """
    mu = np.asarray(mu, np.float64)
    nu = np.asarray(nu, np.float64)
    n = len(mu)
    a = np.ones(n) if a is None else np.asarray(a, np.float64)
    w = np.ones(n)
    v = np.zeros(n)
    done = 0
    converged = False
    for j in range(1, iters + 1):
        v = _div0(mu, heat_apply(Ls, b, a * w))
        w = _div0(nu, heat_apply(Ls, b, a * v))
        done = j
        if eps > 0 and j % 10 == 0:
            err = np.abs(v * heat_apply(Ls, b, a * w) - mu).sum()
            if err < eps:
                converged = True
                break
    finite = bool(np.isfinite(v).all() and np.isfinite(w).all()
                  and (v >= 0).all() and (w >= 0).all())
    W2 = 4.0 * t * float(np.sum(a * (_xlogy0(mu, v) + _xlogy0(nu, w)))) if finite else math.nan
    status = OK if finite else NONFINITE
    if finite and eps > 0 and not converged:
        status = NOT_CONVERGED
    W = math.sqrt(W2) if finite and W2 >= 0 else math.nan
    return dict(v=v, w=w, W2=W2, W=W, iters=done, status=status)


def sinkhorn_grad(Ls, b, mu, nu, t: float, iters: int, a=None):
    """Reverse mode of Algorithm 1 unrolled over ``iters`` iterations (fixed count).

    Returns (W2, dW2/dmu, dW2/dnu).  The filter is its own adjoint because p_K(L, t) is a
    polynomial in the symmetric matrix L.  Conventions: where mu_i = 0 the term mu_i ln v_i
    and its derivative are 0 (likewise for nu).
    """
    mu = np.asarray(mu, np.float64)
    nu = np.asarray(nu, np.float64)
    n = len(mu)
    a = np.ones(n) if a is None else np.asarray(a, np.float64)
    H = lambda x: heat_apply(Ls, b, x)  # noqa: E731
    # forward, keeping every denominator and scaling
    w = np.ones(n)
    S, V, R, Wt = [], [], [], []
    for _ in range(iters):
        s = H(a * w)
        v = _div0(mu, s)
        r = H(a * v)
        w = _div0(nu, r)
        S.append(s); V.append(v); R.append(r); Wt.append(w)
    W2 = 4.0 * t * float(np.sum(a * (_xlogy0(mu, v) + _xlogy0(nu, w))))
    # output adjoints
    vbar = 4.0 * t * a * _div0(mu, v)
    wbar = 4.0 * t * a * _div0(nu, w)
    mubar = 4.0 * t * a * np.where(mu != 0, np.log(np.where(v > 0, v, 1.0)), 0.0)
    nubar = 4.0 * t * a * np.where(nu != 0, np.log(np.where(w > 0, w, 1.0)), 0.0)
    for j in range(iters - 1, -1, -1):
        s, v, r, w = S[j], V[j], R[j], Wt[j]
        # w_j = nu / r_j
        nubar = nubar + wbar / r
        rbar = -wbar * w / r
        # r_j = H(a v_j)
        vbar = vbar + a * H(rbar)
        # v_j = mu / s_j
        mubar = mubar + vbar / s
        sbar = -vbar * v / s
        # s_j = H(a w_{j-1})
        wbar = a * H(sbar)
        vbar = np.zeros(n)
    return W2, mubar, nubar


# --------------------------------------------------------------------------------------------
# Fixed-support barycenter (Sec. 3.3; iterative Bregman projections of the cited
# convolutional-Wasserstein paper)
# --------------------------------------------------------------------------------------------
def _alpha_log(alpha, D):
    """alpha_i ln d_i per column, with a zero weight contributing 0 whatever d_i is."""
    out = np.zeros(D.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        for i in range(D.shape[1]):
            if alpha[i] != 0:
                out[:, i] = alpha[i] * np.log(D[:, i])
    return out


def barycenter(Ls, b, M, alpha, iters: int, a=None, return_state: bool = False):
    """Barycenter of the columns mu_i of M [n, m] with weights alpha (Sec. 3.3).

    v_i <- 1; repeat { for each i: w_i <- mu_i / H(a v_i); d_i <- v_i * H(a w_i);
    mu <- prod_i d_i^alpha_i; for each i: v_i <- v_i * mu / d_i }; return mu.
    H is the heat filter p_K(L, t) applied to all m columns at once.  0 / anything := 0.
    """
    M = np.asarray(M, np.float64)
    alpha = np.asarray(alpha, np.float64)
    n, m = M.shape
    a = np.ones(n) if a is None else np.asarray(a, np.float64)
    Vs = np.ones((n, m))
    mu = np.zeros(n)
    H = lambda X: heat_apply(Ls, b, X)  # noqa: E731
    for _ in range(iters):
        Ws = _div0(M, H(a[:, None] * Vs))
        D = Vs * H(a[:, None] * Ws)
        mu = np.exp(np.sum(_alpha_log(alpha, D), axis=1))
        Vs = _div0(Vs * mu[:, None], D)
    if return_state:
        return mu, Vs
    return mu


def barycentric_distance(Ls, b, MT, alphaT, MC, alphaC, t: float, bary_iters: int, sink_iters: int,
                         a=None):
    """Definition 4.3: gamma(T, C) = W_{H_t}(mu*_T, mu*_C), the Geodesic Sinkhorn distance
    (Algorithm 1, ``sink_iters`` iterations) between the barycenters of the families T and C
    (Sec. 3.3, ``bary_iters`` iterations each).  Each barycenter is divided by its mass first: the
    definition compares distributions, and Algorithm 1 needs two marginals of equal mass.
    Returns dict(muT, muC, W2, W, status) with the normalised barycenters."""
    muT = barycenter(Ls, b, MT, alphaT, bary_iters, a=a)
    muC = barycenter(Ls, b, MC, alphaC, bary_iters, a=a)
    muT = muT / muT.sum()
    muC = muC / muC.sum()
    r = sinkhorn(Ls, b, muT, muC, t, sink_iters, a=a)
    return dict(muT=muT, muC=muC, W2=r["W2"], W=r["W"], status=r["status"])


def barycenter_effect(Y, muT, muC):
    """Definition 4.4: tau = E_{mu*_T}[Y] - E_{mu*_C}[Y] for node features Y [n, d], each
    expectation taken under the barycenter divided by its mass (the closed form: two weighted
    means of the features)."""
    Y = np.asarray(Y, np.float64)
    muT = np.asarray(muT, np.float64)
    muC = np.asarray(muC, np.float64)
    return (muT @ Y) / muT.sum() - (muC @ Y) / muC.sum()


def barycenter_grad(Ls, b, M, alpha, iters: int, mubar, a=None):
    """Reverse mode of ``barycenter`` unrolled over ``iters`` iterations: given the adjoint mubar
    of the returned barycenter, returns (mu, d<mubar, mu>/dalpha)."""
    M = np.asarray(M, np.float64)
    alpha = np.asarray(alpha, np.float64)
    n, m = M.shape
    a = np.ones(n) if a is None else np.asarray(a, np.float64)
    aa = a[:, None]
    H = lambda X: heat_apply(Ls, b, X)  # noqa: E731
    Vs = np.ones((n, m))
    tape = []
    mu = np.zeros(n)
    for _ in range(iters):
        S = H(aa * Vs)
        Ws = _div0(M, S)
        R = H(aa * Ws)
        D = Vs * R
        mu = np.exp(np.sum(_alpha_log(alpha, D), axis=1))
        Vn = _div0(Vs * mu[:, None], D)
        tape.append((Vs, S, Ws, R, D, mu, Vn))
        Vs = Vn
    alphabar = np.zeros(m)
    Vbar = np.zeros((n, m))
    Mbar = np.asarray(mubar, np.float64).copy()
    for j in range(iters - 1, -1, -1):
        Vp, S, Ws, R, D, muj, Vn = tape[j]
        # v_i^j = v_i^{j-1} mu^j / d_i
        vpbar = Vbar * muj[:, None] / D
        Mbar = Mbar + np.sum(Vbar * Vp / D, axis=1)
        Dbar = -Vbar * Vn / D
        # mu^j = exp(sum_i alpha_i ln d_i)
        Lbar = Mbar * muj
        alphabar += np.sum(Lbar[:, None] * np.log(D), axis=0)
        Dbar = Dbar + Lbar[:, None] * alpha[None, :] / D
        # d_i = v_i^{j-1} r_i
        vpbar = vpbar + Dbar * R
        Rbar = Dbar * Vp
        # r_i = H(a w_i);  w_i = mu_i / s_i;  s_i = H(a v_i^{j-1})
        Wbar = aa * H(Rbar)
        Sbar = -Wbar * Ws / S
        vpbar = vpbar + aa * H(Sbar)
        Vbar = vpbar
        Mbar = np.zeros(n)
    return mu, alphabar


def barycenter_distance_grad(Ls, b, src, M, alpha, t: float, bary_iters: int, sink_iters: int,
                             a=None):
    """J(src, alpha) = W2(src, mu*(alpha)): the barycenter of M's columns, then Algorithm 1 from
    ``src`` to it.  Returns (J, dJ/dsrc, dJ/dalpha) by reverse mode through both unrolled loops."""
    mu_star = barycenter(Ls, b, M, alpha, bary_iters, a=a)
    J, gsrc, gmu = sinkhorn_grad(Ls, b, src, mu_star, t, sink_iters, a=a)
    _, galpha = barycenter_grad(Ls, b, M, alpha, bary_iters, gmu, a=a)
    return J, gsrc, galpha
