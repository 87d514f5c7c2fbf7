"""The rounding model behind the log-domain GPU tolerance (CPU only).

The log-domain loop holds every Chebyshev vector as FP32 mantissas with their own binary
exponents and adds a row's terms in FP32 after aligning them to the row's largest exponent by
exact powers of two.  This numpy model does the same arithmetic (summation order aside) on the
2,000-point sphere pair at t = 1, K = 20, 200 iterations, where FP32 scalings overflow, and checks
it against the FP64 oracle: its error is what the GPU test's bounds (5e-4 on ln u, ln v; 1e-5
relative on W^2) are set against.  It shares nothing with the CUDA library.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2211_00805_gb300 import workloads as W

ZERO = -(1 << 30)  # exponent of a zero entry


def _normalise(s, E):
    m, e = np.frexp(s.astype(np.float32))
    return m.astype(np.float32), np.where(m == 0, ZERO, E + e).astype(np.int64)


def _align(m, e, E):
    # m 2^(e - E) in FP32 (terms more than 2^126 below the largest are dropped)
    d = np.where(m != 0, e - E, -1000)
    return np.where(d < -126, np.float32(0), np.ldexp(m, np.clip(d, -126, 0)).astype(np.float32))


class _Model:
    def __init__(self, Ls, t, K):
        rp, col, val = Ls
        self.n = len(rp) - 1
        self.row = np.repeat(np.arange(self.n), np.diff(rp))
        self.col = np.asarray(col, np.int64)
        self.P = (-np.asarray(val)).astype(np.float32)  # P = -(L - Id), zero diagonal
        b = oracle.cheb_coefficients(t, K)
        c = np.array([b[0] / 2] + [(-1) ** k * b[k] for k in range(1, K + 1)])  # in T_k(P)
        cm, ce = np.frexp(c)
        self.cm, self.ce, self.K = cm.astype(np.float32), ce.astype(np.int64), K

    def _spmv(self, xm, xe, scale, zm=None, ze=None):
        # scale P x - z, row by row aligned to the row's largest exponent
        ej = np.where(xm[self.col] != 0, xe[self.col], ZERO)
        E = np.full(self.n, ZERO, np.int64)
        np.maximum.at(E, self.row, ej)
        if zm is not None:
            E = np.maximum(E, np.where(zm != 0, ze, ZERO))
        terms = (np.float32(scale) * self.P) * _align(xm[self.col], xe[self.col], E[self.row])
        s = np.zeros(self.n, np.float32)
        np.add.at(s, self.row, terms)
        if zm is not None:
            s = (s - _align(zm, ze, E)).astype(np.float32)
        return _normalise(s, E)

    def _axpy(self, ym, ye, k, xm, xe):
        pm = (self.cm[k] * xm).astype(np.float32)
        pe = np.where(xm != 0, xe + self.ce[k], ZERO)
        E = np.maximum(np.where(ym != 0, ye, ZERO), pe)
        return _normalise((_align(ym, ye, E) + _align(pm, pe, E)).astype(np.float32), E)

    def log_apply(self, z):
        """ln p_K(e^z) with every vector in the extended form."""
        f = np.floor(z / math.log(2))
        m0 = np.where(np.isneginf(z), 0, 0.5 * np.exp(z - f * math.log(2))).astype(np.float32)
        e0 = np.where(np.isneginf(z), ZERO, f + 1).astype(np.int64)
        x1 = self._spmv(m0, e0, 1.0)
        ym, ye = self._axpy(np.zeros(self.n, np.float32), np.full(self.n, ZERO), 0, m0, e0)
        ym, ye = self._axpy(ym, ye, 1, *x1)
        xa, xb = (m0, e0), x1
        for k in range(2, self.K + 1):
            xn = self._spmv(xb[0], xb[1], 2.0, xa[0], xa[1])
            ym, ye = self._axpy(ym, ye, k, *xn)
            xa, xb = xb, xn
        return np.log(ym.astype(np.float64)) + ye * math.log(2)


def test_extended_range_model_reaches_the_fp64_oracle_where_fp32_overflows():
    p = W.sphere_pair()
    Ls, _ = oracle.build_graph(p.X.astype(np.float64), p.k)
    t, K, iters = 1.0, 20, 200
    a, b = p.a.astype(np.float64), p.b.astype(np.float64)
    model = _Model(Ls, t, K)
    lu, lv = np.zeros(len(a)), np.zeros(len(a))
    for _ in range(iters):
        lu = np.log(a) - model.log_apply(lv)
        lv = np.log(b) - model.log_apply(lu)
    r = oracle.sinkhorn(Ls, oracle.cheb_coefficients(t, K), a, b, t, iters)
    assert r["status"] == oracle.OK
    assert np.abs(np.log(r["v"])).max() > 150  # e^150 is far outside FP32
    err = max(np.abs(lu - np.log(r["v"])).max(), np.abs(lv - np.log(r["w"])).max())
    assert err < 1e-4  # the GPU test allows 5e-4
    W2 = 4 * t * (a @ lu + b @ lv)
    assert W2 == pytest.approx(r["W2"], rel=1e-6)  # the GPU test allows 1e-5
