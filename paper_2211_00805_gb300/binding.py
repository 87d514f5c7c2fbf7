"""Thin ctypes binding of libgeosink.so with the C-ABI's names (argument marshalling only).

Every function takes torch tensors that already live on the GPU, checks dtype / shape /
contiguity, passes raw pointers and sizes to the C entry point of the same name and raises
``GeosinkError`` for a non-OK status.  No arithmetic of the method happens here: all of it runs
in the CUDA kernels of ``csrc/``.  If the shared library is missing this module raises on import;
there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgeosink.so")

STATUS = {0: "GS_OK", 1: "GS_ERR_ARG", 2: "GS_ERR_CUDA", 3: "GS_ERR_OOM", 4: "GS_ERR_NONFINITE",
          5: "GS_ERR_NOT_CONVERGED", 6: "GS_ERR_TIMEOUT", 7: "GS_ERR_UNSUPPORTED"}
GS_OK, GS_ERR_ARG, GS_ERR_CUDA, GS_ERR_OOM, GS_ERR_NONFINITE, GS_ERR_NOT_CONVERGED, \
    GS_ERR_TIMEOUT, GS_ERR_UNSUPPORTED = range(8)

# C-ABI symbols and their argument types (kept in the order of include/geosink.h)
_P, _I, _I64, _D, _F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_float
SIGNATURES = {
    "gs_create": [_P, _I, _P],
    "gs_destroy": [_P],
    "gs_set_stream": [_P, _P],
    "gs_last_error": [_P],
    "gs_sync": [_P],
    "gs_reserve": [_P, _I64],
    "gs_set_option": [_P, _I, _I],
    "gs_get_option": [_P, _I, _P],
    "gs_launch_count": [_P, _P],
    "gs_cheb_coeffs": [_D, _I, _P],
    "gs_sell_step_order": [_P, _I, _P],
    "gs_barycentric_distance": [_P, _P, _P, _I, _P, _P, _I, _P, _P, _D, _I, _I, _I, _P, _P, _P],
    "gs_barycenter_effect": [_P, _P, _I64, _I, _P, _P, _P],
    "gs_heat_apply_implicit": [_P, _P, _D, _I, _P, _I, _P, _D, _I],
    "gs_knn": [_P, _P, _I64, _I, _I, _P, _P],
    "gs_build_graph": [_P, _P, _I64, _I, _I, _F, _P],
    "gs_graph_from_csr": [_P, _I64, _P, _P, _P, _P],
    "gs_graph_info": [_P, _P, _P, _P],
    "gs_graph_layout": [_P, _P, ctypes.c_int],
    "gs_graph_export_csr": [_P, _P, _P, _P, _P, _P],
    "gs_autotune": [_P, _P, _I, _I, _P],
    "gs_autotune_choices": [_P, _P, _I, _I, _P, _I],
    "gs_graph_destroy": [_P],
    "gs_heat_apply": [_P, _P, _D, _I, _P, _I, _P],
    "gs_heat_apply_combinatorial": [_P, _P, _D, _I, _P, _I, _P, _P],
    "gs_heat_apply_noalloc": [_I64, _I64, _P, _P, _P, _D, _I, _P, _I, _P, _P],
    "gs_sinkhorn": [_P, _P, _P, _P, _P, _D, _I, _D, _I, _P, _P, _P, _P],
    "gs_distance": [_P, _P, _P, _P, _P, _D, _I, _D, _I, _P],
    "gs_sinkhorn_log": [_P, _P, _P, _P, _P, _D, _I, _D, _I, _P, _P, _P, _P],
    "gs_barycenter": [_P, _P, _P, _I, _P, _P, _D, _I, _I, _P, _P],
    "gs_sinkhorn_grad": [_P, _P, _P, _P, _P, _D, _I, _I, _I, _P, _P, _P],
    "gs_barycenter_grad": [_P, _P, _P, _I, _P, _P, _D, _I, _I, _I, _P, _P, _P],
    "gs_sinkhorn_batched": [_P, _I, _P, _P, _P, _P, _P, _I, _P, _P, _P],
}


class GeosinkError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run __graft_entry__.build() (nvcc) first")
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name == "gs_last_error" else ctypes.c_int
    return lib


_lib = load_library()


def lib() -> ctypes.CDLL:
    return _lib


# ------------------------------------------------------------------------------- marshalling
def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev(t: torch.Tensor, dtype, name: str, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def _raise(ctx, st):
    if st != GS_OK:
        msg = _lib.gs_last_error(ctx.handle if ctx is not None else None)
        raise GeosinkError(st, msg.decode() if msg else "")


class Context:
    """Owns a gs_ctx bound to a device and a stream (default: torch's current stream)."""

    def __init__(self, device: int | None = None, stream: torch.cuda.Stream | None = None):
        device = torch.cuda.current_device() if device is None else int(device)
        stream = torch.cuda.current_stream(device) if stream is None else stream
        h = ctypes.c_void_p()
        st = _lib.gs_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream))
        if st != GS_OK:
            raise GeosinkError(st, "gs_create failed")
        self.handle = h
        self.device = device
        self.stream = stream

    def set_stream(self, stream: torch.cuda.Stream):
        _raise(self, _lib.gs_set_stream(self.handle, ctypes.c_void_p(stream.cuda_stream)))
        self.stream = stream

    def close(self):
        if getattr(self, "handle", None):
            _lib.gs_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """Owns a gs_graph handle."""

    def __init__(self, handle: ctypes.c_void_p):
        self.handle = handle
        n, nnz, sig = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _lib.gs_graph_info(handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(sig))
        self.n, self.nnz, self.sigma = n.value, nnz.value, sig.value

    def close(self):
        if getattr(self, "handle", None):
            _lib.gs_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------- C-ABI entry points
def gs_sync(ctx: Context):
    _raise(ctx, _lib.gs_sync(ctx.handle))


def gs_reserve(ctx: Context, nbytes: int):
    _raise(ctx, _lib.gs_reserve(ctx.handle, int(nbytes)))


GS_OPT_LOOP = 1
GS_OPT_BARRIER_SELFTEST = 2
GS_OPT_B1_KERNEL = 3
GS_OPT_BLK_KERNEL = 4
GS_OPT_KNN_TENSOR = 5
GS_OPT_PERSIST_SMEM_GRAPH = 6
GS_OPT_PERSIST_SYNC = 7
GS_OPT_PERSIST_BLOCKS = 8
GS_OPT_TAG_WORD = 9
GS_OPT_CHECK_ARGS = 10
GS_OPT_TILE_LANES = 11
GS_OPT_NODE_ORDER = 12
GS_OPT_LOOP_REGS = 13


def gs_set_option(ctx: Context, option: int, value: int):
    _raise(ctx, _lib.gs_set_option(ctx.handle, int(option), int(value)))


def gs_get_option(ctx: Context, option: int) -> int:
    v = ctypes.c_int()
    _raise(ctx, _lib.gs_get_option(ctx.handle, int(option), ctypes.byref(v)))
    return int(v.value)


def gs_launch_count(ctx: Context) -> int:
    c = ctypes.c_int64()
    _raise(ctx, _lib.gs_launch_count(ctx.handle, ctypes.byref(c)))
    return int(c.value)


def gs_cheb_coeffs(t: float, K: int):
    """Host call: list of K+1 FP64 coefficients of exp(-tL) in T_k(P)."""
    buf = (ctypes.c_double * (K + 1))()
    st = _lib.gs_cheb_coeffs(float(t), int(K), buf)
    if st != GS_OK:
        raise GeosinkError(st, "gs_cheb_coeffs")
    return list(buf)


def gs_sell_step_order(idx):
    """Host call: step of every entry of one 32-row slice, given its [W, 32] local cache indices
    (numpy uint16, entry j of row l at [j, l]); returns a [W, 32] uint8 array."""
    import numpy as np
    a = np.ascontiguousarray(idx, dtype=np.uint16)
    if a.ndim != 2 or a.shape[1] != 32:
        raise ValueError("idx must be [W, 32]")
    out = np.empty(a.shape, dtype=np.uint8)
    st = _lib.gs_sell_step_order(a.ctypes.data_as(ctypes.c_void_p), int(a.shape[0]),
                                 out.ctypes.data_as(ctypes.c_void_p))
    if st != GS_OK:
        raise GeosinkError(st, "gs_sell_step_order")
    return out


def gs_knn(ctx: Context, X: torch.Tensor, k: int):
    n, d = X.shape
    _dev(X, torch.float32, "X")
    idx = torch.empty((n, k), dtype=torch.int32, device=X.device)
    dist = torch.empty((n, k), dtype=torch.float32, device=X.device)
    _raise(ctx, _lib.gs_knn(ctx.handle, _ptr(X), n, d, k, _ptr(idx), _ptr(dist)))
    return idx, dist


def gs_build_graph(ctx: Context, X: torch.Tensor, k: int, sigma: float = 0.0) -> Graph:
    n, d = X.shape
    _dev(X, torch.float32, "X")
    h = ctypes.c_void_p()
    _raise(ctx, _lib.gs_build_graph(ctx.handle, _ptr(X), n, d, k, float(sigma), ctypes.byref(h)))
    return Graph(h)


def gs_graph_from_csr(ctx: Context, rowptr: torch.Tensor, col: torch.Tensor, w: torch.Tensor) -> Graph:
    n = rowptr.numel() - 1
    _dev(rowptr, torch.int64, "rowptr")
    _dev(col, torch.int32, "col")
    _dev(w, torch.float32, "w", col.shape)
    h = ctypes.c_void_p()
    _raise(ctx, _lib.gs_graph_from_csr(ctx.handle, n, _ptr(rowptr), _ptr(col), _ptr(w),
                                       ctypes.byref(h)))
    return Graph(h)


def gs_autotune(ctx: Context, g: Graph, B: int, K: int) -> int:
    """Time the order-kernel variants on g for B columns and degree K; returns the chosen one."""
    ch = ctypes.c_int()
    _raise(ctx, _lib.gs_autotune(ctx.handle, g.handle, int(B), int(K), ctypes.byref(ch)))
    return int(ch.value)


AUTOTUNE_FIELDS = ("kernel", "lanes", "columns_per_pass", "loop_mode", "persist_sync", "recorded")


def gs_autotune_choices(ctx: Context, g: Graph, B: int, K: int) -> dict:
    """The autotuner's recorded decision for graphs of g's size and B columns (see the header)."""
    out = (ctypes.c_int * len(AUTOTUNE_FIELDS))()
    _raise(ctx, _lib.gs_autotune_choices(ctx.handle, g.handle, int(B), int(K), out, len(AUTOTUNE_FIELDS)))
    return dict(zip(AUTOTUNE_FIELDS, list(out)))


GRAPH_LAYOUT_FIELDS = ("slices", "sell_entries", "cache_tables", "blocks", "rows_per_block",
                       "max_block_entries", "max_block_distinct", "sum_block_distinct", "max_deps")


def gs_graph_layout(g: Graph) -> dict:
    out = (ctypes.c_int64 * len(GRAPH_LAYOUT_FIELDS))()
    _raise(None, _lib.gs_graph_layout(g.handle, out, len(GRAPH_LAYOUT_FIELDS)))
    return dict(zip(GRAPH_LAYOUT_FIELDS, list(out)))


def gs_graph_export_csr(ctx: Context, g: Graph):
    dev = torch.device("cuda", ctx.device)
    rowptr = torch.empty(g.n + 1, dtype=torch.int64, device=dev)
    col = torch.empty(g.nnz, dtype=torch.int32, device=dev)
    A = torch.empty(g.nnz, dtype=torch.float32, device=dev)
    P = torch.empty(g.nnz, dtype=torch.float32, device=dev)
    _raise(ctx, _lib.gs_graph_export_csr(ctx.handle, g.handle, _ptr(rowptr), _ptr(col), _ptr(A), _ptr(P)))
    return rowptr, col, A, P


def gs_heat_apply(ctx: Context, g: Graph, t: float, K: int, V: torch.Tensor, out: torch.Tensor | None = None):
    squeeze = V.dim() == 1
    V2 = V.reshape(V.shape[0], -1)
    _dev(V2, torch.float32, "V")
    if V2.shape[0] != g.n:
        raise ValueError("V must have n rows")
    Y = torch.empty_like(V2) if out is None else _dev(out, torch.float32, "Y").view(V2.shape)
    _raise(ctx, _lib.gs_heat_apply(ctx.handle, g.handle, float(t), int(K), _ptr(V2), V2.shape[1], _ptr(Y)))
    return Y.view(V.shape) if squeeze else Y


def gs_heat_apply_combinatorial(ctx: Context, g: Graph, t: float, K: int, V: torch.Tensor,
                                out: torch.Tensor | None = None):
    """exp(-t (D - A)) V by the Chebyshev filter on the rescaled combinatorial Laplacian; returns
    (Y, lam) with lam = 2 max_i D_ii, the bound the operator was rescaled by."""
    squeeze = V.dim() == 1
    V2 = V.reshape(V.shape[0], -1)
    _dev(V2, torch.float32, "V")
    if V2.shape[0] != g.n:
        raise ValueError("V must have n rows")
    Y = torch.empty_like(V2) if out is None else _dev(out, torch.float32, "Y").view(V2.shape)
    lam = ctypes.c_double()
    _raise(ctx, _lib.gs_heat_apply_combinatorial(ctx.handle, g.handle, float(t), int(K), _ptr(V2), V2.shape[1],
                                                 _ptr(Y), ctypes.byref(lam)))
    return (Y.view(V.shape) if squeeze else Y), float(lam.value)


def gs_heat_apply_noalloc(rowptr32: torch.Tensor, col: torch.Tensor, pval: torch.Tensor, t: float,
                          K: int, V: torch.Tensor, out: torch.Tensor | None = None,
                          stream: torch.cuda.Stream | None = None):
    """Allocation-free heat filter on caller-held CSR arrays (int32 rowptr); the output buffer
    is allocated here by torch only when ``out`` is None.  The library works on the current
    device, so the call runs with V's device current; every array must live on that device."""
    n = rowptr32.numel() - 1
    _dev(rowptr32, torch.int32, "rowptr32")
    _dev(col, torch.int32, "col")
    _dev(pval, torch.float32, "pval", col.shape)
    squeeze = V.dim() == 1
    V2 = V.reshape(V.shape[0], -1)
    _dev(V2, torch.float32, "V")
    if V2.shape[0] != n:
        raise ValueError("V must have n = rowptr32.numel() - 1 rows")
    Y = torch.empty_like(V2) if out is None else _dev(out, torch.float32, "Y").view(V2.shape)
    for name, x in (("rowptr32", rowptr32), ("col", col), ("pval", pval), ("Y", Y)):
        if x.device != V.device:
            raise ValueError(f"{name} is on {x.device}, V on {V.device}")
    with torch.cuda.device(V.device):
        stream = torch.cuda.current_stream(V.device) if stream is None else stream
        st = _lib.gs_heat_apply_noalloc(n, col.numel(), _ptr(rowptr32), _ptr(col), _ptr(pval), float(t),
                                        int(K), _ptr(V2), V2.shape[1], _ptr(Y),
                                        ctypes.c_void_p(stream.cuda_stream))
    if st != GS_OK:
        raise GeosinkError(st, "gs_heat_apply_noalloc")
    return Y.view(V.shape) if squeeze else Y


def gs_sinkhorn(ctx: Context, g: Graph, a: torch.Tensor, b: torch.Tensor, t: float, K: int,
                iters: int, eps: float = 0.0, vol: torch.Tensor | None = None, u=None, v=None,
                dist=None, iters_done=None):
    """Returns (u, v, dist[2] FP64 = (W^2, W), iters_done[1] int32), all device tensors."""
    n = g.n
    _dev(a, torch.float32, "a", (n,))
    _dev(b, torch.float32, "b", (n,))
    if vol is not None:
        _dev(vol, torch.float32, "vol", (n,))
    dev = a.device
    u = torch.empty(n, dtype=torch.float32, device=dev) if u is None else _dev(u, torch.float32, "u", (n,))
    v = torch.empty(n, dtype=torch.float32, device=dev) if v is None else _dev(v, torch.float32, "v", (n,))
    dist = torch.empty(2, dtype=torch.float64, device=dev) if dist is None else _dev(dist, torch.float64, "dist", (2,))
    iters_done = (torch.empty(1, dtype=torch.int32, device=dev) if iters_done is None
                  else _dev(iters_done, torch.int32, "iters_done", (1,)))
    _raise(ctx, _lib.gs_sinkhorn(ctx.handle, g.handle, _ptr(a), _ptr(b), _ptr(vol), float(t), int(K),
                                 float(eps), int(iters), _ptr(u), _ptr(v), _ptr(dist), _ptr(iters_done)))
    return u, v, dist, iters_done


def gs_sinkhorn_log(ctx: Context, g: Graph, a: torch.Tensor, b: torch.Tensor, t: float, K: int,
                    iters: int, eps: float = 0.0, vol: torch.Tensor | None = None, log_u=None, log_v=None,
                    dist=None, iters_done=None):
    """Algorithm 1 with FP64 potentials; returns (ln u, ln v, dist[2] FP64 = (W^2, W),
    iters_done[1] int32), device tensors."""
    n = g.n
    _dev(a, torch.float32, "a", (n,))
    _dev(b, torch.float32, "b", (n,))
    if vol is not None:
        _dev(vol, torch.float32, "vol", (n,))
    dev = a.device
    log_u = (torch.empty(n, dtype=torch.float64, device=dev) if log_u is None
             else _dev(log_u, torch.float64, "log_u", (n,)))
    log_v = (torch.empty(n, dtype=torch.float64, device=dev) if log_v is None
             else _dev(log_v, torch.float64, "log_v", (n,)))
    dist = torch.empty(2, dtype=torch.float64, device=dev) if dist is None else _dev(dist, torch.float64, "dist", (2,))
    iters_done = (torch.empty(1, dtype=torch.int32, device=dev) if iters_done is None
                  else _dev(iters_done, torch.int32, "iters_done", (1,)))
    _raise(ctx, _lib.gs_sinkhorn_log(ctx.handle, g.handle, _ptr(a), _ptr(b), _ptr(vol), float(t), int(K),
                                     float(eps), int(iters), _ptr(log_u), _ptr(log_v), _ptr(dist),
                                     _ptr(iters_done)))
    return log_u, log_v, dist, iters_done


def gs_distance(ctx: Context, g: Graph, a: torch.Tensor, b: torch.Tensor, t: float, K: int,
                iters: int, eps: float = 0.0, vol: torch.Tensor | None = None, dist=None):
    n = g.n
    _dev(a, torch.float32, "a", (n,))
    _dev(b, torch.float32, "b", (n,))
    if vol is not None:
        _dev(vol, torch.float32, "vol", (n,))
    dist = (torch.empty(2, dtype=torch.float64, device=a.device) if dist is None
            else _dev(dist, torch.float64, "dist", (2,)))
    _raise(ctx, _lib.gs_distance(ctx.handle, g.handle, _ptr(a), _ptr(b), _ptr(vol), float(t), int(K),
                                 float(eps), int(iters), _ptr(dist)))
    return dist


def gs_barycenter(ctx: Context, g: Graph, M: torch.Tensor, alpha: torch.Tensor, t: float, K: int,
                  iters: int, vol: torch.Tensor | None = None, mu=None, v_state=None):
    n, m = M.shape
    _dev(M, torch.float32, "M", (g.n, m))
    _dev(alpha, torch.float64, "alpha", (m,))
    if vol is not None:
        _dev(vol, torch.float32, "vol", (n,))
    mu = torch.empty(n, dtype=torch.float32, device=M.device) if mu is None else _dev(mu, torch.float32, "mu", (n,))
    if v_state is not None:
        _dev(v_state, torch.float32, "v_state", (n, m))
    _raise(ctx, _lib.gs_barycenter(ctx.handle, g.handle, _ptr(M), m, _ptr(alpha), _ptr(vol), float(t),
                                   int(K), int(iters), _ptr(mu), _ptr(v_state)))
    return mu


def gs_heat_apply_implicit(ctx: Context, g: Graph, t: float, K: int, V: torch.Tensor, tol: float = 1e-7,
                           iters: int = 30, out: torch.Tensor | None = None):
    """Euler implicit kernel (I + (t/K) L)^{-K} V by K conjugate-gradient solves; V is [n] or [n, B]."""
    B = 1 if V.dim() == 1 else V.shape[1]
    _dev(V, torch.float32, "V", (g.n,) if V.dim() == 1 else (g.n, B))
    Y = torch.empty_like(V) if out is None else out
    _raise(ctx, _lib.gs_heat_apply_implicit(ctx.handle, g.handle, float(t), int(K), _ptr(V), int(B), _ptr(Y),
                                            float(tol), int(iters)))
    return Y


def gs_barycentric_distance(ctx: Context, g: Graph, MT: torch.Tensor, alphaT: torch.Tensor,
                            MC: torch.Tensor, alphaC: torch.Tensor, t: float, K: int, bary_iters: int,
                            sink_iters: int, vol: torch.Tensor | None = None):
    """Definition 4.3: returns (dist[2] FP64 = (gamma^2, gamma), muT, muC) as device tensors, the
    normalised barycenters of the two families included."""
    n = g.n
    mT, mC = MT.shape[1], MC.shape[1]
    _dev(MT, torch.float32, "MT", (n, mT))
    _dev(MC, torch.float32, "MC", (n, mC))
    _dev(alphaT, torch.float64, "alphaT", (mT,))
    _dev(alphaC, torch.float64, "alphaC", (mC,))
    if vol is not None:
        _dev(vol, torch.float32, "vol", (n,))
    muT = torch.empty(n, dtype=torch.float32, device=MT.device)
    muC = torch.empty(n, dtype=torch.float32, device=MT.device)
    dist = torch.empty(2, dtype=torch.float64, device=MT.device)
    _raise(ctx, _lib.gs_barycentric_distance(ctx.handle, g.handle, _ptr(MT), mT, _ptr(alphaT), _ptr(MC), mC,
                                             _ptr(alphaC), _ptr(vol), float(t), int(K), int(bary_iters),
                                             int(sink_iters), _ptr(muT), _ptr(muC), _ptr(dist)))
    return dist, muT, muC


def gs_barycenter_effect(ctx: Context, Y: torch.Tensor, muT: torch.Tensor, muC: torch.Tensor):
    """Definition 4.4: [d] FP64 device tensor E_muT[Y] - E_muC[Y]."""
    n, d = Y.shape
    _dev(Y, torch.float32, "Y", (n, d))
    _dev(muT, torch.float32, "muT", (n,))
    _dev(muC, torch.float32, "muC", (n,))
    out = torch.empty(d, dtype=torch.float64, device=Y.device)
    _raise(ctx, _lib.gs_barycenter_effect(ctx.handle, _ptr(Y), int(n), int(d), _ptr(muT), _ptr(muC), _ptr(out)))
    return out


def gs_sinkhorn_grad(ctx: Context, g: Graph, a: torch.Tensor, b: torch.Tensor, t: float, K: int,
                     iters: int, checkpoint: int = 20, vol: torch.Tensor | None = None):
    """Returns (dist[2] FP64 = (W^2, W), dW^2/da, dW^2/db) as device tensors."""
    n = g.n
    _dev(a, torch.float32, "a", (n,))
    _dev(b, torch.float32, "b", (n,))
    if vol is not None:
        _dev(vol, torch.float32, "vol", (n,))
    dist = torch.empty(2, dtype=torch.float64, device=a.device)
    ga = torch.empty(n, dtype=torch.float32, device=a.device)
    gb = torch.empty(n, dtype=torch.float32, device=a.device)
    _raise(ctx, _lib.gs_sinkhorn_grad(ctx.handle, g.handle, _ptr(a), _ptr(b), _ptr(vol), float(t),
                                      int(K), int(iters), int(checkpoint), _ptr(dist), _ptr(ga),
                                      _ptr(gb)))
    return dist, ga, gb


def gs_barycenter_grad(ctx: Context, g: Graph, M: torch.Tensor, alpha: torch.Tensor, t: float,
                       K: int, iters: int, mubar: torch.Tensor, checkpoint: int = 20,
                       vol: torch.Tensor | None = None):
    """Returns (mu [n], d<mubar, mu>/dalpha [m] FP64) as device tensors."""
    n, m = M.shape
    _dev(M, torch.float32, "M", (g.n, m))
    _dev(alpha, torch.float64, "alpha", (m,))
    _dev(mubar, torch.float32, "mubar", (n,))
    if vol is not None:
        _dev(vol, torch.float32, "vol", (n,))
    mu = torch.empty(n, dtype=torch.float32, device=M.device)
    galpha = torch.empty(m, dtype=torch.float64, device=M.device)
    _raise(ctx, _lib.gs_barycenter_grad(ctx.handle, g.handle, _ptr(M), m, _ptr(alpha), _ptr(vol),
                                        float(t), int(K), int(iters), int(checkpoint), _ptr(mubar),
                                        _ptr(mu), _ptr(galpha)))
    return mu, galpha


def gs_sinkhorn_batched(ctx: Context, graphs, a_list, b_list, t_list, K_list, iters: int,
                        u_list=None, v_list=None, dist=None):
    """Many problems in one launch.  Returns (u_list, v_list, dist [nprob, 2] FP64)."""
    nprob = len(graphs)
    dev = torch.device("cuda", ctx.device)
    for i, (g, a, b) in enumerate(zip(graphs, a_list, b_list)):
        _dev(a, torch.float32, f"a[{i}]", (g.n,))
        _dev(b, torch.float32, f"b[{i}]", (g.n,))
    u_list = [torch.empty(g.n, dtype=torch.float32, device=dev) for g in graphs] if u_list is None else u_list
    v_list = [torch.empty(g.n, dtype=torch.float32, device=dev) for g in graphs] if v_list is None else v_list
    dist = torch.empty((nprob, 2), dtype=torch.float64, device=dev) if dist is None else dist
    P = ctypes.c_void_p * nprob
    hg = P(*[g.handle.value for g in graphs])
    ha = P(*[x.data_ptr() for x in a_list])
    hb = P(*[x.data_ptr() for x in b_list])
    hu = P(*[x.data_ptr() for x in u_list])
    hv = P(*[x.data_ptr() for x in v_list])
    ht = (ctypes.c_double * nprob)(*[float(x) for x in t_list])
    hk = (ctypes.c_int * nprob)(*[int(x) for x in K_list])
    _raise(ctx, _lib.gs_sinkhorn_batched(ctx.handle, nprob, hg, ha, hb, ht, hk, int(iters), hu, hv,
                                         _ptr(dist)))
    return u_list, v_list, dist
