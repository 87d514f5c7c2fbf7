"""The allocation-free heat filter (gs_heat_apply_noalloc) against the FP64 oracle and against the
regular gs_heat_apply.

Some callers cannot allocate device memory: plug-ins whose host application owns every device
allocation, and real-time loops that must never enter the allocator.  They call
gs_heat_apply_noalloc with caller-held CSR arrays; its scratch is a fixed array inside the
library, so n * B is limited to 2^20.  This file is collected last on purpose, so that a run
stopping at the first failure has already run every other test; it also passes alone in a fresh
process.

Tolerance (the heat-filter tolerance of the parity tests): |gpu - ref| <= 1e-4 |ref| + 1e-6 max|ref|.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2211_00805_gb300 import workloads as W
from tests.gpu_common import assert_close, to_dev, to_np

pytestmark = pytest.mark.gpu

RTOL, ATOL_REL = 1e-4, 1e-6
MAX_FLOATS = 2 ** 20  # n * B limit of the fixed scratch array


def _close(a, b, what=""):
    b = np.asarray(b, np.float64)
    assert_close(np.asarray(a, np.float64), b, RTOL, ATOL_REL * np.abs(b).max(), what)


def _oracle_operator(n, d, k, seed):
    """Oracle kNN graph of seeded points; returns the oracle's Ls and the CSR of P the GPU gets
    (P = -Ls, from the FP32-rounded affinities)."""
    X = np.random.default_rng(seed).standard_normal((n, d))
    idx, dist = oracle.knn(X, k)
    # sigma = the largest kNN distance: no affinity of an outlying point underflows in FP32
    rp, col, A = oracle.affinity_graph(idx, dist, float(dist.max()))
    A32 = A.astype(np.float32).astype(np.float64)
    _, L = oracle.laplacian(rp, col, A32)
    Ls = oracle.shifted(L)
    rp_s, col_s, val_s = Ls
    dev = (to_dev(rp_s, torch.int32), to_dev(col_s, torch.int32), to_dev(-val_s, torch.float32))
    return Ls, dev


@pytest.mark.parametrize("B", [1, 6, 32])
def test_noalloc_matches_oracle(B):
    from paper_2211_00805_gb300 import binding as gs
    n = 1500
    Ls, (rp, col, pval) = _oracle_operator(n, 3, 8, seed=40 + B)
    V = np.random.default_rng(B).random((n, B)).astype(np.float32)
    for t, K in [(5.0, 30), (1.0, 20), (2.0, 1)]:
        Y = to_np(gs.gs_heat_apply_noalloc(rp, col, pval, t, K, to_dev(V)))
        ref = oracle.heat_apply(Ls, oracle.cheb_coefficients(t, K), V.astype(np.float64))
        _close(Y, ref, f"B={B} t={t} K={K}")


def test_noalloc_at_the_size_limit_matches_oracle():
    # n * B = 2^20 exactly: the largest block the scratch array holds
    from paper_2211_00805_gb300 import binding as gs
    n, B = 2 ** 15, 32
    assert n * B == MAX_FLOATS
    Ls, (rp, col, pval) = _oracle_operator(n, 3, 10, seed=5)
    V = np.random.default_rng(11).random((n, B)).astype(np.float32)
    t, K = 5.0, 30
    Y = to_np(gs.gs_heat_apply_noalloc(rp, col, pval, t, K, to_dev(V)))
    ref = oracle.heat_apply(Ls, oracle.cheb_coefficients(t, K), V.astype(np.float64))
    _close(Y, ref, "n*B = 2^20")
    with pytest.raises(gs.GeosinkError) as e:  # one column more is rejected before any launch
        gs.gs_heat_apply_noalloc(rp, col, pval, t, K, torch.zeros((n, B + 1), device="cuda"))
    assert e.value.status == gs.GS_ERR_UNSUPPORTED


@pytest.mark.parametrize("B", [32, 6])
def test_noalloc_output_off_a_16_byte_boundary(B):
    # Y starts 4 bytes into its storage: the float4 path must not be taken for it
    from paper_2211_00805_gb300 import binding as gs
    n = 900
    Ls, (rp, col, pval) = _oracle_operator(n, 3, 8, seed=77)
    V = np.random.default_rng(7).random((n, B)).astype(np.float32)
    store = torch.full((n * B + 1,), float("nan"), dtype=torch.float32, device="cuda")
    Yd = store[1:].view(n, B)
    gs.gs_heat_apply_noalloc(rp, col, pval, 3.0, 25, to_dev(V), out=Yd)
    ref = oracle.heat_apply(Ls, oracle.cheb_coefficients(3.0, 25), V.astype(np.float64))
    _close(to_np(Yd), ref, f"offset Y, B={B}")
    assert torch.isnan(store[0]).item()  # nothing written in front of Y


@pytest.mark.parametrize("B", [1, 32])
def test_noalloc_matches_heat_apply_twice(B):
    from paper_2211_00805_gb300 import binding as gs
    ctx = gs.Context()
    p = W.sphere_pair()
    g = gs.gs_build_graph(ctx, torch.from_numpy(p.X).cuda(), p.k)
    rowptr, col, A, P = gs.gs_graph_export_csr(ctx, g)
    rowptr32 = rowptr.to(torch.int32)
    gen = torch.Generator().manual_seed(B)
    for t, K in [(5.0, 30), (1.0, 20)]:  # two calls in a row
        V = torch.rand((g.n, B), generator=gen).cuda()
        ref = gs.gs_heat_apply(ctx, g, t, K, V)
        out = gs.gs_heat_apply_noalloc(rowptr32, col, P, t, K, V)
        torch.cuda.synchronize()
        _close(to_np(out), to_np(ref), f"B={B} t={t} K={K}")
    gs.gs_sync(ctx)


def test_noalloc_leaves_free_device_memory_unchanged():
    # After a first call (address look-up, kernel loading), further calls take no device memory.
    from paper_2211_00805_gb300 import binding as gs
    n, B = 4000, 8
    _, (rp, col, pval) = _oracle_operator(n, 3, 8, seed=3)
    V = torch.rand((n, B), generator=torch.Generator().manual_seed(1)).cuda()
    Y = torch.empty_like(V)
    gs.gs_heat_apply_noalloc(rp, col, pval, 5.0, 30, V, out=Y)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        gs.gs_heat_apply_noalloc(rp, col, pval, 5.0, 30, V, out=Y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_oversized_blocks():
    from paper_2211_00805_gb300 import binding as gs
    n = MAX_FLOATS + 1
    rowptr32 = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    pval = torch.zeros(1, dtype=torch.float32, device="cuda")
    V = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(gs.GeosinkError) as e:
        gs.gs_heat_apply_noalloc(rowptr32, col, pval, 1.0, 5, V)
    assert e.value.status == gs.GS_ERR_UNSUPPORTED


def test_noalloc_wide_blocks_need_aligned_blocks():
    # B > 256 columns are read as float4 only: V and Y must start on 16-byte boundaries
    from paper_2211_00805_gb300 import binding as gs
    n, B = 1000, 260
    Ls, (rp, col, pval) = _oracle_operator(n, 3, 8, seed=9)
    V = np.random.default_rng(4).random((n, B)).astype(np.float32)
    Y = to_np(gs.gs_heat_apply_noalloc(rp, col, pval, 2.0, 15, to_dev(V)))
    ref = oracle.heat_apply(Ls, oracle.cheb_coefficients(2.0, 15), V.astype(np.float64))
    _close(Y, ref, "B = 260")
    Yoff = torch.empty(n * B + 1, dtype=torch.float32, device="cuda")[1:].view(n, B)
    with pytest.raises(gs.GeosinkError) as e:
        gs.gs_heat_apply_noalloc(rp, col, pval, 2.0, 15, to_dev(V), out=Yoff)
    assert e.value.status == gs.GS_ERR_UNSUPPORTED
