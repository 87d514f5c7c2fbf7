"""The allocation-free heat filter (gs_heat_apply_noalloc) against the regular gs_heat_apply.

Callers that cannot allocate device memory (graph-capture regions, host applications that own
all device memory) use gs_heat_apply_noalloc with caller-held CSR arrays; its scratch is a fixed
array inside the library.  This file is collected last on purpose, so that a run stopping at the
first failure has already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_2211_00805_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL, ATOL_REL = 1e-4, 1e-6  # the heat-filter tolerance of the parity tests


def _close(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    assert np.all(np.abs(a - b) <= RTOL * np.abs(b) + ATOL_REL * np.abs(b).max())


@pytest.mark.parametrize("B", [1, 32])
def test_noalloc_matches_heat_apply_twice(B):
    from paper_2211_00805_gb300 import binding as gs
    ctx = gs.Context()
    p = W.sphere_pair()
    g = gs.gs_build_graph(ctx, torch.from_numpy(p.X).cuda(), p.k)
    rowptr, col, A, P = gs.gs_graph_export_csr(ctx, g)
    rowptr32 = rowptr.to(torch.int32)
    gen = torch.Generator().manual_seed(B)
    for call, (t, K) in enumerate([(5.0, 30), (1.0, 20)]):  # two calls in a row
        V = torch.rand((g.n, B), generator=gen).cuda()
        ref = gs.gs_heat_apply(ctx, g, t, K, V)
        out = gs.gs_heat_apply_noalloc(rowptr32, col, P, t, K, V)
        torch.cuda.synchronize()
        _close(out, ref)
    gs.gs_sync(ctx)


def test_noalloc_rejects_oversized_blocks():
    from paper_2211_00805_gb300 import binding as gs
    n = 2 ** 20 + 1
    rowptr32 = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    pval = torch.zeros(1, dtype=torch.float32, device="cuda")
    V = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(gs.GeosinkError) as e:
        gs.gs_heat_apply_noalloc(rowptr32, col, pval, 1.0, 5, V)
    assert e.value.status == gs.GS_ERR_UNSUPPORTED
