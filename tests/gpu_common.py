"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch


def to_dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dtype, device="cuda")


def to_np(t):
    return t.detach().cpu().numpy()


def report(gpu, ref):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(gpu - ref)
    rel = err / np.maximum(np.abs(ref), 1e-300)
    return float(err.max(initial=0.0)), float(rel.max(initial=0.0))


def assert_close(gpu, ref, rtol, atol=0.0, what="", mask=None):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    if mask is not None:
        gpu, ref = gpu[mask], ref[mask]
    err = np.abs(gpu - ref)
    bound = rtol * np.abs(ref) + atol
    bad = ~(err <= bound)
    if bad.any():
        i = int(np.argmax(np.where(bad, err - bound, -np.inf)))
        raise AssertionError(
            f"{what}: {int(bad.sum())}/{bad.size} entries outside rtol={rtol} atol={atol:g}; "
            f"worst gpu={gpu.flat[i]!r} ref={ref.flat[i]!r} max_abs={err.max():.3e}")


def oracle_csr_to_dev(rowptr, col, A):
    return (to_dev(rowptr, torch.int64), to_dev(col, torch.int32), to_dev(A, torch.float32))


def knn_lists_match(gidx, gdist, ref_idx, ref_dist, X, rows=None):
    """kNN tolerance: the GPU's lists equal the oracle's exactly, except that a neighbour on one
    side only is allowed when its exact FP64 distance (direct differences, computed here from the
    coordinates for a neighbour only the GPU returned) ties the oracle's k-th distance within 1e-6
    relative.  The returned distances, sorted on both sides, agree to FP32 rounding on every row.
    Returns the number of rows whose lists differ."""
    X = np.asarray(X, np.float64)
    gidx = np.asarray(gidx)
    q_ids = np.arange(len(gidx)) if rows is None else np.asarray(rows)
    mism = 0
    for r, q in enumerate(q_ids):
        a, b = gidx[r], ref_idx[r]
        assert len(set(a.tolist())) == len(a) and int(q) not in set(a.tolist()), f"row {q}: self or repeat"
        if np.array_equal(a, b):
            continue
        mism += 1
        dk = ref_dist[r, -1]
        sa, sb = set(a.tolist()), set(b.tolist())
        for j in sa - sb:
            dj = float(np.sqrt(((X[q] - X[j]) ** 2).sum()))
            assert abs(dj - dk) <= 1e-6 * dk, f"row {q}: GPU neighbour {j} at {dj} vs k-th {dk}"
        for j in sb - sa:
            dj = ref_dist[r, int(np.nonzero(b == j)[0][0])]
            assert abs(dj - dk) <= 1e-6 * dk, f"row {q}: oracle neighbour {j} at {dj} vs k-th {dk}"
    if gdist is not None:
        np.testing.assert_allclose(np.asarray(gdist, np.float64), ref_dist, rtol=1e-6)
    return mism
