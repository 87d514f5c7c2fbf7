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
