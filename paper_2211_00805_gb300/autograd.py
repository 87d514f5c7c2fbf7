"""torch.autograd.Function wrappers over the C ABI's forward and hand-written reverse sweeps.

``geodesic_sinkhorn_distance(ctx, g, a, b, ...)`` returns W^2 (Algorithm 1's value) as a 0-d FP64
tensor whose backward gives dW^2/da and dW^2/db; ``geodesic_barycenter(ctx, g, M, alpha, ...)``
returns the barycenter (Sec. 3.3) with a backward for alpha.  Both backwards call the library's
reverse-mode kernels (gs_sinkhorn_grad / gs_barycenter_grad), which re-run the forward loop with
checkpoints every ``checkpoint`` iterations and sweep back with the same fused filter (the heat
filter is its own adjoint).  No arithmetic of the method runs in Python.
"""
from __future__ import annotations

import torch

from . import binding as gs


class _SinkhornDistance(torch.autograd.Function):
    @staticmethod
    def forward(fctx, a, b, ctx, g, t, K, iters, checkpoint, vol):
        dist = gs.gs_distance(ctx, g, a.detach().contiguous(), b.detach().contiguous(), t, K, iters, vol=vol)
        fctx.save_for_backward(a.detach(), b.detach())
        fctx.args = (ctx, g, t, K, iters, checkpoint, vol)
        return dist[0].clone()

    @staticmethod
    def backward(fctx, gout):
        a, b = fctx.saved_tensors
        ctx, g, t, K, iters, checkpoint, vol = fctx.args
        _, ga, gb = gs.gs_sinkhorn_grad(ctx, g, a.contiguous(), b.contiguous(), t, K, iters,
                                        checkpoint=checkpoint, vol=vol)
        scale = gout.to(torch.float32)
        return (ga * scale if fctx.needs_input_grad[0] else None,
                gb * scale if fctx.needs_input_grad[1] else None,
                None, None, None, None, None, None, None)


class _Barycenter(torch.autograd.Function):
    @staticmethod
    def forward(fctx, alpha, M, ctx, g, t, K, iters, checkpoint, vol):
        mu = gs.gs_barycenter(ctx, g, M.detach().contiguous(), alpha.detach().contiguous(), t, K,
                              iters, vol=vol)
        fctx.save_for_backward(alpha.detach(), M.detach())
        fctx.args = (ctx, g, t, K, iters, checkpoint, vol)
        return mu

    @staticmethod
    def backward(fctx, mubar):
        alpha, M = fctx.saved_tensors
        ctx, g, t, K, iters, checkpoint, vol = fctx.args
        _, galpha = gs.gs_barycenter_grad(ctx, g, M.contiguous(), alpha.contiguous(), t, K, iters,
                                          mubar.detach().to(torch.float32).contiguous(),
                                          checkpoint=checkpoint, vol=vol)
        return galpha, None, None, None, None, None, None, None, None


def geodesic_sinkhorn_distance(ctx, g, a, b, t, K, iters, checkpoint=20, vol=None):
    """W^2 between marginals a and b on graph g (differentiable in a and b)."""
    return _SinkhornDistance.apply(a, b, ctx, g, t, K, iters, checkpoint, vol)


def geodesic_barycenter(ctx, g, M, alpha, t, K, iters, checkpoint=20, vol=None):
    """Barycenter of M's columns with weights alpha (FP64, differentiable in alpha)."""
    return _Barycenter.apply(alpha, M, ctx, g, t, K, iters, checkpoint, vol)
