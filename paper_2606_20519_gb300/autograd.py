"""torch.autograd wrapper of the projection and its Daleckii-Krein VJP.

Forward calls scs_psd_proj_batched; backward calls scs_psd_proj_vjp, which
recomputes the eigendecomposition from the saved input instead of storing the
eigenvectors (App. E of the paper back-propagates through the
eigendecomposition; recomputing keeps the memory of a batch at the size of
its inputs).
"""
from __future__ import annotations

import torch

from . import _lib


class PsdProjection(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, sides, opts=None):
        offsets, sides_a = _lib.shapes(sides)
        y = _lib.proj_batched(x, sides_a, opts=opts, offsets=offsets)
        ctx.save_for_backward(x)
        ctx.shapes = (offsets, sides_a)
        ctx.opts = opts
        return y

    @staticmethod
    def backward(ctx, gy):
        (x,) = ctx.saved_tensors
        offsets, sides_a = ctx.shapes
        gx = _lib.proj_vjp(x, gy.contiguous(), sides_a, opts=ctx.opts, offsets=offsets)
        return gx, None, None


def psd_project(x, sides, opts=None):
    """Differentiable projection of packed svec cones onto the PSD cone."""
    return PsdProjection.apply(x, sides, opts)
