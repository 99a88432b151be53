"""torch.autograd wrapper of the projection and its Daleckii-Krein VJP.

App. E of the paper back-propagates through the eigendecomposition.  The
backward pass needs every eigenpair of every cone; the forward pass can
either keep them (scs_psd_proj_store, then scs_psd_vjp_stored: no second
eigensolve, sum n^2 + n extra doubles held until backward) or keep only its
input and recompute them in backward (scs_psd_proj_vjp: memory of a batch
stays at the size of its inputs).  opts.recompute picks: 0 keeps them when
the kept bytes fit opts.mem_budget_bytes (0 = no limit), 1 always
recomputes, 2 always keeps.  Both give bit-identical gradients.
"""
from __future__ import annotations

import torch

from . import _lib


def stores_eigenpairs(sides, opts=None) -> bool:
    """Whether the forward pass keeps the eigendecomposition for backward."""
    recompute = opts.recompute if opts is not None else 0
    if recompute == 1:
        return False
    if recompute == 2:
        return True
    budget = opts.mem_budget_bytes if opts is not None else 0
    nv, nl = _lib.eig_sizes(sides)
    return budget <= 0 or 8 * (nv + nl) <= budget


class PsdProjection(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, sides, opts=None):
        offsets, sides_a = _lib.shapes(sides)
        ctx.shapes = (offsets, sides_a)
        ctx.opts = opts
        ctx.stored = stores_eigenpairs(sides_a, opts)
        if ctx.stored:
            y, V, lam = _lib.proj_store(x, sides_a, opts=opts, offsets=offsets)
            ctx.save_for_backward(V, lam)
        else:
            y = _lib.proj_batched(x, sides_a, opts=opts, offsets=offsets)
            ctx.save_for_backward(x)
        return y

    @staticmethod
    def backward(ctx, gy):
        offsets, sides_a = ctx.shapes
        if ctx.stored:
            V, lam = ctx.saved_tensors
            gx = _lib.vjp_stored(V, lam, gy.contiguous(), sides_a, opts=ctx.opts, offsets=offsets)
        else:
            (x,) = ctx.saved_tensors
            gx = _lib.proj_vjp(x, gy.contiguous(), sides_a, opts=ctx.opts, offsets=offsets)
        return gx, None, None


def psd_project(x, sides, opts=None):
    """Differentiable projection of packed svec cones onto the PSD cone."""
    return PsdProjection.apply(x, sides, opts)
