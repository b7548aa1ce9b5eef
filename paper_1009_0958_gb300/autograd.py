"""The directional filters as a differentiable torch operation.

``DirectionalFilterFn.apply(x, win, filter, p, dist, q, precision)`` filters a
B x 3 x M x N float32 CUDA batch with the library's kernels (by default the
FP32 certified path with its FP64 recheck, which selects what the FP64 path
selects) and saves the selected-member index map; its backward pass scatters the upstream gradient
to the selected source pixels with the library's gather kernel.  Both passes
run on the current CUDA stream.
"""
from __future__ import annotations

import torch

from . import vdf


class DirectionalFilterFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, win=3, filter="ddf", p=0.5, dist="exact", q=4, precision="fp32"):
        y, idx = vdf.filter_f32(x, win, filter, p, dist, q, precision)
        ctx.save_for_backward(idx)
        ctx.win = win
        ctx.mark_non_differentiable(idx)
        return y, idx

    @staticmethod
    def backward(ctx, grad_y, grad_idx=None):
        (idx,) = ctx.saved_tensors
        gx = vdf.backward_f32(grad_y, idx, ctx.win)
        return gx, None, None, None, None, None, None


def directional_filter(x, win=3, filter="ddf", p=0.5, dist="exact", q=4, precision="fp32"):
    """Differentiable filter; returns the filtered batch (the index map is
    kept for the backward pass)."""
    y, _ = DirectionalFilterFn.apply(x, win, filter, p, dist, q, precision)
    return y
