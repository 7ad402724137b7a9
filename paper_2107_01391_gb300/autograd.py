"""Differentiable stable sort along the last dimension.

``RSSortFunction.apply(x)`` returns (sorted values, stable permutation) for a
float32/float64 CUDA tensor.  Forward: one ``rs_sort_segmented`` launch with
every row a segment and the argsort payload (the within-row index of each
sorted key).  Backward: the ``rs_scatter_rows`` kernel sends the upstream
gradient back through the permutation, grad_x[r, perm[r, j]] = g[r, j] --
sorting is a permutation, so its Jacobian is a permutation matrix.  Both are
hand-written CUDA kernels behind the C ABI; torch only allocates.
"""
from __future__ import annotations

import torch

from . import binding


class RSSortFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x: torch.Tensor):
        if x.dtype not in (torch.float32, torch.float64) or not x.is_cuda:
            raise TypeError("RSSortFunction sorts float32/float64 CUDA tensors")
        shape = x.shape
        cols = shape[-1] if x.dim() else 1
        rows = x.numel() // max(cols, 1)
        flat = x.contiguous().reshape(-1)
        if flat.numel() == 0:
            values, perm = flat.clone(), torch.empty(0, dtype=torch.int64, device=x.device)
        else:
            values, perm = binding.rs_sort_segmented(flat, None, num_segs=rows, argsort=True,
                                                     index_dtype=torch.int64)
        values, perm = values.view(shape), perm.view(shape)
        ctx.save_for_backward(perm)
        ctx.mark_non_differentiable(perm)
        return values, perm

    @staticmethod
    def backward(ctx, grad_values, grad_perm):
        (perm,) = ctx.saved_tensors
        if grad_values is None:
            return None
        shape = perm.shape
        cols = shape[-1] if perm.dim() else 1
        g = grad_values.contiguous().reshape(-1, max(cols, 1))
        if g.numel() == 0:
            return grad_values.clone()
        out = binding.rs_scatter_rows(g, perm.reshape(-1, max(cols, 1)))
        return out.view(shape)


def sort(x: torch.Tensor):
    """Stable ascending sort of the last dimension with gradients:
    returns (values, indices) like ``torch.sort(x, stable=True)``."""
    return RSSortFunction.apply(x)
