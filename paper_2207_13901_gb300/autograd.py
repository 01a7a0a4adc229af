"""Differentiable SpMM: Y = A X with a hand-written backward.

    forward   Y(i,l)  = A(i,j) X(j,l)                       (spd_spmm)
    backward  dA(i,j) = dY(i,l) X(j,l) on A's pattern only  (spd_sddmm with B = pattern)
              dX(j,l) = A(i,j) dY(i,l)                      (spd_spmm over A^T, or spd_spmm_t)

The gradient with respect to A's values is the sampled dense-dense product of dY and X
on A's sparsity pattern, i.e. SDDMM (Section VI-A) with every B value equal to 1. The
backward computes in A's value type: a binary32 gradient dY is rounded to bfloat16 when
the values are bfloat16.

dX is computed by default over A^T: its structure is formed once per pattern (a stable
sort of A's positions by column, cached on the pattern) and dX is then an ordinary,
deterministic SpMM. ``dx="atomic"`` scatters into dX with atomic adds instead and needs
no transposed structure.
"""
from __future__ import annotations

import torch

from . import ops


class SpMMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, X, pattern, split, tune, dx):
        A = pattern.with_vals(vals)
        Y = ops.spmm(A, X, split=split, tune=tune)
        ctx.save_for_backward(vals, X)
        ctx.pattern = pattern
        ctx.split = split
        ctx.tune = tune
        ctx.dx = dx
        return Y

    @staticmethod
    def backward(ctx, dY):
        vals, X = ctx.saved_tensors
        dY = dY.to(vals.dtype).contiguous()
        dvals = dX = None
        if ctx.needs_input_grad[0]:
            dvals = ops.sddmm(ctx.pattern.with_vals(None), dY, X, split=ctx.split, tune=ctx.tune).to(vals.dtype)
        if ctx.needs_input_grad[1]:
            A = ctx.pattern.with_vals(vals)
            dX = ops.spmm_t(A, dY, split=ctx.split, tune=ctx.tune, method=ctx.dx).to(X.dtype)
        return dvals, dX, None, None, None, None


def spmm(A: "ops.CSR", X: torch.Tensor, split: str = "nnz", tune=None, dx: str = "transpose") -> torch.Tensor:
    """Y = A X, differentiable with respect to A.vals and X. ``dx`` picks how dX is
    formed: "transpose" (deterministic, A^T cached per pattern) or "atomic"."""
    return SpMMFunction.apply(A.vals, X, A.with_vals(None), split, tune, dx)
