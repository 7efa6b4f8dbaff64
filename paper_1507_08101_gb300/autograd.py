"""y = A x as a differentiable torch operation over the SELL-C-sigma library.

Forward: one sp_spmv call.  Backward: one sp_spmv_adjoint call, which gives
  dL/dx    = A^T g           (the product with the transposed SELL matrix)
  dL/dvals = g_i . x_j       (the sampled product over the pattern, CSR order)
Both are hand-written kernels; this module only marshals tensors.
"""
from __future__ import annotations

import torch

from . import sellcs


class SpMV(torch.autograd.Function):
    """``SpMV.apply(mat, vals, x, values_current)`` with ``vals`` the CSR-order
    values of ``mat`` (float32 or float64, same order as given at creation).
    The matrix values are refreshed from ``vals`` first (sp_mat_update_values,
    a value-only conversion) unless ``values_current`` promises that ``mat``
    already holds exactly ``vals``."""

    @staticmethod
    def forward(ctx, mat: sellcs.SellMatrix, vals: torch.Tensor, x: torch.Tensor, values_current: bool = False):
        if not values_current:
            mat.update_values(vals.detach().contiguous())
        nrows, _ = mat.shape
        shape = (nrows,) if x.dim() == 1 else (nrows, x.shape[1])
        y = torch.empty(shape, dtype=x.dtype, device=x.device)
        xc = x.detach().contiguous()
        sellcs.spmv(mat, xc, y)
        ctx.mat = mat
        ctx.save_for_backward(xc)
        ctx.vals_dtype = vals.dtype
        ctx.nnz = vals.numel()
        return y

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        mat = ctx.mat
        g = g.contiguous()
        dx = torch.empty_like(x) if ctx.needs_input_grad[2] else None
        dvals = None
        if ctx.needs_input_grad[1]:
            dvals = torch.empty(ctx.nnz, dtype=x.dtype, device=x.device)
        if dx is not None or dvals is not None:
            x2 = x if x.dim() == 2 else x[:, None]
            g2 = g if g.dim() == 2 else g[:, None]
            dx2 = None if dx is None else (dx if dx.dim() == 2 else dx[:, None])
            sellcs.spmv_adjoint(mat, g2, x=x2 if dvals is not None else None, dx=dx2, dvals=dvals)
        if dvals is not None and dvals.dtype != ctx.vals_dtype:
            dvals = dvals.to(ctx.vals_dtype)
        return None, dvals, dx, None


def spmv(mat: sellcs.SellMatrix, vals: torch.Tensor, x: torch.Tensor, values_current: bool = False) -> torch.Tensor:
    return SpMV.apply(mat, vals, x, values_current)
