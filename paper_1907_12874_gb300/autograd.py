"""Differentiable multi-RHS solve: torch.autograd.Function over the CUDA library.

Forward: X = A^-1 B with BiCGStab (bicgk_solve).  Backward, for a loss L with
upstream gradient G = dL/dX: the adjoint system A^T Lambda = G is solved with
BiCGStab on the transposed operator (bicgk_op_transpose: the SpMM kernel over a
transposed CSR copy), then
    dL/dB        = Lambda,
    dL/dA_ij     = -sum_c Lambda_ic X_jc   on the sparsity pattern (bicgk_sddmm),
which follows from dX = -A^-1 (dA) X + A^-1 dB.  Every step runs in the
library's kernels; this module only orders the calls.  Not part of the paper:
a systems extension that leaves the method unchanged.
"""
from __future__ import annotations

import torch

from . import bicgk


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, B, rowptr, colidx, tol, maxit, variant):
        op = bicgk.Operator(rowptr=rowptr, colidx=colidx, vals=vals.detach().contiguous())
        r = op.solve(B.detach().contiguous(), tol=tol, maxit=maxit, variant=variant, want_hist=False)
        if not (r.status == 0).all():
            raise RuntimeError(f"forward solve did not converge: status {r.status.tolist()}")
        ctx.op = op
        ctx.tol, ctx.maxit, ctx.variant = tol, maxit, variant
        ctx.save_for_backward(r.X)
        return r.X

    @staticmethod
    def backward(ctx, gX):
        (X,) = ctx.saved_tensors
        op = ctx.op
        opT = op.transpose()
        try:
            ra = opT.solve(gX.contiguous(), tol=ctx.tol, maxit=ctx.maxit, variant=ctx.variant, want_hist=False)
            if not (ra.status == 0).all():
                raise RuntimeError(f"adjoint solve did not converge: status {ra.status.tolist()}")
            lam = ra.X
            dvals = op.sddmm(lam, X, alpha=-1.0) if ctx.needs_input_grad[0] else None
        finally:
            opT.close()
        op.close()
        dB = lam if ctx.needs_input_grad[1] else None
        return dvals, dB, None, None, None, None, None


def solve(vals: torch.Tensor, B: torch.Tensor, rowptr: torch.Tensor, colidx: torch.Tensor, tol: float = 1e-10,
          maxit: int = 5000, variant: str = "classical_merged") -> torch.Tensor:
    """X with A X = B, differentiable in vals (the CSR values, pattern rowptr/colidx) and B.

    All tensors are CUDA: rowptr/colidx int32, vals float64 (nnz), B float64 (n, k).
    """
    return _Solve.apply(vals, B, rowptr, colidx, tol, maxit, variant)
