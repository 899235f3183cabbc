"""Differentiable multi-RHS solve: torch.autograd.Function over the CUDA library.

Forward: X = A^-1 B with BiCGStab (bicgk_solve).  Backward, for a loss L with
upstream gradient G = dL/dX: the adjoint system A^T Lambda = G is solved with
BiCGStab on the transposed operator (bicgk_op_transpose: A^T's CSR built on the
GPU, then the same SpMM and BiCGStab kernels), then
    dL/dB        = Lambda,
    dL/dA_ij     = -sum_c Lambda_ic X_jc   on the sparsity pattern (bicgk_sddmm),
which follows from dX = -A^-1 (dA) X + A^-1 dB.  Every step runs in the
library's kernels; this module only orders the calls.  Not part of the paper:
a systems extension that leaves the method unchanged.

Operators are cached per sparsity pattern (the rowptr/colidx tensors, held by
the cache so their memory cannot be reused for another pattern while cached):
a call with new values copies them into the cached operator on the device
(bicgk_op_set_values), so the CSR upload, the pattern check, the CUDA-graph
captures and the transposed operator are paid once per pattern.  The pattern
tensors must not be modified in place while cached; clear_cache() drops every
cached operator.
"""
from __future__ import annotations

from collections import OrderedDict

import torch

from . import bicgk

_CACHE_SIZE = 4
_cache: "OrderedDict[tuple, dict]" = OrderedDict()


def clear_cache() -> None:
    """Release every cached operator (and its transposed operator)."""
    while _cache:
        _, ent = _cache.popitem()
        if ent.get("opT") is not None:
            ent["opT"].close()
        ent["op"].close()


def _operator(vals, rowptr, colidx):
    key = (rowptr.device.index, rowptr.data_ptr(), colidx.data_ptr(), rowptr.shape[0], colidx.shape[0])
    ent = _cache.get(key)
    if ent is None:
        ent = {"op": bicgk.Operator(rowptr=rowptr, colidx=colidx, vals=vals), "opT": None,
               "pattern": (rowptr, colidx)}
        _cache[key] = ent
        while len(_cache) > _CACHE_SIZE:
            _, old = _cache.popitem(last=False)
            if old.get("opT") is not None:
                old["opT"].close()
            old["op"].close()
    else:
        _cache.move_to_end(key)
        ent["op"].set_values(vals)
    return ent


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, B, rowptr, colidx, tol, maxit, variant):
        v = vals.detach().contiguous()
        ent = _operator(v, rowptr, colidx)
        r = ent["op"].solve(B.detach().contiguous(), tol=tol, maxit=maxit, variant=variant, want_hist=False)
        if not (r.status == 0).all():
            raise RuntimeError(f"forward solve did not converge: status {r.status.tolist()}")
        ctx.ent = ent
        ctx.tol, ctx.maxit, ctx.variant = tol, maxit, variant
        ctx.save_for_backward(r.X, v)
        return r.X

    @staticmethod
    def backward(ctx, gX):
        X, v = ctx.saved_tensors
        ent = ctx.ent
        op = ent["op"]
        op.set_values(v)              # the values of this forward (the cached operator may have moved on)
        if ent["opT"] is None:
            ent["opT"] = op.transpose()
        else:
            op.transpose_refresh(ent["opT"])
        ra = ent["opT"].solve(gX.contiguous(), tol=ctx.tol, maxit=ctx.maxit, variant=ctx.variant, want_hist=False)
        if not (ra.status == 0).all():
            raise RuntimeError(f"adjoint solve did not converge: status {ra.status.tolist()}")
        lam = ra.X
        dvals = op.sddmm(lam, X, alpha=-1.0) if ctx.needs_input_grad[0] else None
        dB = lam if ctx.needs_input_grad[1] else None
        return dvals, dB, None, None, None, None, None


def solve(vals: torch.Tensor, B: torch.Tensor, rowptr: torch.Tensor, colidx: torch.Tensor, tol: float = 1e-10,
          maxit: int = 5000, variant: str = "classical_merged") -> torch.Tensor:
    """X with A X = B, differentiable in vals (the CSR values, pattern rowptr/colidx) and B.

    All tensors are CUDA: rowptr/colidx int32, vals float64 (nnz), B float64 (n, k).
    """
    return _Solve.apply(vals, B, rowptr, colidx, tol, maxit, variant)
