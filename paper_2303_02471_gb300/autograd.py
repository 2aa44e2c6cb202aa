"""Differentiable sparse products on fixed patterns (torch.autograd).

Gradients are taken with respect to the stored values of A and B; the
patterns are fixed.  Forward and backward both run in libspgemm.so:
spgemm_symbolic + spgemm_numeric for C = A B, spgemm_backward for
dA = (dC B^T) on pattern(A) and dB = (A^T dC) on pattern(B) (masked products
that reuse the forward's column bins), spg_csc_transpose / spg_permute_values
for M^T.  The paper (arXiv 2303.02471) has no backward; these are the
derivatives of C_ij = sum_k A_ik B_kj.

:func:`galerkin` builds the coarse operator P^T (A P) of an aggregation
prolongation P, differentiable in the values of P (and of A).
"""
from __future__ import annotations

from typing import Optional

import torch

from . import _native as N
from . import ops
from .ops import Config, CscMatrix


class _SpGEMM(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a_values, b_values, A: CscMatrix, B: CscMatrix, config, holder):
        Av = A.with_values(a_values.detach().contiguous())
        Bv = B.with_values(b_values.detach().contiguous())
        C, plan = ops.spgemm(Av, Bv, config)
        ctx.plan, ctx.A, ctx.B, ctx.C = plan, Av, Bv, C
        holder.append(C)
        return C.values

    @staticmethod
    def backward(ctx, dc):
        need_a, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        dA, dB = ops.spgemm_backward(ctx.plan, ctx.A, ctx.B, ctx.C, dc.contiguous(), need_a, need_b)
        return dA, dB, None, None, None, None


def spgemm(A: CscMatrix, B: CscMatrix, config: Optional[Config] = None) -> CscMatrix:
    """C = A B with C.values differentiable w.r.t. A.values and B.values."""
    holder = []
    vals = _SpGEMM.apply(A.values, B.values, A, B, config, holder)
    C = holder[0]
    return CscMatrix(C.nrows, C.ncols, C.colptr, C.rowidx, vals)


def _permute(src: torch.Tensor, idx: torch.Tensor, scatter: bool) -> torch.Tensor:
    out = torch.empty_like(src)
    dt = {torch.float64: N.SPG_F64, torch.float32: N.SPG_F32}[src.dtype]
    N.check(N.lib().spg_permute_values(ops._ptr(src.contiguous()), ops._ptr(idx), ops._ptr(out),
                                       src.numel(), dt, int(scatter), ops._stream()),
            "spg_permute_values")
    return out


class _Permute(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, perm):
        ctx.save_for_backward(perm)
        return _permute(values, perm, scatter=False)

    @staticmethod
    def backward(ctx, g):
        (perm,) = ctx.saved_tensors
        return _permute(g.contiguous(), perm, scatter=True), None


def transpose(M: CscMatrix) -> CscMatrix:
    """M^T with values differentiable w.r.t. M.values (a permutation)."""
    T, perm = ops.csc_transpose(M.with_values(None), with_perm=True)
    return CscMatrix(T.nrows, T.ncols, T.colptr, T.rowidx, _Permute.apply(M.values, perm))


def galerkin(A: CscMatrix, P: CscMatrix, config: Optional[Config] = None) -> CscMatrix:
    """C = P^T (A P); differentiable w.r.t. P.values (and A.values)."""
    M = spgemm(A, P, config)
    return spgemm(transpose(P), M, config)
