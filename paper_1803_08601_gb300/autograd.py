"""Autograd for C = A @ B with a fixed CSR pattern, differentiable in the stored
values of A and in B (argument marshalling only; every step runs in the library).

Backward of L(vals, B) with dC = dL/dC:
  dB    = A^T dC            (spmm on the transpose, built once and cached)
  dvals = SDDMM(dC, B)      (dvals[p] = <dC[row(p), :], B[col(p), :]>)
There is no gradient with respect to the pattern.
"""
from __future__ import annotations

import torch

from . import ALG_AUTO_GB300, csr_transpose, gather_values, max_row_length, sddmm, spmm


class CSRMatrix:
    """A CSR pattern on the device (int32 row_ptr [m+1], col_ind [nnz]) with shape (m, k);
    caches its longest row and its transpose."""

    def __init__(self, row_ptr: torch.Tensor, col_ind: torch.Tensor, shape):
        self.row_ptr, self.col_ind = row_ptr, col_ind
        self.m, self.k = int(shape[0]), int(shape[1])
        self.nnz = int(col_ind.numel())
        self._max_row = None
        self._t = None

    @property
    def max_row(self) -> int:
        if self._max_row is None:
            self._max_row = max_row_length(self.row_ptr)
        return self._max_row

    def transpose_pattern(self):
        """(row_ptr_t, col_ind_t, perm, max_row_t) of A^T, built on first use."""
        if self._t is None:
            rpt, cit, perm = csr_transpose(self.row_ptr, self.col_ind, self.k)
            self._t = (rpt, cit, perm, max_row_length(rpt))
        return self._t

    def spmm(self, vals, B, alg=ALG_AUTO_GB300, **kw):
        tuning = dict(kw.pop("tuning", None) or {})
        tuning.setdefault("max_row_len", self.max_row)
        return spmm(self.row_ptr, self.col_ind, vals, B, alg=alg, nnz=self.nnz, tuning=tuning, **kw)

    def spmm_t(self, vals, dC, alg=ALG_AUTO_GB300):
        """A^T @ dC with vals in A's order (gathered into A^T's order on the device)."""
        rpt, cit, perm, max_row_t = self.transpose_pattern()
        vals_t = gather_values(perm, vals)
        return spmm(rpt, cit, vals_t, dC, alg=alg, nnz=self.nnz, tuning={"max_row_len": max_row_t})


class SpMMFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A: CSRMatrix, vals: torch.Tensor, B: torch.Tensor, alg: int = ALG_AUTO_GB300):
        ctx.A, ctx.alg = A, alg
        ctx.save_for_backward(vals, B)
        return A.spmm(vals, B.contiguous(), alg=alg)

    @staticmethod
    def backward(ctx, dC):
        vals, B = ctx.saved_tensors
        A = ctx.A
        dC = dC.contiguous()
        dvals = dB = None
        if ctx.needs_input_grad[1]:
            dvals = sddmm(A.row_ptr, A.col_ind, dC, B.contiguous(), out_dtype=vals.dtype)
        if ctx.needs_input_grad[2]:
            dB = A.spmm_t(vals, dC, alg=ctx.alg)
        return None, dvals, dB, None


def spmm_autograd(A: CSRMatrix, vals: torch.Tensor, B: torch.Tensor, alg: int = ALG_AUTO_GB300):
    return SpMMFunction.apply(A, vals, B, alg)
