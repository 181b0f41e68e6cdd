"""Differentiable PCG-S solves: x = A(vals)^{-1} b as a torch.autograd.Function.

Forward solves with the CUDA library.  Backward recomputes x (no solution is kept between the
two passes; the solver handle is), solves the adjoint system A^T lambda = dL/dx with the same
s-step kernels and handle (A is SPD, so A^T = A), and forms
dL/dA_ij = -lambda_i x_j on A's stored pattern with sstep_pattern_grad; dL/db = lambda.
The paper has no differentiated form; this is the standard adjoint of a linear solve.
"""
from __future__ import annotations

import torch

from . import sstep


class CSRPattern:
    """Fixed sparsity pattern: device tensors rowptr (int64, n+1) and colind (int32, nnz)."""

    def __init__(self, rowptr, colind):
        self.rowptr = rowptr.contiguous()
        self.colind = colind.contiguous()
        self.n = int(rowptr.shape[0]) - 1
        self.nnz = int(colind.shape[0])


def _solve(S, rhs):
    out = torch.zeros_like(rhs)
    info = S.solve(rhs.detach().contiguous(), out)
    if info.status != sstep.OK:
        raise sstep.SstepError(info.status, f"solve stopped with relres {info.relres:.3e}")
    return out


class _SStepSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vals, b, pattern, opts):
        A = sstep.CSR(pattern.rowptr, pattern.colind, vals.detach().contiguous())
        S = sstep.Solver(A, **opts)
        try:
            x = _solve(S, b)
        except Exception:
            S.free()
            raise
        ctx.save_for_backward(vals, b)
        ctx.pattern = pattern
        ctx.opts = opts
        # the handle (operator copy, preconditioner set-up, Chebyshev interval) is kept for the
        # backward pass; x itself is not kept and is recomputed there
        ctx.solver = S
        return x

    @staticmethod
    def backward(ctx, gx):
        vals, b = ctx.saved_tensors
        pattern = ctx.pattern
        S = ctx.solver
        ctx.solver = None
        if S is None:  # a second backward through the same graph: set the handle up again
            A = sstep.CSR(pattern.rowptr, pattern.colind, vals.detach().contiguous())
            S = sstep.Solver(A, **ctx.opts)
        try:
            x = _solve(S, b)             # x recomputed
            lam = _solve(S, gx)          # A^T lambda = dL/dx (A symmetric)
        finally:
            S.free()
        gvals = None
        if ctx.needs_input_grad[0]:
            gvals = torch.empty_like(vals)
            sstep.pattern_grad(pattern.rowptr, pattern.colind, lam, x, gvals,
                               stream=ctx.opts.get("stream"))
        return gvals, (lam if ctx.needs_input_grad[1] else None), None, None


def solve(vals, b, pattern: CSRPattern, **opts):
    """x = A^{-1} b with A = CSR(pattern, vals), differentiable in vals and b; opts are
    sstep.Solver keywords (s, sweeps, rtol, precond, ...).  The solves are ordered on torch's
    current stream unless opts names another."""
    if "stream" not in opts:
        opts = dict(opts, stream=torch.cuda.current_stream(b.device).cuda_stream or None)
    return _SStepSolve.apply(vals, b, pattern, opts)


class Q1Assembly:
    """vals = S kappa: the Q1 finite-element operator's CSR values as a linear map of the
    per-cell conductivities, applied with index_add on the device so that gradients reach the
    conductivity field (and through kappa = exp(theta), the log-conductivity)."""

    def __init__(self, dims, device):
        from . import inputs
        rp, ci, sr, sc, sv = inputs.q1_assembly(dims)
        self.pattern = CSRPattern(torch.from_numpy(rp).to(device), torch.from_numpy(ci).to(device))
        self.rows = torch.from_numpy(sr).to(device)
        self.cells = torch.from_numpy(sc).to(device)
        self.coef = torch.from_numpy(sv).to(device)

    def values(self, kappa_flat):
        out = torch.zeros(self.pattern.nnz, dtype=kappa_flat.dtype, device=kappa_flat.device)
        return out.index_add(0, self.rows, self.coef * kappa_flat[self.cells])
