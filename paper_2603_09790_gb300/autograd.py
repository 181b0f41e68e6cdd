"""Differentiable PCG-S solves as torch.autograd.Functions.

Forward solves with the CUDA library.  Backward recomputes x (no solution is kept between the
two passes; the solver handle is), solves the adjoint system A^T lambda = dL/dx with the same
s-step kernels and handle (A is SPD, so A^T = A), and forms the gradient with the library's
kernels; dL/db = lambda.  Three forms:

* ``solve(vals, b, pattern)``: a CSR operator, differentiable in its stored values:
  dL/dA_ij = -lambda_i x_j on the pattern (sstep_pattern_grad).
* ``q1_solve(theta, b, dims)``: the Q1 diffusion operator with cell log-conductivities theta
  (kappa = exp(theta), sstep_q1_exp): matrix-free with Jacobi, or assembled on the device
  (sstep_q1_assemble) for the AMG preconditioner; dL/dtheta_c = -kappa_c lambda_c^T K_ref x_c
  (sstep_q1_grad).  No arithmetic of the chain runs in torch.
* ``batched_solve(wc, wo, bs, grids)``: a batch of 7-point systems A_i = wc_i I + wo_i N, several
  right-hand sides each, through one batched persistent solve per pass; differentiable in the
  weights (sstep_stencil7_weight_grad) and the right-hand sides.

The paper has no differentiated form; this is the standard adjoint of a linear solve.
"""
from __future__ import annotations

import numpy as np
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


class Q1Pattern:
    """The CSR pattern of the Q1 operator on the nx x ny x nz interior vertices (27-point
    neighbourhood without the face neighbours, whose couplings vanish), on the device."""

    def __init__(self, dims, device):
        from . import inputs
        nx, ny, nz = (int(d) for d in dims)
        rp, ci, _ = inputs.q1_csr((nx, ny, nz), np.ones((nz + 1, ny + 1, nx + 1)))
        self.dims = (nx, ny, nz)
        self.pattern = CSRPattern(torch.from_numpy(rp).to(device), torch.from_numpy(ci).to(device))

    def values(self, kappa, stream=None):
        """CSR values for cell conductivities kappa (device, (nx+1)(ny+1)(nz+1)), assembled by
        sstep_q1_assemble (not differentiable; q1_solve is)."""
        vals = torch.empty(self.pattern.nnz, dtype=torch.float64, device=kappa.device)
        sstep.q1_assemble(self.dims, kappa.detach().contiguous(), self.pattern.rowptr,
                          self.pattern.colind, vals, stream=stream)
        return vals


def _q1_handle(dims, kappa, patt, opts):
    nx, ny, nz = dims
    if opts.get("precond", "jacobi") == "amg":
        vals = patt.values(kappa, stream=opts.get("stream"))
        A = sstep.CSR(patt.pattern.rowptr, patt.pattern.colind, vals)
    else:
        A = sstep.Q1(nx, ny, nz, kappa)
    return sstep.Solver(A, **opts)


class _Q1Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, b, patt, opts):
        kappa = torch.empty_like(theta)
        sstep.q1_exp(theta.detach().contiguous(), kappa, stream=opts.get("stream"))
        S = _q1_handle(patt.dims, kappa, patt, opts)
        try:
            x = _solve(S, b)
        except Exception:
            S.free()
            raise
        ctx.save_for_backward(kappa, b)
        ctx.patt, ctx.opts, ctx.solver = patt, opts, S
        return x

    @staticmethod
    def backward(ctx, gx):
        kappa, b = ctx.saved_tensors
        S = ctx.solver
        ctx.solver = None
        if S is None:  # a second backward through the same graph: set the handle up again
            S = _q1_handle(ctx.patt.dims, kappa, ctx.patt, ctx.opts)
        try:
            x = _solve(S, b)             # x recomputed
            lam = _solve(S, gx)          # A^T lambda = dL/dx (A symmetric)
        finally:
            S.free()
        gtheta = None
        if ctx.needs_input_grad[0]:
            gtheta = torch.empty_like(kappa)
            sstep.q1_grad(ctx.patt.dims, kappa, lam, x, gtheta, wrt_log=True,
                          stream=ctx.opts.get("stream"))
        return gtheta, (lam if ctx.needs_input_grad[1] else None), None, None


def q1_solve(theta, b, patt: Q1Pattern, **opts):
    """x = A(exp(theta))^{-1} b for the Q1 diffusion operator of `patt` (cell log-conductivity
    theta, (nx+1)(ny+1)(nz+1) device doubles), differentiable in theta and b; opts are
    sstep.Solver keywords (precond "jacobi": matrix-free operator; "amg": assembled CSR)."""
    if "stream" not in opts:
        opts = dict(opts, stream=torch.cuda.current_stream(b.device).cuda_stream or None)
    return _Q1Solve.apply(theta, b, patt, opts)


def _batched(S, bs):
    xs = [torch.zeros_like(v) for v in bs]
    infos = S.solve_batched([v.detach().contiguous() for v in bs], xs)
    bad = [i for i, inf in enumerate(infos) if inf.status != sstep.OK]
    if bad:
        raise sstep.SstepError(infos[bad[0]].status, f"batched solve: {len(bad)} problems stopped early")
    return xs


class _BatchedSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, wc, wo, grids, nrhs, opts, *bs):
        ops = [sstep.Stencil(*g, points=7, weights=[o, o, o, c, o, o, o])
               for g, c, o in zip(grids, wc.tolist(), wo.tolist())]
        S = sstep.Solver(ops, **opts)
        try:
            xs = _batched(S, bs)
        except Exception:
            S.free()
            raise
        ctx.save_for_backward(wc, *bs)
        ctx.grids, ctx.nrhs, ctx.opts, ctx.ops, ctx.solver = grids, nrhs, opts, ops, S
        return tuple(xs)

    @staticmethod
    def backward(ctx, *gxs):
        wc, *bs = ctx.saved_tensors
        S = ctx.solver
        ctx.solver = None
        if S is None:
            S = sstep.Solver(ctx.ops, **ctx.opts)
        try:
            xs = _batched(S, bs)                                   # x recomputed
            lams = _batched(S, [g.contiguous() for g in gxs])      # A^T lambda = dL/dx
        finally:
            S.free()
        gw = None
        if ctx.needs_input_grad[0] or ctx.needs_input_grad[1]:
            gw = torch.empty(2 * len(ctx.grids), dtype=torch.float64, device=wc.device)
            sstep.stencil7_weight_grad(ctx.grids, ctx.nrhs, lams, xs, gw,
                                       stream=ctx.opts.get("stream"))
        gwc = gw[0::2] if ctx.needs_input_grad[0] else None
        gwo = gw[1::2] if ctx.needs_input_grad[1] else None
        return (gwc, gwo, None, None, None) + tuple(lams)


def batched_solve(wc, wo, bs, grids, **opts):
    """x_ir = A_i^{-1} b_ir for the 7-point systems A_i = wc_i I + wo_i N on grids[i]
    (N: six-neighbour sum, Dirichlet), nrhs = len(bs) / len(grids) right-hand sides per system
    (system-major), all solved by one batched persistent launch; differentiable in wc, wo
    (device tensors of len(grids)) and every b.  opts: sstep.Solver keywords."""
    nsys = len(grids)
    if len(bs) % nsys:
        raise ValueError("len(bs) must be a multiple of the number of systems")
    if "stream" not in opts:
        opts = dict(opts, stream=torch.cuda.current_stream(bs[0].device).cuda_stream or None)
    return _BatchedSolve.apply(wc, wo, [tuple(int(v) for v in g) for g in grids],
                               len(bs) // nsys, opts, *bs)
