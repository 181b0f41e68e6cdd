"""Adjoint gradients of the CUDA solve (paper_2603_09790_gb300.autograd).

The gradient of L(x(theta)) with A(theta) x = b is -lambda^T (dA/dtheta) x with A lambda = dL/dx.
It is checked against (a) the same formula evaluated densely in FP64 numpy from a direct solve,
and (b) central finite differences of L through the CUDA solver at rtol 1e-13 on 32 random cells.
With both solves at rtol 1e-12 the adjoint gradient is accurate to about rtol * kappa(A)
relative, far inside the 1e-6 used here; the finite differences carry an O(h^2) truncation
(h = 1e-4 on theta of order 1) and are checked at 1e-5.
"""
import numpy as np
import pytest
import torch

from paper_2603_09790_gb300 import autograd as AG
from paper_2603_09790_gb300 import inputs as I
from paper_2603_09790_gb300 import sstep

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def test_pattern_grad_matches_numpy():
    rng = np.random.default_rng(3)
    dims = (9, 7, 6)
    nx, ny, nz = dims
    rp, ci, v = I.q1_csr(dims, np.ones((nz + 1, ny + 1, nx + 1)))
    n = nx * ny * nz
    lam, x = rng.standard_normal(n), rng.standard_normal(n)
    rows = np.repeat(np.arange(n), np.diff(rp))
    want = (-0.75 * lam[rows]) * x[ci]
    g = torch.full((ci.size,), 123.0, dtype=torch.float64, device=DEV)
    RP, CI = torch.from_numpy(rp).to(DEV), torch.from_numpy(ci).to(DEV)
    L, X = torch.from_numpy(lam).to(DEV), torch.from_numpy(x).to(DEV)
    sstep.pattern_grad(RP, CI, L, X, g, scale=0.75)
    assert np.array_equal(g.cpu().numpy(), want)
    sstep.pattern_grad(RP, CI, L, X, g, scale=0.75, accumulate=True)
    assert np.allclose(g.cpu().numpy(), 2 * want, rtol=1e-15, atol=0)


def _problem(dims, seed):
    nx, ny, nz = dims
    theta = np.log(I.lognormal_conductivity((nx + 1, ny + 1, nz + 1), 1.0, 2.0, seed=seed)).reshape(-1)
    b = I.uniform_pm1(seed + 7, nx * ny * nz)
    target = I.uniform_pm1(seed + 11, nx * ny * nz)
    return theta, b, target


def _loss_fn(asm, b, target, opts):
    def f(theta):
        vals = asm.values(torch.exp(theta))
        x = AG.solve(vals, b, asm.pattern, **opts)
        return 0.5 * torch.sum((x - target) ** 2), x
    return f


@pytest.mark.parametrize("precond", ["jacobi", "amg"])
def test_q1_theta_gradient(precond):
    dims = (12, 10, 9)
    theta0, b0, t0 = _problem(dims, 5)
    asm = AG.Q1Assembly(dims, DEV)
    pk = dict(precond=precond, amg_coarse_max=64) if precond == "amg" else {}
    opts = dict(s=4, sweeps=30, rtol=1e-12, **pk)
    b, target = torch.from_numpy(b0).to(DEV), torch.from_numpy(t0).to(DEV)
    theta = torch.from_numpy(theta0).to(DEV).requires_grad_(True)
    f = _loss_fn(asm, b, target, opts)
    loss, x = f(theta)
    loss.backward()
    g = theta.grad.cpu().numpy()

    # (a) dense FP64: x = A^-1 b, lam = A^-1 (x - t), dL/dkappa_c = -sum_t lam_i x_j S_t, * kappa
    rp, ci, sr, sc, sv = I.q1_assembly(dims)
    kappa = np.exp(theta0)
    vals = np.zeros(ci.size)
    np.add.at(vals, sr, sv * kappa[sc])
    n = rp.size - 1
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    A[rows, ci] = vals
    xd = np.linalg.solve(A, b0)
    lam = np.linalg.solve(A, xd - t0)
    gv = -lam[rows] * xd[ci]
    gk = np.zeros(kappa.size)
    np.add.at(gk, sc, sv * gv[sr])
    gd = gk * kappa
    assert np.linalg.norm(x.detach().cpu().numpy() - xd) <= 1e-9 * np.linalg.norm(xd)
    assert np.linalg.norm(g - gd) <= 1e-6 * np.linalg.norm(gd)

    # (b) central differences through the CUDA solver on 32 random cells
    rng = np.random.default_rng(9)
    cells = rng.choice(np.flatnonzero(np.abs(gd) > 1e-3 * np.abs(gd).max()), 32, replace=False)
    fo = _loss_fn(asm, b, target, dict(s=4, sweeps=30, rtol=1e-13, **pk))
    h = 1e-4
    for c in cells:
        tp = torch.from_numpy(theta0).to(DEV)
        tm = tp.clone()
        tp[c] += h
        tm[c] -= h
        with torch.no_grad():
            fd = (fo(tp)[0].item() - fo(tm)[0].item()) / (2 * h)
        assert abs(fd - g[c]) <= 1e-5 * np.abs(gd).max(), (c, fd, g[c])


def test_rhs_gradient_is_adjoint():
    dims = (10, 8, 8)
    theta0, b0, t0 = _problem(dims, 2)
    asm = AG.Q1Assembly(dims, DEV)
    vals = asm.values(torch.exp(torch.from_numpy(theta0).to(DEV)))
    b = torch.from_numpy(b0).to(DEV).requires_grad_(True)
    w = torch.from_numpy(t0).to(DEV)
    x = AG.solve(vals, b, asm.pattern, s=4, sweeps=30, rtol=1e-12)
    torch.sum(w * x).backward()
    # d(w^T A^-1 b)/db = A^-1 w (A symmetric)
    lam = AG.solve(vals, w, asm.pattern, s=4, sweeps=30, rtol=1e-12)
    assert torch.allclose(b.grad, lam, rtol=0, atol=1e-12 * lam.abs().max().item())


def test_update_values_matches_fresh_setup():
    dims = (10, 9, 8)
    theta0, b0, _ = _problem(dims, 4)
    asm = AG.Q1Assembly(dims, DEV)
    v1 = asm.values(torch.exp(torch.from_numpy(theta0).to(DEV)))
    v2 = asm.values(torch.exp(torch.from_numpy(theta0 * 0.5).to(DEV)))
    b = torch.from_numpy(b0).to(DEV)
    A1 = sstep.CSR(asm.pattern.rowptr, asm.pattern.colind, v1)
    A2 = sstep.CSR(asm.pattern.rowptr, asm.pattern.colind, v2)
    with sstep.Solver(A2, s=4, sweeps=3, rtol=1e-10) as S2:
        bi = S2.get_basis_info()
        x2 = torch.zeros_like(b)
        S2.solve(b, x2)
    kw = dict(s=4, sweeps=3, rtol=1e-10, lambda_min=bi["lambda_min"], lambda_max=bi["lambda_max"])
    with sstep.Solver(A2, **kw) as Sf, sstep.Solver(A1, **kw) as Su:
        xf, xu = torch.zeros_like(b), torch.zeros_like(b)
        i1 = Sf.solve(b, xf)
        Su.solve(b, xu)            # captures the handle's graphs with the old values
        xu.zero_()
        Su.update_values(v2)
        i2 = Su.solve(b, xu)
    assert i1.outer_iters == i2.outer_iters
    assert torch.equal(xf, xu)


def test_second_backward_sets_the_handle_up_again():
    dims = (8, 7, 6)
    theta0, b0, t0 = _problem(dims, 6)
    asm = AG.Q1Assembly(dims, DEV)
    theta = torch.from_numpy(theta0).to(DEV).requires_grad_(True)
    b = torch.from_numpy(b0).to(DEV)
    x = AG.solve(asm.values(torch.exp(theta)), b, asm.pattern, s=4, sweeps=30, rtol=1e-12)
    loss = torch.sum(x * x)
    loss.backward(retain_graph=True)
    g1 = theta.grad.clone()
    theta.grad = None
    loss.backward()
    assert torch.allclose(theta.grad, g1, rtol=1e-9, atol=1e-14 * g1.abs().max().item())
