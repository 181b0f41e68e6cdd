"""Adjoint gradients of the CUDA solve (paper_2603_09790_gb300.autograd) and the kernels behind
them (sstep_pattern_grad, sstep_q1_exp / q1_assemble / q1_grad, sstep_stencil7_weight_grad).

The gradient of L(x(theta)) with A(theta) x = b is -lambda^T (dA/dtheta) x with A lambda = dL/dx.
It is checked against (a) the same formula evaluated densely in FP64 numpy from a direct solve,
and (b) central finite differences of L through the CUDA solver at rtol 1e-13 on 32 random cells.
With both solves at rtol 1e-12 the adjoint gradient is accurate to about rtol * kappa(A)
relative, far inside the 1e-6 used here; the finite differences carry an O(h^2) truncation
(h = 1e-4 on theta of order 1) and are checked at 1e-5.  The assembly kernel reproduces the
input generator's values bit for bit (same products, same order of the cell sums).
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_q1_exp_and_assemble_match_generator():
    dims = (13, 11, 7)
    nx, ny, nz = dims
    theta0, _, _ = _problem(dims, 3)
    kappa = torch.empty(theta0.size, dtype=torch.float64, device=DEV)
    sstep.q1_exp(dev(theta0), kappa)
    assert torch.allclose(kappa, dev(np.exp(theta0)), rtol=2e-16, atol=0)
    k_np = kappa.cpu().numpy()
    rp, ci, v = I.q1_csr(dims, k_np.reshape(nz + 1, ny + 1, nx + 1))
    patt = AG.Q1Pattern(dims, DEV)
    assert np.array_equal(patt.pattern.rowptr.cpu().numpy(), rp)
    got = patt.values(kappa).cpu().numpy()
    assert np.array_equal(got, v)


def test_q1_assemble_rejects_foreign_pattern():
    dims = (5, 4, 3)
    patt = AG.Q1Pattern(dims, DEV)
    ci = patt.pattern.colind.clone()
    ci[7] = 59  # an entry of row 1, vertex (1, 0, 0); column 59 is vertex (4, 3, 2)
    kappa = torch.ones((6 * 5 * 4,), dtype=torch.float64, device=DEV)
    vals = torch.empty(ci.numel(), dtype=torch.float64, device=DEV)
    with pytest.raises(sstep.SstepError) as e:
        sstep.q1_assemble(dims, kappa, patt.pattern.rowptr, ci, vals)
    assert e.value.status == sstep.ERR_INVALID


def test_q1_grad_is_the_assembly_transpose():
    """q1_grad = -S^T (lambda_i x_j on the pattern), with S the generator's linear map from the
    cell conductivities to the CSR values (sum over its triplets)."""
    dims = (9, 8, 6)
    theta0, _, _ = _problem(dims, 8)
    rng = np.random.default_rng(4)
    n = 9 * 8 * 6
    lam, x = rng.standard_normal(n), rng.standard_normal(n)
    rp, ci, sr, sc, sv = I.q1_assembly(dims)
    rows = np.repeat(np.arange(n), np.diff(rp))
    gv = -lam[rows] * x[ci]
    gk = np.zeros(theta0.size)
    np.add.at(gk, sc, sv * gv[sr])
    kappa = np.exp(theta0)
    out = torch.full((theta0.size,), 5.0, dtype=torch.float64, device=DEV)
    sstep.q1_grad(dims, dev(kappa), dev(lam), dev(x), out, wrt_log=False)
    scale = np.abs(sv).max() * np.abs(lam).max() * np.abs(x).max() * 8
    assert np.max(np.abs(out.cpu().numpy() - gk)) <= 1e-13 * scale
    sstep.q1_grad(dims, dev(kappa), dev(lam), dev(x), out, wrt_log=True, accumulate=True)
    assert np.max(np.abs(out.cpu().numpy() - gk * (1 + kappa))) <= 1e-13 * scale * (1 + kappa.max())


def _dense_q1(dims, theta0):
    rp, ci, sr, sc, sv = I.q1_assembly(dims)
    kappa = np.exp(theta0)
    vals = np.zeros(ci.size)
    np.add.at(vals, sr, sv * kappa[sc])
    n = rp.size - 1
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    A[rows, ci] = vals
    return A, (rp, ci, sr, sc, sv, rows)


@pytest.mark.parametrize("precond", ["jacobi", "amg"])
def test_q1_theta_gradient(precond):
    dims = (12, 10, 9)
    theta0, b0, t0 = _problem(dims, 5)
    patt = AG.Q1Pattern(dims, DEV)
    pk = dict(precond=precond, amg_coarse_max=64) if precond == "amg" else {}
    opts = dict(s=4, sweeps=30, rtol=1e-12, **pk)
    b, target = dev(b0), dev(t0)
    theta = dev(theta0).requires_grad_(True)
    x = AG.q1_solve(theta, b, patt, **opts)
    loss = 0.5 * torch.sum((x - target) ** 2)
    loss.backward()
    g = theta.grad.cpu().numpy()

    # (a) dense FP64: x = A^-1 b, lam = A^-1 (x - t), dL/dkappa_c = -sum_t lam_i x_j S_t, * kappa
    A, (rp, ci, sr, sc, sv, rows) = _dense_q1(dims, theta0)
    xd = np.linalg.solve(A, b0)
    lam = np.linalg.solve(A, xd - t0)
    gv = -lam[rows] * xd[ci]
    gk = np.zeros(theta0.size)
    np.add.at(gk, sc, sv * gv[sr])
    gd = gk * np.exp(theta0)
    assert np.linalg.norm(x.detach().cpu().numpy() - xd) <= 1e-9 * np.linalg.norm(xd)
    assert np.linalg.norm(g - gd) <= 1e-6 * np.linalg.norm(gd)

    # (b) central differences through the CUDA solver on 32 random cells
    rng = np.random.default_rng(9)
    cells = rng.choice(np.flatnonzero(np.abs(gd) > 1e-3 * np.abs(gd).max()), 32, replace=False)
    o13 = dict(opts, rtol=1e-13)
    h = 1e-4
    for c in cells:
        tp = dev(theta0)
        tm = tp.clone()
        tp[c] += h
        tm[c] -= h
        with torch.no_grad():
            fp = 0.5 * torch.sum((AG.q1_solve(tp, b, patt, **o13) - target) ** 2).item()
            fm = 0.5 * torch.sum((AG.q1_solve(tm, b, patt, **o13) - target) ** 2).item()
        fd = (fp - fm) / (2 * h)
        assert abs(fd - g[c]) <= 1e-5 * np.abs(gd).max(), (c, fd, g[c])


def test_rhs_gradient_is_adjoint():
    dims = (10, 8, 8)
    theta0, b0, t0 = _problem(dims, 2)
    patt = AG.Q1Pattern(dims, DEV)
    theta = dev(theta0)
    b = dev(b0).requires_grad_(True)
    w = dev(t0)
    x = AG.q1_solve(theta, b, patt, s=4, sweeps=30, rtol=1e-12)
    torch.sum(w * x).backward()
    # d(w^T A^-1 b)/db = A^-1 w (A symmetric)
    lam = AG.q1_solve(theta, w, patt, s=4, sweeps=30, rtol=1e-12)
    assert torch.allclose(b.grad, lam, rtol=0, atol=1e-12 * lam.abs().max().item())


def test_csr_values_gradient_matches_dense():
    """solve(vals, b, pattern): dL/dvals = -lambda_i x_j on the stored pattern."""
    dims = (8, 7, 6)
    theta0, b0, t0 = _problem(dims, 12)
    patt = AG.Q1Pattern(dims, DEV)
    vals = patt.values(dev(np.exp(theta0))).requires_grad_(True)
    x = AG.solve(vals, dev(b0), patt.pattern, s=4, sweeps=30, rtol=1e-12)
    torch.sum((x - dev(t0)) ** 2).backward()
    A, (rp, ci, sr, sc, sv, rows) = _dense_q1(dims, theta0)
    xd = np.linalg.solve(A, b0)
    lam = np.linalg.solve(A, 2 * (xd - t0))
    gv = -lam[rows] * xd[ci]
    assert np.linalg.norm(vals.grad.cpu().numpy() - gv) <= 1e-7 * np.linalg.norm(gv)


def test_update_values_matches_fresh_setup():
    dims = (10, 9, 8)
    theta0, b0, _ = _problem(dims, 4)
    patt = AG.Q1Pattern(dims, DEV)
    v1 = patt.values(dev(np.exp(theta0)))
    v2 = patt.values(dev(np.exp(theta0 * 0.5)))
    b = dev(b0)
    A1 = sstep.CSR(patt.pattern.rowptr, patt.pattern.colind, v1)
    A2 = sstep.CSR(patt.pattern.rowptr, patt.pattern.colind, v2)
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
    patt = AG.Q1Pattern(dims, DEV)
    theta = dev(theta0).requires_grad_(True)
    x = AG.q1_solve(theta, dev(b0), patt, s=4, sweeps=30, rtol=1e-12)
    loss = torch.sum(x * x)
    loss.backward(retain_graph=True)
    g1 = theta.grad.clone()
    theta.grad = None
    loss.backward()
    assert torch.allclose(theta.grad, g1, rtol=1e-9, atol=1e-14 * g1.abs().max().item())


# ---------------------------------------------------------------- batched adjoint

def _dense7(g, wc, wo):
    nx, ny, nz = g
    n = nx * ny * nz
    Nm = np.zeros((n, n))
    for i in range(n):
        ix, iy, iz = i % nx, (i // nx) % ny, i // (nx * ny)
        for d, (ok, off) in enumerate(((ix > 0, -1), (ix + 1 < nx, 1), (iy > 0, -nx),
                                       (iy + 1 < ny, nx), (iz > 0, -nx * ny), (iz + 1 < nz, nx * ny))):
            if ok:
                Nm[i, i + off] = 1.0
    return wc * np.eye(n) + wo * Nm, Nm


def test_batched_adjoint_matches_dense():
    """Weights (wc_i, wo_i) of three 7-point systems with two right-hand sides each, all solved
    by one batched launch per pass; gradient of 0.5 sum ||x - t||^2 against dense FP64."""
    grids = [(6, 5, 4), (7, 6, 5), (5, 5, 6)]
    nrhs = 2
    wc0, wo0 = np.array([6.5, 7.0, 6.2]), np.array([-1.0, -1.1, -0.9])
    bs0 = [I.uniform_pm1(20 + p, int(np.prod(grids[p // nrhs]))) for p in range(3 * nrhs)]
    ts0 = [I.uniform_pm1(40 + p, int(np.prod(grids[p // nrhs]))) for p in range(3 * nrhs)]
    wc, wo = dev(wc0).requires_grad_(True), dev(wo0).requires_grad_(True)
    bs = [dev(v).requires_grad_(True) for v in bs0]
    xs = AG.batched_solve(wc, wo, bs, grids, s=4, sweeps=30, rtol=1e-12)
    loss = sum(0.5 * torch.sum((x - dev(t)) ** 2) for x, t in zip(xs, ts0))
    loss.backward()
    gwc, gwo = np.zeros(3), np.zeros(3)
    for p in range(3 * nrhs):
        i = p // nrhs
        A, Nm = _dense7(grids[i], wc0[i], wo0[i])
        xd = np.linalg.solve(A, bs0[p])
        lam = np.linalg.solve(A, xd - ts0[p])
        assert np.linalg.norm(xs[p].detach().cpu().numpy() - xd) <= 1e-9 * np.linalg.norm(xd)
        assert np.linalg.norm(bs[p].grad.cpu().numpy() - lam) <= 1e-9 * np.linalg.norm(lam)
        gwc[i] -= lam @ xd
        gwo[i] -= lam @ (Nm @ xd)
    assert np.allclose(wc.grad.cpu().numpy(), gwc, rtol=1e-8, atol=0)
    assert np.allclose(wo.grad.cpu().numpy(), gwo, rtol=1e-8, atol=0)
