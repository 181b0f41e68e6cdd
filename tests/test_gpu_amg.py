"""The library's aggregation AMG (precond "amg") against the oracle's (oracle/amg.c).

Set-up is integer and summation-order work done in the same fixed order on both sides, so the
hierarchy must agree bit for bit: aggregation maps, coarse sparsity patterns and coarse values.
The V-cycle differs only in rounding (fused multiply-adds, reciprocal of the l1 diagonal, the
coarsest solve through an explicit inverse instead of two triangular solves), so one
application agrees to 1e-12 relative; whole PCG-S solves with it are compared like the Jacobi
ones (fixed outer count to 1e-9 at nu = 30, free-running counts +-1).
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_09790_gb300 import inputs as I
from paper_2603_09790_gb300 import sstep

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def q1(dims, seed=3, sigma=1.0, corr=4.0):
    (rp, ci, v), _, _, _ = I.q1_lognormal_problem(dims, sigma=sigma, corr=corr, seed=seed)
    return rp, ci, v


CASES = [("q1", (14, 12, 10), 64), ("poisson", (20, 18, 16), 100), ("q1", (9, 17, 11), 30),
         ("q1", (40, 36, 32), 512)]  # large enough for the threaded host set-up (>= 8192 rows)


def problem(kind, dims):
    if kind == "q1":
        return q1(dims)
    return I.poisson_csr(dims, 7)


@pytest.mark.parametrize("kind,dims,cmax", CASES)
def test_hierarchy_is_bit_identical(kind, dims, cmax):
    rp, ci, v = problem(kind, dims)
    csr = O.CSR(rp, ci, v)
    M = O.AMG(csr, coarse_max=cmax, max_levels=25)
    with sstep.Solver(sstep.CSR(dev(rp), dev(ci), dev(v)), precond="amg", amg_coarse_max=cmax,
                      amg_max_levels=25, lambda_max=2.0) as S:
        levels = S.amg_levels()
    assert len(levels) == M.nlevels >= 2
    for l, ((grp, gci, gv), gagg) in enumerate(levels):
        ref, ragg = M.level(l)
        assert np.array_equal(grp, ref.rowptr) and np.array_equal(gci, ref.colind)
        assert np.array_equal(gv, ref.vals)  # bit for bit
        if ragg is None:
            assert gagg is None
        else:
            assert np.array_equal(gagg, ragg)


@pytest.mark.parametrize("kind,dims,cmax", CASES)
def test_vcycle_matches_oracle(kind, dims, cmax):
    rp, ci, v = problem(kind, dims)
    csr = O.CSR(rp, ci, v)
    M = O.AMG(csr, coarse_max=cmax)
    with sstep.Solver(sstep.CSR(dev(rp), dev(ci), dev(v)), precond="amg", amg_coarse_max=cmax,
                      lambda_max=2.0) as S:
        for seed in (1, 2):
            b = I.uniform_pm1(seed, csr.n)
            x = torch.empty(csr.n, dtype=torch.float64, device=DEV)
            S.amg_apply(dev(b), x)
            assert relerr(x.cpu().numpy(), M.apply(b)) <= 1e-12


def test_power_method_matches_oracle():
    rp, ci, v = q1((14, 12, 10))
    csr = O.CSR(rp, ci, v)
    M = O.AMG(csr, coarse_max=64)
    v0 = I.power_start(csr.n)
    ref, _ = O.power(csr, "amg", v0, 20, 0.0, amg=M)
    with sstep.Solver(sstep.CSR(dev(rp), dev(ci), dev(v)), precond="amg", amg_coarse_max=64,
                      power_iters=20, power_tol=0.0, power_v0=dev(v0)) as S:
        bi = S.get_basis_info()
    assert abs(bi["lambda_max"] - ref) <= 1e-10 * ref
    assert bi["lambda_min"] == 0.0 or bi["lambda_min"] >= 0.0


@pytest.mark.parametrize("algo,s,K", [("literal", 4, 8), ("onesync", 4, 8), ("literal", 2, 12),
                                      ("literal", 8, 4)])
def test_solve_fixed_count_matches_oracle(algo, s, K):
    rp, ci, v = q1((14, 12, 10))
    csr = O.CSR(rp, ci, v)
    M = O.AMG(csr, coarse_max=64)
    b = I.uniform_pm1(9, csr.n)
    with sstep.Solver(sstep.CSR(dev(rp), dev(ci), dev(v)), precond="amg", amg_coarse_max=64,
                      s=s, sweeps=30, rtol=0.0, max_outer=K, algo=algo, power_iters=20,
                      power_tol=0.0) as S:
        x = torch.zeros(csr.n, dtype=torch.float64, device=DEV)
        info = S.solve(dev(b), x)
        bi = S.get_basis_info()
    assert info.status == sstep.NOT_CONVERGED and info.outer_iters == K
    ref = O.pcgs(csr, b, s=s, nu=30, rtol=0.0, max_outer=K, algo=algo, prec="amg", amg=M,
                 lambda_min=bi["lambda_min"], lambda_max=bi["lambda_max"])
    assert relerr(x.cpu().numpy(), ref.x) <= 1e-9


def test_solve_free_running_matches_oracle():
    rp, ci, v = q1((20, 18, 16), corr=8.0)
    csr = O.CSR(rp, ci, v)
    M = O.AMG(csr, coarse_max=128)
    b = I.uniform_pm1(4, csr.n)
    with sstep.Solver(sstep.CSR(dev(rp), dev(ci), dev(v)), precond="amg", amg_coarse_max=128,
                      s=4, sweeps=30, rtol=1e-8, power_iters=20, power_tol=0.0) as S:
        x = torch.zeros(csr.n, dtype=torch.float64, device=DEV)
        info = S.solve(dev(b), x)
        bi = S.get_basis_info()
    ref = O.pcgs(csr, b, s=4, nu=30, rtol=1e-8, prec="amg", amg=M,
                 lambda_min=bi["lambda_min"], lambda_max=bi["lambda_max"])
    assert info.status == sstep.OK and ref.status == O.OK
    assert abs(info.outer_iters - ref.iters) <= 1 and info.relres_true <= 2e-8
    if info.outer_iters == ref.iters:
        assert relerr(x.cpu().numpy(), ref.x) <= 1e-9
    jac = O.pcgs(csr, b, s=4, nu=30, rtol=1e-8, prec="jacobi", power_iters=20, power_tol=0.0)
    assert info.outer_iters < jac.iters  # the V-cycle is the stronger preconditioner


def test_update_values_rebuilds_the_hierarchy():
    rp, ci, v1 = q1((12, 11, 10), seed=1)
    _, _, v2 = q1((12, 11, 10), seed=2)
    b = dev(I.uniform_pm1(3, rp.size - 1))
    kw = dict(precond="amg", amg_coarse_max=64, s=4, sweeps=30, rtol=1e-10, lambda_max=1.5)
    with sstep.Solver(sstep.CSR(dev(rp), dev(ci), dev(v2)), **kw) as S:
        xf = torch.zeros_like(b)
        i1 = S.solve(b, xf)
        lv2 = S.amg_levels()
    with sstep.Solver(sstep.CSR(dev(rp), dev(ci), dev(v1)), **kw) as S:
        xu = torch.zeros_like(b)
        S.solve(b, xu)
        S.update_values(dev(v2))
        xu.zero_()
        i2 = S.solve(b, xu)
        lvu = S.amg_levels()
    assert i1.outer_iters == i2.outer_iters and torch.equal(xf, xu)
    assert all(np.array_equal(a[0][2], c[0][2]) for a, c in zip(lv2, lvu))


def test_amg_rejects_unsupported():
    rp, ci, v = q1((8, 8, 8))
    A = sstep.CSR(dev(rp), dev(ci), dev(v))
    for kw in (dict(algo="pcg"), dict(precision="fp32_rr"), dict(amg_coarse_max=5000)):
        with pytest.raises(sstep.SstepError):
            sstep.Solver(A, precond="amg", lambda_max=2.0, **kw)
    with pytest.raises(sstep.SstepError) as e:
        sstep.Solver(sstep.Stencil(8, 8, 8, 7), precond="amg", lambda_max=2.0)
    assert e.value.status == sstep.ERR_UNSUPPORTED
    with sstep.Solver(A, lambda_max=2.0) as S:  # Jacobi handle: no hierarchy
        with pytest.raises(sstep.SstepError):
            S.amg_levels()
