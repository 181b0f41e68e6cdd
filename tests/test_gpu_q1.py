"""The matrix-free Q1 operator (sstep.Q1, SSTEP_MATRIX_Q1) against the oracle run on the CSR
matrix that the input generator assembles from the same conductivities.

The two sides build A independently: the generator sums kappa_e K_ref[i, j] over the cells of a
pair (K_ref from the Kronecker form of the element stiffness), the kernel forms 1/3, -1/12 and
pair sums of conductivities on the fly.  They agree to rounding (a few units in the last place
of each entry), so one application agrees to 1e-13 of sum_j |a_ij x_j|, and whole solves are
held to the FP64 contract: relative error <= 1e-9 at a fixed outer count, free-running counts
within +-1.  The FP32-basis form is held to the FP64 true residual, like the CSR form.
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


def problem(dims, seed=0, corr=4.0, sigma=1.0):
    (rp, ci, v), kappa, xt, b = I.q1_lognormal_problem(dims, sigma=sigma, corr=corr, seed=seed)
    return O.CSR(rp, ci, v), kappa, b


def q1(dims, kappa, on_device=True):
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    return sstep.Q1(*dims, dev(k) if on_device else k)


# several tiles in x and y, z chunks, a ragged tail in every direction, and degenerate sizes
DIMS = [(1, 1, 1), (2, 3, 4), (33, 9, 5), (40, 17, 12), (65, 18, 20)]


@pytest.mark.parametrize("dims", DIMS)
def test_spmv_matches_oracle(dims):
    csr, kappa, _ = problem(dims, seed=1)
    n = csr.n
    x = I.uniform_pm1(5, n)
    ref = O.spmv(csr, x)
    scale = O.spmv(O.CSR(csr.rowptr, csr.colind, np.abs(csr.vals)), np.abs(x))
    with sstep.Solver(q1(dims, kappa), lambda_max=2.0) as S:
        y = torch.empty(n, dtype=torch.float64, device=DEV)
        S.spmv(dev(x), y)
        got = y.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-13 * scale)


@pytest.mark.parametrize("dims", [(2, 2, 2), (12, 10, 9), (33, 9, 5)])
@pytest.mark.parametrize("prec", ["jacobi", "none"])
def test_gershgorin_and_power_match_oracle(dims, prec):
    csr, kappa, _ = problem(dims, seed=2)
    v0 = I.power_start(csr.n)
    lo = O.gershgorin_lower(csr, prec)
    lam, _ = O.power(csr, prec, v0, 20, 0.0)
    with sstep.Solver(q1(dims, kappa), precond=prec, lambda_min=-1.0, power_iters=20,
                      power_tol=0.0, power_v0=dev(v0)) as S:
        bi = S.get_basis_info()
    assert abs(bi["lambda_min"] - max(lo, 0.0)) <= 1e-12 * max(1.0, abs(lo))
    assert abs(bi["lambda_max"] - lam) <= 1e-11 * lam


@pytest.mark.parametrize("algo,s,nu,K", [("literal", 4, 30, 10), ("literal", 8, 3, 6),
                                         ("onesync", 4, 30, 10), ("literal", 1, 2, 25),
                                         ("literal", 6, 30, 5)])
def test_fixed_count_matches_oracle(algo, s, nu, K):
    dims = (33, 20, 14)
    csr, kappa, b = problem(dims)
    lmax = 1.98
    with sstep.Solver(q1(dims, kappa), s=s, sweeps=nu, rtol=0.0, max_outer=K, algo=algo,
                      lambda_max=lmax) as S:
        x = torch.zeros(csr.n, dtype=torch.float64, device=DEV)
        info = S.solve(dev(b), x)
    assert info.status == sstep.NOT_CONVERGED and info.outer_iters == K
    ref = O.pcgs(csr, b, s=s, nu=nu, rtol=0.0, max_outer=K, algo=algo, lambda_min=0.0,
                 lambda_max=lmax)
    assert relerr(x.cpu().numpy(), ref.x) <= 1e-9


def test_free_running_and_pcg_match_oracle():
    dims = (40, 17, 12)
    csr, kappa, b = problem(dims, corr=8.0)
    v0 = I.power_start(csr.n)
    with sstep.Solver(q1(dims, kappa), s=4, sweeps=30, rtol=1e-8, power_iters=20, power_tol=0.0,
                      power_v0=dev(v0)) as S:
        x = torch.zeros(csr.n, dtype=torch.float64, device=DEV)
        info = S.solve(dev(b), x)
        bi = S.get_basis_info()
    ref = O.pcgs(csr, b, s=4, nu=30, rtol=1e-8, lambda_min=bi["lambda_min"],
                 lambda_max=bi["lambda_max"])
    assert info.status == sstep.OK and ref.status == O.OK
    assert abs(info.outer_iters - ref.iters) <= 1 and info.relres_true <= 2e-8
    if info.outer_iters == ref.iters:
        assert relerr(x.cpu().numpy(), ref.x) <= 1e-9
    with sstep.Solver(q1(dims, kappa), algo="pcg", rtol=1e-8, lambda_max=2.0) as S:
        xp = torch.zeros(csr.n, dtype=torch.float64, device=DEV)
        ip = S.solve(dev(b), xp)
    rp = O.pcg(csr, b, rtol=1e-8)
    assert ip.status == sstep.OK and abs(ip.outer_iters - rp.iters) <= 1
    if ip.outer_iters == rp.iters:
        assert relerr(xp.cpu().numpy(), rp.x) <= 1e-9


@pytest.mark.parametrize("dims,s", [((24, 20, 16), 8), ((33, 9, 13), 4), ((64, 8, 8), 2)])
def test_fp32_basis_reaches_fp64_true_residual(dims, s):
    csr, kappa, b = problem(dims, corr=8.0)
    v0 = dev(I.power_start(csr.n))
    kw = dict(s=s, sweeps=30, rtol=1e-8, power_v0=v0)
    with sstep.Solver(q1(dims, kappa), precision="fp32_rr", rr_period=s, **kw) as S:
        x = torch.zeros(csr.n, dtype=torch.float64, device=DEV)
        info = S.solve(dev(b), x)
    assert info.status == sstep.OK and info.relres_true <= 2e-8
    # same solve with the assembled CSR matrix: the operator is the same up to rounding
    with sstep.Solver(sstep.CSR(dev(csr.rowptr), dev(csr.colind), dev(csr.vals)),
                      precision="fp32_rr", rr_period=s, **kw) as S:
        xc = torch.zeros(csr.n, dtype=torch.float64, device=DEV)
        ic = S.solve(dev(b), xc)
    assert ic.status == sstep.OK and abs(info.outer_iters - ic.outer_iters) <= 2
    ref = O.pcg(csr, b, rtol=1e-12)
    lam = np.linalg.eigvalsh(csr.dense())
    assert relerr(x.cpu().numpy(), ref.x) <= 2e-8 * lam[-1] / lam[0]


def test_host_kappa_and_update_values():
    dims = (20, 14, 11)
    csr1, k1, b = problem(dims, seed=1)
    _, k2, _ = problem(dims, seed=2)
    kw = dict(s=4, sweeps=30, rtol=1e-10, lambda_max=1.9)
    bd = dev(b)
    outs = []
    for A in (q1(dims, k2), q1(dims, k2, on_device=False)):
        with sstep.Solver(A, **kw) as S:
            x = torch.zeros_like(bd)
            outs.append((S.solve(bd, x).outer_iters, x))
    assert outs[0][0] == outs[1][0] and torch.equal(outs[0][1], outs[1][1])
    with sstep.Solver(q1(dims, k1), **kw) as S:
        x = torch.zeros_like(bd)
        S.solve(bd, x)
        S.update_values(dev(np.ascontiguousarray(k2)))
        x.zero_()
        it = S.solve(bd, x).outer_iters
    assert it == outs[0][0] and torch.equal(x, outs[0][1])


def test_q1_rejects_invalid():
    dims = (6, 5, 4)
    _, kappa, _ = problem(dims)
    for bad in (0.0, -1.0, np.nan, np.inf):
        k = kappa.copy()
        k[2, 3, 1] = bad
        with pytest.raises(sstep.SstepError) as e:
            sstep.Solver(q1(dims, k), lambda_max=2.0)
        assert e.value.status == sstep.ERR_INVALID
    with pytest.raises(ValueError):
        sstep.Solver(sstep.Q1(6, 5, 4, dev(kappa[:, :, :-1].copy())), lambda_max=2.0)
    with pytest.raises(sstep.SstepError) as e:
        sstep.Solver(q1(dims, kappa), precond="amg", lambda_max=2.0)
    assert e.value.status == sstep.ERR_UNSUPPORTED
    with sstep.Solver(q1(dims, kappa), lambda_max=2.0) as S:
        k = kappa.copy()
        k[0, 0, 0] = -2.0
        with pytest.raises(sstep.SstepError):
            S.update_values(dev(k))


@pytest.mark.parametrize("dims", [(72, 10, 9), (76, 12, 17), (128, 24, 20), (96, 33, 8),
                                  (64, 24, 20)])
def test_fp32_tma_steps_equal_plain_loads(dims, monkeypatch):
    """nx a multiple of 4 and the grid no smaller than the copy boxes (nx >= 72, ny >= 10): the
    middle MPK steps take the tensor-memory-accelerator kernel (64 x 8 vertex tiles: one full
    tile, a ragged x tail, several tiles and z chunks).  It does the plain kernel's arithmetic
    in the same order, so both give the same iterates bit for bit; the solve reaches the FP64
    true residual.  (64, 24, 20) is below the box width and takes plain loads either way."""
    csr, kappa, b = problem(dims, corr=4.0)
    kw = dict(s=8, sweeps=30, rtol=1e-8, precision="fp32_rr", rr_period=8, lambda_max=1.97)
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("SSTEP_Q1_TMA", flag)
        with sstep.Solver(q1(dims, kappa), **kw) as S:
            x = torch.zeros(csr.n, dtype=torch.float64, device=DEV)
            info = S.solve(dev(b), x)
        out.append((info, x))
    (i1, x1), (i0, x0) = out
    assert i1.status == sstep.OK and i1.relres_true <= 2e-8
    assert i1.outer_iters == i0.outer_iters and torch.equal(x1, x0)


@pytest.mark.parametrize("dims", [(24, 20, 16), (33, 9, 13), (76, 12, 17), (128, 24, 20)])
def test_fp32_pcg_matrix_free(dims, monkeypatch):
    """Classical PCG in the FP32-basis recipe on the matrix-free operator (A p and p^T A p in the
    FP32 Q1 kernels): it reaches the FP64 true residual with a count close to the oracle's PCG on
    the assembled matrix, and on the small grids its solution agrees with the oracle's to the
    kappa-scaled FP64 bound.  Where the TMA-fed kernel applies (nx a multiple of 4, nx >= 72,
    ny >= 10) the plain-load kernel gives the same solve up to the order of the p^T A p sums."""
    csr, kappa, b = problem(dims, corr=4.0)
    kw = dict(algo="pcg", rtol=1e-8, precision="fp32_rr", lambda_max=2.0)
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("SSTEP_Q1_TMA", flag)
        with sstep.Solver(q1(dims, kappa), **kw) as S:
            x = torch.zeros(csr.n, dtype=torch.float64, device=DEV)
            info = S.solve(dev(b), x)
        out.append((info, x.cpu().numpy()))
    (i1, x1), (i0, x0) = out
    ref = O.pcg(csr, b, rtol=1e-8)
    for info in (i1, i0):
        assert info.status == sstep.OK and info.relres_true <= 2e-8
        assert abs(info.outer_iters - ref.iters) <= max(3, 0.05 * ref.iters), (info.outer_iters,
                                                                             ref.iters)
    assert abs(i1.outer_iters - i0.outer_iters) <= 2
    if csr.n <= 8000:
        lam = np.linalg.eigvalsh(csr.dense())
        exact = O.pcg(csr, b, rtol=1e-13).x
        for x in (x1, x0):
            assert relerr(x, exact) <= 2e-8 * lam[-1] / lam[0]
