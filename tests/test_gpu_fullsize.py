"""Full-size checks of the side workloads in the launch configuration the benchmark times,
through properties the oracle can confirm at that size.

* 192^3 Q1 log-normal diffusion, FP32 basis, s = 8, nu = 30, with the CSR matrix and with the
  matrix-free operator: the solve converges and the oracle's product confirms
  ||b - A x|| <= 2e-8 ||b|| (the FP32-form tolerance); one matrix-free product agrees with the
  oracle's on every row.
* 128^3 Q1 diffusion with theta ~ N(0, 0.5^2) per cell: the library's AMG hierarchy equals the
  oracle's bit for bit on every level, and one V-cycle agrees to 1e-12.
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


@pytest.fixture(scope="module")
def q1_192():
    return I.q1_lognormal_problem((192, 192, 192))


@pytest.mark.parametrize("form", ["csr", "matrix_free"])
def test_q1_192_fp32_s8_converges_to_fp64_residual(q1_192, form):
    (rp, ci, v), kappa, xt, b = q1_192
    A = sstep.CSR(dev(rp), dev(ci), dev(v)) if form == "csr" else sstep.Q1(192, 192, 192, dev(kappa))
    with sstep.Solver(A, s=8, sweeps=30, rtol=1e-8, precision="fp32_rr", rr_period=8,
                      power_iters=20, power_tol=0.0, lambda_min=-1.0) as S:
        x = torch.zeros(b.size, dtype=torch.float64, device=DEV)
        info = S.solve(dev(b), x)
    assert info.status == sstep.OK and info.relres_true <= 2e-8
    xh = x.cpu().numpy()
    r = b - O.spmv(O.CSR(rp, ci, v), xh)
    assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(b)


def test_q1_192_matrix_free_product_matches_oracle(q1_192):
    """Every row of one matrix-free product at the benchmark's size, in its launch shape."""
    (rp, ci, v), kappa, xt, b = q1_192
    csr = O.CSR(rp, ci, v)
    x = I.uniform_pm1(7, csr.n)
    ref = O.spmv(csr, x)
    scale = O.spmv(O.CSR(rp, ci, np.abs(v)), np.abs(x))
    with sstep.Solver(sstep.Q1(192, 192, 192, dev(kappa)), lambda_max=2.0) as S:
        y = torch.empty(csr.n, dtype=torch.float64, device=DEV)
        S.spmv(dev(x), y)
        got = y.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-13 * scale)


def test_amg_128_hierarchy_and_vcycle_match_oracle():
    N = 128
    dims = (N, N, N)
    kappa = np.exp(0.5 * I.normal_pm(0, (N + 1) ** 3)).reshape(N + 1, N + 1, N + 1)
    rp, ci, v = I.q1_csr(dims, kappa)
    csr = O.CSR(rp, ci, v)
    M = O.AMG(csr, coarse_max=512)
    with sstep.Solver(sstep.CSR(dev(rp), dev(ci), dev(v)), precond="amg", amg_coarse_max=512,
                      lambda_max=2.0) as S:
        levels = S.amg_levels()
        b = I.uniform_pm1(3, csr.n)
        x = torch.empty(csr.n, dtype=torch.float64, device=DEV)
        S.amg_apply(dev(b), x)
    assert len(levels) == M.nlevels
    for l, ((grp, gci, gv), gagg) in enumerate(levels):
        ref, ragg = M.level(l)
        assert np.array_equal(grp, ref.rowptr) and np.array_equal(gci, ref.colind)
        assert np.array_equal(gv, ref.vals)
        assert (gagg is None) == (ragg is None)
        if ragg is not None:
            assert np.array_equal(gagg, ragg)
    ref = M.apply(b)
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
