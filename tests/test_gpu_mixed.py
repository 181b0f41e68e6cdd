"""The FP32-basis path (precision = fp32_rr) against the FP64 oracle and the FP64 CUDA path.

Tolerance.  The basis Z, AZ, Q, AQ and the MPK SpMV are FP32 (unit roundoff 6e-8); Gram sums
and the x, r increments are double-float (about 48 bits); r = b - A x is recomputed in FP64
every rr_period outer iterations.  So the solve reaches the same FP64 true residual as the FP64
path (checked at <= 2e-8 for rtol 1e-8), and its solution differs from the FP64 oracle's by at
most what two solutions at rtol 1e-8 can differ: about rtol * kappa(A).  Iterates at a fixed
outer count differ from the FP64 path by the FP32 rounding of the basis, amplified by the
iteration: a few 1e-6 on these problems (checked at 1e-4).
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


def solve(A, b, **kw):
    with sstep.Solver(A, **kw) as S:
        x = dev(np.zeros_like(b))
        info = S.solve(dev(b), x)
        torch.cuda.synchronize()
        return x.cpu().numpy(), info, S.get_basis_info()


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def poisson_kappa(dims, points):
    """kappa(A) of the Dirichlet Poisson matrix from its closed-form spectrum: with
    theta = k pi / (N + 1), k = 1..N per axis, lambda = sum_d (2 - 2 cos theta_d) (5/7 points)
    or 27 - prod_d (1 + 2 cos theta_d) (27 points); the extremes sit at k = 1 or k = N."""
    ends = [np.cos(np.array([1, N]) * np.pi / (N + 1)) for N in dims]
    if points in (5, 7):
        lmin = sum(2 - 2 * c[0] for c in ends)
        lmax = sum(2 - 2 * c[1] for c in ends)
    else:
        prods = [a * b * c for a in 1 + 2 * ends[0] for b in 1 + 2 * ends[1] for c in 1 + 2 * ends[2]]
        lmin, lmax = 27 - max(prods), 27 - min(prods)
    return lmax / lmin


@pytest.mark.parametrize("form,dims,points,s,nu", [
    ("stencil", (40, 36, 28), 7, 4, 30), ("stencil", (40, 36, 28), 7, 4, 3),
    ("csr", (64, 64), 5, 4, 30), ("stencil", (64, 64), 5, 2, 3), ("csr", (30, 26, 22), 27, 8, 30)])
def test_mixed_reaches_fp64_true_residual(form, dims, points, s, nu):
    csr = O.CSR(*I.poisson_csr(dims, points))
    nx, ny, nz = (tuple(dims) + (1,))[:3]
    A = sstep.Stencil(nx, ny, nz, points) if form == "stencil" else \
        sstep.CSR(dev(csr.rowptr), dev(csr.colind), dev(csr.vals))
    xt, b = I.poisson_problem(dims, points)
    x, info, bi = solve(A, b, s=s, sweeps=nu, rtol=1e-8, precision="fp32_rr",
                        power_v0=dev(I.power_start(csr.n)))
    assert info.status == sstep.OK
    assert info.relres_true <= 2e-8
    ref = O.pcgs(csr, b, s=s, nu=nu, rtol=1e-8, algo="literal", lambda_max=bi["lambda_max"])
    assert ref.status == O.OK
    assert relerr(x, ref.x) <= 2e-8 * poisson_kappa((nx, ny, nz)[:len(dims)], points) + 1e-10


def test_mixed_q1_lognormal_s8():
    """Variable-coefficient Q1 diffusion with log-normal conductivity (sigma 1, correlation
    8 cells), s = 8, residual replacement every s outer iterations."""
    dims = (24, 20, 16)
    (rp, ci, v), kappa, xt, b = I.q1_lognormal_problem(dims)
    csr = O.CSR(rp, ci, v)
    A = sstep.CSR(dev(rp), dev(ci), dev(v))
    x, info, bi = solve(A, b, s=8, sweeps=30, rtol=1e-8, precision="fp32_rr", rr_period=8,
                        power_v0=dev(I.power_start(csr.n)))
    assert info.status == sstep.OK and info.relres_true <= 2e-8
    x64, info64, _ = solve(A, b, s=8, sweeps=30, rtol=1e-8, power_v0=dev(I.power_start(csr.n)))
    ref = O.pcg(csr, b, rtol=1e-12)
    lam = np.linalg.eigvalsh(csr.dense())
    kappa_A = lam[-1] / lam[0]
    assert relerr(x, ref.x) <= 2e-8 * kappa_A
    assert relerr(x64, ref.x) <= 2e-8 * kappa_A


@pytest.mark.parametrize("s", [1, 2, 4, 6, 8])
def test_mixed_fixed_count_close_to_fp64(s):
    dims = (30, 26, 22)
    A = sstep.Stencil(*dims, points=7)
    xt, b = I.poisson_problem(dims, 7)
    K = 12
    kw = dict(s=s, sweeps=30, rtol=0.0, max_outer=K, lambda_max=1.95)
    xm, im, _ = solve(A, b, precision="fp32_rr", **kw)
    xd, idd, _ = solve(A, b, **kw)
    assert im.outer_iters == K and idd.outer_iters == K
    assert relerr(xm, xd) <= 1e-4


@pytest.mark.parametrize("s", [5, 7, 8])
def test_mixed_wide_update_one_pass_equals_two_pass(s, monkeypatch):
    """For 5 <= s <= 8 the Q/AQ update and W, b1 run as one pass (two points per thread); the
    two-pass form (SSTEP_FP32_UPD_TWO_PASS=1) does the same arithmetic with the Gram sums in
    another order.  On a grid with an odd number of points (the one-point tail) both stay
    within the FP32 recipe's distance of the FP64 solve at a fixed outer count and agree with
    each other to the level of that summation-order difference."""
    dims = (31, 25, 21)
    A = sstep.Stencil(*dims, points=7)
    xt, b = I.poisson_problem(dims, 7)
    K = 10
    kw = dict(s=s, sweeps=30, rtol=0.0, max_outer=K, lambda_max=1.95)
    xs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("SSTEP_FP32_UPD_TWO_PASS", flag)
        x, info, _ = solve(A, b, precision="fp32_rr", **kw)
        assert info.outer_iters == K
        xs.append(x)
    xd, idd, _ = solve(A, b, **kw)
    for x in xs:
        assert relerr(x, xd) <= 1e-4
    assert relerr(xs[0], xs[1]) <= 1e-5


def test_mixed_rejects_unsupported():
    A = sstep.Stencil(10, 10, 10, 7)
    for kw in (dict(s=9), dict(algo="onesync"), dict(gram="cholesky")):
        with pytest.raises(sstep.SstepError) as e:
            sstep.Solver(A, precision="fp32_rr", lambda_max=2.0, **kw)
        assert e.value.status == sstep.ERR_UNSUPPORTED
    with pytest.raises(sstep.SstepError):
        sstep.Solver(sstep.Stencil(10, 10, 10, 27), precision="fp32_rr", lambda_max=2.0)


# ---------------------------------------------------------------- FP32 PCG comparator
# Classical PCG in the same precision recipe: p and A p in FP32, x and r as double-float
# increments between FP64 residual replacements, reductions in double-float.  Tolerances as
# above: the FP64 true residual at rtol, the solution within rtol * kappa(A) of the oracle's,
# the iteration count within a few percent of the FP64 oracle's (FP32 directions perturb
# the Krylov recurrence at the 1e-7 level).


@pytest.mark.parametrize("form,dims,points,rrp", [
    ("stencil", (40, 36, 28), 7, 0), ("stencil", (37, 31, 23), 7, 5), ("stencil", (64, 64), 5, 0),
    ("csr", (64, 64), 5, 1), ("csr", (30, 26, 22), 27, 0)])
def test_pcg_fp32_reaches_fp64_true_residual(form, dims, points, rrp):
    csr = O.CSR(*I.poisson_csr(dims, points))
    nx, ny, nz = (tuple(dims) + (1,))[:3]
    A = sstep.Stencil(nx, ny, nz, points) if form == "stencil" else \
        sstep.CSR(dev(csr.rowptr), dev(csr.colind), dev(csr.vals))
    xt, b = I.poisson_problem(dims, points)
    x, info, _ = solve(A, b, algo="pcg", rtol=1e-8, precision="fp32_rr", rr_period=rrp,
                       lambda_max=2.0)
    assert info.status == sstep.OK
    assert info.relres_true <= 2e-8
    ref = O.pcg(csr, b, rtol=1e-8)
    assert ref.status == O.OK
    assert relerr(x, ref.x) <= 2e-8 * poisson_kappa(dims, points) + 1e-10
    assert abs(info.outer_iters - ref.iters) <= max(3, 0.05 * ref.iters), (info.outer_iters, ref.iters)


@pytest.mark.parametrize("dims", [(30, 26, 22), (33, 17, 9)])
def test_pcg_fp32_fixed_count_close_to_fp64(dims):
    A = sstep.Stencil(*dims, points=7)
    xt, b = I.poisson_problem(dims, 7)
    K = 40
    kw = dict(algo="pcg", rtol=0.0, max_outer=K, lambda_max=2.0)
    xm, im, _ = solve(A, b, precision="fp32_rr", **kw)
    xd, idd, _ = solve(A, b, **kw)
    assert im.outer_iters == K and idd.outer_iters == K
    assert relerr(xm, xd) <= 1e-4


def test_pcg_fp32_zero_rhs():
    A = sstep.Stencil(12, 10, 8, 7)
    x, info, _ = solve(A, np.zeros(960), algo="pcg", precision="fp32_rr", lambda_max=2.0)
    assert info.status == sstep.OK and info.outer_iters == 0 and not x.any()


# ---------------------------------------------------------------- TMA-fed 7-point steps
# With nx a multiple of 4, nx >= 72 and ny >= 18 the FP32 MPK steps and the FP32 PCG product
# take the kernel whose u planes arrive by tensor-memory-accelerator copies (64 x 16 tiles of a
# z chunk, 72 x 18 boxes).  SSTEP_STENCIL_TMA=0 keeps the register-fed kernel, which does the
# same arithmetic in the same order.

ANISO7 = [-0.5, -1.0, -2.0, 7.5, -2.0, -1.0, -0.5]  # -z, -y, -x, centre, +x, +y, +z


@pytest.mark.parametrize("dims,weights,s", [
    ((72, 18, 9), None, 4), ((76, 19, 17), None, 4), ((136, 40, 30), None, 8),
    ((76, 35, 21), ANISO7, 3), ((68, 18, 9), None, 4)])
def test_fp32_stencil_tma_steps_equal_register_fed(dims, weights, s, monkeypatch):
    """One full tile; ragged x and y tails; several tiles and z chunks at s = 8; weights that
    are not Poisson's; and a grid narrower than the box (plain loads either way).  The MPK
    steps carry no reduction, so the two kernels give the same basis and the same iterates bit
    for bit; the solve reaches the FP64 true residual."""
    A = sstep.Stencil(*dims, points=7, weights=weights)
    xt, b = I.poisson_problem(dims, 7)
    kw = dict(s=s, sweeps=30, rtol=1e-8, precision="fp32_rr", lambda_max=2.0)
    out = []
    for flag in ("1", "0"):
        monkeypatch.setenv("SSTEP_STENCIL_TMA", flag)
        x, info, _ = solve(A, b, **kw)
        out.append((info, x))
    (i1, x1), (i0, x0) = out
    assert i1.status == sstep.OK and i1.relres_true <= 2e-8
    assert i1.outer_iters == i0.outer_iters and np.array_equal(x1, x0)


def test_fp32_stencil_tma_against_oracle():
    """The TMA-fed steps on a grid with ragged tiles against the FP64 oracle (Algorithm 1, same
    Chebyshev interval): the solution within rtol * kappa(A) of the oracle's."""
    dims = (80, 21, 19)
    csr = O.CSR(*I.poisson_csr(dims, 7))
    xt, b = I.poisson_problem(dims, 7)
    x, info, bi = solve(sstep.Stencil(*dims, points=7), b, s=4, sweeps=3, rtol=1e-8,
                        precision="fp32_rr", power_v0=dev(I.power_start(csr.n)))
    assert info.status == sstep.OK and info.relres_true <= 2e-8
    ref = O.pcgs(csr, b, s=4, nu=3, rtol=1e-8, algo="literal", lambda_max=bi["lambda_max"])
    assert ref.status == O.OK
    assert relerr(x, ref.x) <= 2e-8 * poisson_kappa(dims, 7) + 1e-10


@pytest.mark.parametrize("dims", [(76, 19, 17), (128, 36, 24)])
def test_fp32_pcg_stencil_tma(dims, monkeypatch):
    """The FP32 PCG product (A p with p^T A p) on the TMA-fed kernel: both kernels reach the
    FP64 true residual with counts close to the oracle's PCG; the grids differ (one wave of
    resident CTAs each), so p^T A p is summed in another order and the counts may differ by a
    step or two."""
    csr = O.CSR(*I.poisson_csr(dims, 7))
    xt, b = I.poisson_problem(dims, 7)
    ref = O.pcg(csr, b, rtol=1e-8)
    assert ref.status == O.OK
    its = []
    for flag in ("1", "0"):
        monkeypatch.setenv("SSTEP_STENCIL_TMA", flag)
        x, info, _ = solve(sstep.Stencil(*dims, points=7), b, algo="pcg", rtol=1e-8,
                           precision="fp32_rr", lambda_max=2.0)
        assert info.status == sstep.OK and info.relres_true <= 2e-8
        assert abs(info.outer_iters - ref.iters) <= max(3, 0.05 * ref.iters)
        assert relerr(x, ref.x) <= 2e-8 * poisson_kappa(dims, 7) + 1e-10
        its.append(info.outer_iters)
    assert abs(its[0] - its[1]) <= 2
