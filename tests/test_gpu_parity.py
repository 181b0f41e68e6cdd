"""CUDA path (libsstep.so, through its C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances.  Every step is FP64; the kernels differ from the oracle only in summation order
(fused multiply-adds, tree reductions, the z-form of the Chebyshev recurrence), so single steps
agree to a few ulps times the conditioning of the step (1e-12 relative).  Whole solves are
compared at a fixed outer count (rtol = 0, max_outer = K) where the oracle itself is stable
under 1-ulp perturbations of b, with ||x - x_or|| / ||x_or|| <= 1e-9; free-running iteration
counts are compared (+-1) in the regime where the oracle's own count is stable (nu >= 10, or
exact Gram solves, or classical PCG).
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


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def operators(dims, points, form):
    csr = O.CSR(*I.poisson_csr(dims, points))
    nx, ny, nz = (tuple(dims) + (1,))[:3]
    if form == "stencil":
        A = sstep.Stencil(nx, ny, nz, points)
    else:
        A = sstep.CSR(dev(csr.rowptr), dev(csr.colind), dev(csr.vals))
    return A, csr


# ---------------------------------------------------------------- single steps

@pytest.mark.parametrize("dims,points,form", [
    ((37, 29), 5, "stencil"), ((37, 29, 19), 7, "stencil"), ((33, 17, 21), 27, "stencil"),
    ((37, 29), 5, "csr"), ((37, 29, 19), 7, "csr"), ((33, 17, 21), 27, "csr"),
    ((1, 1, 1), 7, "stencil"), ((64, 8, 9), 7, "stencil"), ((5, 70, 3), 27, "stencil")])
def test_spmv(dims, points, form):
    A, csr = operators(dims, points, form)
    x = I.uniform_pm1(7, csr.n)
    with sstep.Solver(A, lambda_max=2.0) as S:
        y = torch.empty(csr.n, dtype=torch.float64, device=DEV)
        S.spmv(dev(x), y)
        ref = O.spmv(csr, x)
        assert np.max(np.abs(host(y) - ref)) <= 1e-13 * max(1.0, np.abs(ref).max())


def test_spmv_general_weights():
    dims = (23, 18, 11)
    rng = np.random.default_rng(2)
    for points in (7, 27):
        w = -rng.uniform(0.1, 1.0, points)
        c = points // 2
        w[c] = -w.sum() + 0.5 + w[c]
        rp, ci, v = I.poisson_csr(dims, points)
        offs = I.stencil_offsets(points)
        # rebuild values with the given weights, entry by entry
        nx, ny, nz = dims
        for i in range(rp.size - 1):
            for k in range(rp[i], rp[i + 1]):
                d = int(ci[k]) - i
                for j, (dx, dy, dz) in enumerate(offs):
                    if dx + nx * (dy + ny * dz) == d:
                        v[k] = w[j]
        csr = O.CSR(rp, ci, v)
        x = I.uniform_pm1(3, csr.n)
        with sstep.Solver(sstep.Stencil(*dims, points=points, weights=w), lambda_max=2.0) as S:
            y = torch.empty(csr.n, dtype=torch.float64, device=DEV)
            S.spmv(dev(x), y)
            assert np.max(np.abs(host(y) - O.spmv(csr, x))) <= 1e-13 * 10


@pytest.mark.parametrize("dims,points,form,prec,s", [
    ((40, 33), 5, "csr", "jacobi", 4), ((40, 33), 5, "stencil", "jacobi", 4),
    ((26, 19, 13), 7, "stencil", "jacobi", 8), ((26, 19, 13), 7, "csr", "none", 3),
    ((17, 15, 13), 27, "stencil", "jacobi", 5), ((17, 15, 13), 27, "csr", "jacobi", 2),
    ((26, 19, 13), 7, "stencil", "none", 1)])
def test_mpk(dims, points, form, prec, s):
    """Algorithm 2: Z and A Z against the oracle for the same Chebyshev interval."""
    A, csr = operators(dims, points, form)
    n = csr.n
    r = I.uniform_pm1(11, n)
    lmin, lmax = 0.0, 1.9 if prec == "jacobi" else 2.0 * I.STENCIL_DIAG[points]
    with sstep.Solver(A, precond=prec, s=s, lambda_min=lmin, lambda_max=lmax) as S:
        info = S.get_basis_info()
        Z = torch.empty(s * n, dtype=torch.float64, device=DEV)
        AZ = torch.empty(s * n, dtype=torch.float64, device=DEV)
        S.mpk(dev(r), Z, AZ)
        Zg, AZg = host(Z).reshape(s, n), host(AZ).reshape(s, n)
    Zo, Po = O.mpk(csr, prec, r, s, info["c_alpha"], info["c_sigma"], info["c_gamma"])
    for j in range(s):
        scale = np.abs(Zo[j]).max()
        assert np.max(np.abs(Zg[j] - Zo[j])) <= 1e-12 * scale * (j + 1), j
        scale = np.abs(Po[j + 1]).max()
        assert np.max(np.abs(AZg[j] - Po[j + 1])) <= 1e-12 * scale * (j + 1), j


@pytest.mark.parametrize("n", [1, 255, 256, 257, 100003, 1 << 20])
def test_block_gram(n):
    rng = np.random.default_rng(n)
    nl, nr = 9, 11
    L = [rng.standard_normal(n) for _ in range(nl)]
    R = [rng.standard_normal(n) for _ in range(nr)]
    pairs = [(i, j) for i in range(nl) for j in range(nr) if (i + 2 * j) % 3 != 1]
    Ld, Rd = [dev(v) for v in L], [dev(v) for v in R]
    out = torch.zeros(len(pairs), dtype=torch.float64, device=DEV)
    sstep.block_gram(Ld, Rd, pairs, out)
    G = O.gram(np.array(L), np.array(R))
    got = host(out)
    for e, (i, j) in enumerate(pairs):
        bound = 1e-14 * np.sqrt(n) * np.linalg.norm(L[i]) * np.linalg.norm(R[j]) + 1e-300
        assert abs(got[e] - G[i, j]) <= bound
    # bit-reproducible
    out2 = torch.zeros_like(out)
    sstep.block_gram(Ld, Rd, pairs, out2)
    assert torch.equal(out, out2)


@pytest.mark.parametrize("s,nrhs,nu,solver", [
    (1, 1, 2, "fgs"), (4, 1, 2, "fgs"), (4, 4, 3, "fgs"), (8, 8, 30, "fgs"), (16, 16, 60, "fgs"),
    (5, 3, 0, "fgs"), (6, 6, 0, "cholesky"), (16, 2, 0, "cholesky")])
def test_fgs(s, nrhs, nu, solver):
    rng = np.random.default_rng(s * 100 + nrhs)
    G = rng.standard_normal((s, s))
    Qm, _ = np.linalg.qr(G)
    W = Qm @ np.diag(np.geomspace(1, 50, s)) @ Qm.T
    d = rng.uniform(0.3, 3.0, s)
    W = W * np.outer(d, d)
    W = (W + W.T) / 2
    B = rng.standard_normal((nrhs, s))
    X = torch.zeros((nrhs, s), dtype=torch.float64, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    sstep.fgs(dev(W.T.copy()), dev(B), nu, X, solver=solver, status=st)
    Xg = host(X)
    assert int(host(st)[0]) == 0
    for c in range(nrhs):
        ref = O.chol_solve(W, B[c]) if solver == "cholesky" else O.fgs(W, B[c], nu)
        assert np.max(np.abs(Xg[c] - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("s,nrhs,nu", [(1, 1, 1), (2, 3, 2), (3, 2, 3), (4, 4, 3), (4, 1, 30),
                                       (4, 2, 1), (5, 5, 7), (5, 2, 0), (4, 4, 64), (6, 3, 5),
                                       (7, 7, 30), (8, 8, 30), (8, 2, 1), (6, 1, 0), (8, 16, 3)])
def test_fgs_operator(s, nrhs, nu):
    """The operator form of the nu sweeps (P_nu by doubling, then X = P_nu B) against the oracle's
    sweeps: equal up to rounding, bounded by the magnitudes the products involve."""
    rng = np.random.default_rng(1000 + s * 10 + nu)
    G = rng.standard_normal((s, s))
    Qm, _ = np.linalg.qr(G)
    W = Qm @ np.diag(np.geomspace(1, 50, s)) @ Qm.T
    d = rng.uniform(0.3, 3.0, s)
    W = W * np.outer(d, d)
    W = (W + W.T) / 2
    B = rng.standard_normal((nrhs, s))
    X = torch.zeros((nrhs, s), dtype=torch.float64, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    sstep.fgs(dev(W.T.copy()), dev(B), nu, X, solver="fgs_operator", status=st)
    Xg = host(X)
    assert int(host(st)[0]) == 0
    Pref = np.column_stack([O.fgs(W, np.eye(s)[:, j], nu) for j in range(s)])
    for c in range(nrhs):
        ref = O.fgs(W, B[c], nu)
        bound = 1e-13 * (2 + np.log2(nu + 1)) * (np.abs(Pref) @ np.abs(B[c])).max() + 1e-300
        assert np.max(np.abs(Xg[c] - ref)) <= bound, (np.max(np.abs(Xg[c] - ref)), bound)


def test_fgs_operator_rejects_large_s():
    W = np.eye(9)
    X = torch.zeros((1, 9), dtype=torch.float64, device=DEV)
    with pytest.raises(sstep.SstepError) as e:
        sstep.fgs(dev(W), dev(np.ones((1, 9))), 2, X, solver="fgs_operator")
    assert e.value.status == sstep.ERR_UNSUPPORTED


def test_fgs_operator_breakdown_reported():
    W = np.array([[1.0, 0.2], [0.2, -1.0]])
    X = torch.zeros((1, 2), dtype=torch.float64, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    sstep.fgs(dev(W), dev(np.ones((1, 2))), 2, X, solver="fgs_operator", status=st)
    assert int(host(st)[0]) == sstep.ERR_BREAKDOWN


def test_fgs_breakdown_reported():
    W = np.array([[1.0, 0.2], [0.2, -1.0]])
    X = torch.zeros((1, 2), dtype=torch.float64, device=DEV)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    sstep.fgs(dev(W), dev(np.ones((1, 2))), 2, X, status=st)
    assert int(host(st)[0]) == sstep.ERR_BREAKDOWN


@pytest.mark.parametrize("s,first", [(1, False), (4, True), (4, False), (7, False), (16, False)])
def test_block_update(s, first):
    """The block updates of Section 2 (x, r and Eq. blockdirupdate) against their definitions."""
    n = 50021
    rng = np.random.default_rng(s)
    Z, AZ, Q, AQ = (rng.standard_normal((s, n)) for _ in range(4))
    x, r = rng.standard_normal(n), rng.standard_normal(n)
    alpha = rng.standard_normal(s)
    beta = rng.standard_normal((s, s)) * 0.3  # beta[l, j]
    with sstep.Solver(sstep.Stencil(n, 1, 1, 7), s=s, lambda_max=2.0) as S:
        t = [dev(a.copy()) for a in (Z, AZ, Q, AQ, x, r)]
        rr = torch.zeros(1, dtype=torch.float64, device=DEV)
        S.block_update(t[0], t[1], t[2], t[3], dev(alpha), None if first else dev(beta.T.copy()),
                       t[4], t[5], rr)
        Qg, AQg, xg, rg = host(t[2]).reshape(s, n), host(t[3]).reshape(s, n), host(t[4]), host(t[5])
    Qn = Z.copy() if first else Z + beta.T @ Q
    AQn = AZ.copy() if first else AZ + beta.T @ AQ
    xn = x + alpha @ Qn
    rn = r - alpha @ AQn
    for got, ref in ((Qg, Qn), (AQg, AQn), (xg, xn), (rg, rn)):
        assert np.max(np.abs(got - ref)) <= 1e-13 * max(1.0, np.abs(ref).max()) * s
    assert abs(float(host(rr)[0]) - rn @ rn) <= 1e-12 * (rn @ rn)


@pytest.mark.parametrize("dims,points,form", [((64, 64), 5, "csr"), ((20, 18, 16), 7, "stencil"),
                                              ((12, 11, 10), 27, "stencil")])
def test_power_method(dims, points, form):
    A, csr = operators(dims, points, form)
    v0 = I.power_start(csr.n)
    ref20, _ = O.power(csr, "jacobi", v0, 20, 0.0)
    ref, it = O.power(csr, "jacobi", v0, 50, 1e-3)
    with sstep.Solver(A, power_iters=20, power_tol=0.0, power_v0=dev(v0)) as S:
        info = S.get_basis_info()
        assert info["power_iters"] == 20
        assert abs(info["lambda_max"] - ref20) <= 1e-12 * ref20
    with sstep.Solver(A, power_iters=50, power_tol=1e-3, power_v0=dev(v0)) as S:
        info = S.get_basis_info()
        assert info["power_iters"] == it and abs(info["lambda_max"] - ref) <= 1e-12 * ref
    # NULL start vector: the library's own SplitMix64 seed-1 stream equals the input module's
    with sstep.Solver(A, power_iters=20, power_tol=0.0) as S:
        assert abs(S.get_basis_info()["lambda_max"] - ref20) <= 1e-12 * ref20


def test_gershgorin_lower_bound():
    rp, ci, v = I.poisson_csr((9, 8, 7), 7)
    d = np.zeros(rp.size - 1)
    for i in range(d.size):  # shift the diagonal by 2: rows become strictly dominant
        for k in range(rp[i], rp[i + 1]):
            if ci[k] == i:
                v[k] += 2.0
    csr = O.CSR(rp, ci, v)
    A = sstep.CSR(dev(rp), dev(ci), dev(v))
    with sstep.Solver(A, lambda_min=-1.0, lambda_max=2.0) as S:
        assert abs(S.get_basis_info()["lambda_min"] - O.gershgorin_lower(csr, "jacobi")) < 1e-15
    w = [-1.0] * 7
    w[3] = 8.0
    with sstep.Solver(sstep.Stencil(9, 8, 7, 7, weights=w), lambda_min=-1.0, lambda_max=2.0) as S:
        assert abs(S.get_basis_info()["lambda_min"] - O.gershgorin_lower(csr, "jacobi")) < 1e-15
    with sstep.Solver(sstep.Stencil(9, 8, 7, 7), lambda_min=-1.0, lambda_max=2.0) as S:
        assert S.get_basis_info()["lambda_min"] == 0.0


# ---------------------------------------------------------------- whole solves

def gpu_solve(A, b, x0=None, **kw):
    with sstep.Solver(A, **kw) as S:
        bd = dev(b)
        xd = dev(np.zeros_like(b) if x0 is None else x0)
        info = S.solve(bd, xd)
        hist = S.get_history()
        bi = S.get_basis_info()
        return host(xd), info, hist, bi


@pytest.mark.parametrize("dims,points,form,s,nu,algo,gram,K", [
    ((64, 64), 5, "csr", 4, 2, "onesync", "fgs", 40),        # the 64x64 workload, stable horizon
    ((64, 64), 5, "stencil", 4, 2, "onesync", "fgs", 40),
    ((64, 64), 5, "csr", 4, 2, "literal", "fgs", 40),
    ((30, 26, 22), 7, "stencil", 2, 3, "onesync", "fgs", 30),
    ((30, 26, 22), 7, "stencil", 8, 3, "onesync", "fgs", 12),
    ((30, 26, 22), 7, "csr", 4, 30, "onesync", "fgs", 25),
    ((30, 26, 22), 7, "stencil", 4, 30, "literal", "fgs", 25),
    ((19, 17, 15), 27, "stencil", 4, 30, "onesync", "fgs", 10),
    ((30, 26, 22), 7, "stencil", 4, 0, "onesync", "cholesky", 20),
    ((30, 26, 22), 7, "stencil", 1, 1, "onesync", "fgs", 60),
    # the operator form of the sweeps (equal to the oracle's sweeps up to rounding)
    ((64, 64), 5, "csr", 4, 2, "literal", "fgs_operator", 40),
    ((30, 26, 22), 7, "stencil", 4, 30, "literal", "fgs_operator", 25),
    ((30, 26, 22), 7, "stencil", 5, 3, "onesync", "fgs_operator", 12),
    ((30, 26, 22), 7, "stencil", 8, 3, "onesync", "fgs_operator", 12),
    ((30, 26, 22), 7, "stencil", 6, 30, "literal", "fgs_operator", 12)])
def test_solve_fixed_count(dims, points, form, s, nu, algo, gram, K):
    A, csr = operators(dims, points, form)
    xt, b = I.poisson_problem(dims, points)
    v0 = I.power_start(csr.n)
    x, info, hist, bi = gpu_solve(A, b, s=s, sweeps=nu, rtol=0.0, max_outer=K, algo=algo, gram=gram,
                                  power_iters=20, power_tol=0.0, power_v0=dev(v0), lambda_min=-1.0)
    assert info.status == sstep.NOT_CONVERGED and info.outer_iters == K
    ref = O.pcgs(csr, b, s=s, nu=nu, rtol=0.0, max_outer=K, algo=algo,
                 gram="fgs" if gram == "fgs_operator" else gram,
                 lambda_min=bi["lambda_min"], lambda_max=bi["lambda_max"], history=True)
    assert relerr(x, ref.x) <= 1e-9
    assert np.allclose(hist[1:K + 1], ref.hist[1:K + 1], rtol=1e-8)


@pytest.mark.parametrize("dims,points,form,s,nu,gram", [
    ((48, 40, 32), 7, "stencil", 4, 30, "fgs"), ((64, 64), 5, "csr", 4, 30, "fgs"),
    ((40, 36, 28), 7, "csr", 2, 0, "cholesky"), ((24, 22, 20), 27, "stencil", 4, 30, "fgs"),
    ((48, 40, 32), 7, "stencil", 4, 30, "fgs_operator")])
def test_solve_free_running(dims, points, form, s, nu, gram):
    A, csr = operators(dims, points, form)
    xt, b = I.poisson_problem(dims, points)
    x, info, hist, bi = gpu_solve(A, b, s=s, sweeps=nu, rtol=1e-8, gram=gram,
                                  power_v0=dev(I.power_start(csr.n)))
    ref = O.pcgs(csr, b, s=s, nu=nu, rtol=1e-8, algo="onesync",
                 gram="fgs" if gram == "fgs_operator" else gram,
                 lambda_min=bi["lambda_min"], lambda_max=bi["lambda_max"])
    assert info.status == sstep.OK and ref.status == O.OK
    assert abs(info.outer_iters - ref.iters) <= 1
    assert info.relres <= 1e-8 and info.relres_true <= 2e-8
    if info.outer_iters == ref.iters:
        assert relerr(x, ref.x) <= 1e-9


@pytest.mark.parametrize("dims,points,form,prec", [
    ((64, 64), 5, "csr", "jacobi"), ((40, 33, 27), 7, "stencil", "jacobi"),
    ((40, 33, 27), 7, "csr", "none"), ((21, 19, 17), 27, "stencil", "jacobi")])
def test_pcg(dims, points, form, prec):
    A, csr = operators(dims, points, form)
    xt, b = I.poisson_problem(dims, points)
    x, info, hist, _ = gpu_solve(A, b, algo="pcg", precond=prec, rtol=1e-8, lambda_max=2.0)
    ref = O.pcg(csr, b, rtol=1e-8, prec=prec, history=True)
    assert info.status == sstep.OK and abs(info.outer_iters - ref.iters) <= 1
    if info.outer_iters == ref.iters:
        assert relerr(x, ref.x) <= 1e-9
    K = 30
    x, info, hist, _ = gpu_solve(A, b, algo="pcg", precond=prec, rtol=0.0, max_outer=K, lambda_max=2.0)
    ref = O.pcg(csr, b, rtol=0.0, max_iters=K, prec=prec, history=True)
    assert relerr(x, ref.x) <= 1e-10
    assert np.allclose(hist[1:K + 1], ref.hist[1:K + 1], rtol=1e-9)


def test_workload_64x64_converges():
    """The 64x64 5-point workload (s = 4, nu = 2, 20 power iterations, Gershgorin lower bound)
    reaches rtol 1e-8 on the GPU; the count lies within the spread the oracle itself shows
    under 1-ulp perturbations of b (nu = 2 makes the outer iteration sensitive)."""
    dims = (64, 64)
    A, csr = operators(dims, 5, "csr")
    xt, b = I.poisson_problem(dims, 5)
    v0 = I.power_start(csr.n)
    x, info, hist, bi = gpu_solve(A, b, s=4, sweeps=2, rtol=1e-8, power_iters=20, power_tol=0.0,
                                  power_v0=dev(v0), lambda_min=-1.0)
    assert info.status == sstep.OK and info.relres <= 1e-8 and info.relres_true <= 2e-8
    counts = []
    for k in range(4):
        bb = b.copy()
        if k:
            bb[7 * k] = np.nextafter(bb[7 * k], np.inf)
        counts.append(O.pcgs(csr, bb, s=4, nu=2, rtol=1e-8, algo="onesync",
                             lambda_min=bi["lambda_min"], lambda_max=bi["lambda_max"]).iters)
    lo, hi = min(counts), max(counts)
    assert 0.8 * lo <= info.outer_iters <= 1.25 * hi, (info.outer_iters, counts)


def test_edge_cases():
    dims = (13, 12, 11)
    A, csr = operators(dims, 7, "stencil")
    xt, b = I.poisson_problem(dims, 7)
    n = csr.n
    with sstep.Solver(A, s=4, sweeps=2, lambda_max=2.0) as S:
        # b = 0 -> x = 0, no iterations
        x = dev(np.ones(n))
        info = S.solve(dev(np.zeros(n)), x)
        assert info.status == sstep.OK and info.outer_iters == 0 and float(x.abs().max()) == 0.0
        # x0 is the solution -> no iterations
        x = dev(xt)
        info = S.solve(dev(b), x)
        assert info.status == sstep.OK and info.outer_iters == 0
        # non-finite b
        bb = b.copy()
        bb[5] = np.nan
        info = S.solve(dev(bb), dev(np.zeros(n)), check=False)
        assert info.status == sstep.ERR_NONFINITE
        # host (numpy) buffers give the same answer as device buffers
        xh = np.zeros(n)
        ih = S.solve(b, xh)
        xd = dev(np.zeros(n))
        idd = S.solve(dev(b), xd)
        assert ih.outer_iters == idd.outer_iters and np.array_equal(xh, host(xd))
        # solving twice with the same handle is reproducible bit for bit
        xd2 = dev(np.zeros(n))
        S.solve(dev(b), xd2)
        assert torch.equal(xd, xd2)
    with sstep.Solver(A, s=3, sweeps=2, rtol=1e-14, max_outer=3, lambda_max=2.0) as S:
        info = S.solve(dev(b), dev(np.zeros(n)))
        assert info.status == sstep.NOT_CONVERGED and info.outer_iters == 3
    with sstep.Solver(A, s=3, sweeps=2, max_outer=0, lambda_max=2.0) as S:
        info = S.solve(dev(b), dev(np.zeros(n)))
        assert info.outer_iters == 0
    for bad in (dict(s=0), dict(s=17), dict(sweeps=-1), dict(algo="onesync", rtol=-1.0)):
        with pytest.raises(sstep.SstepError) as e:
            sstep.Solver(A, lambda_max=2.0, **bad)
        assert e.value.status == sstep.ERR_INVALID
    with pytest.raises(sstep.SstepError):
        sstep.Solver(sstep.Stencil(4, 4, 2, points=5), lambda_max=2.0)


def test_solve_batched():
    dims = (20, 17, 14)
    A, csr = operators(dims, 7, "stencil")
    bs = [I.poisson_problem(dims, 7, seed=k)[1] for k in range(3)]
    with sstep.Solver(A, s=4, sweeps=30, rtol=1e-9, power_v0=dev(I.power_start(csr.n))) as S:
        xs = [dev(np.zeros(csr.n)) for _ in bs]
        infos = S.solve_batched([dev(b) for b in bs], xs)
        for b, x, info in zip(bs, xs, infos):
            assert info.status == sstep.OK
            xs1 = dev(np.zeros(csr.n))
            S.solve(dev(b), xs1)
            assert torch.equal(x, xs1)


@pytest.fixture(scope="module")
def big_problem():
    """The 256^3 7-point workload the benchmark times (x_true seed 0, b = A x_true)."""
    dims = (256, 256, 256)
    csr = O.CSR(*I.poisson_csr(dims, 7))
    xt, b = I.poisson_problem(dims, 7)
    return dims, csr, b


def test_full_size_mpk_and_two_outer_iterations(big_problem):
    """At the benchmark's size and launch configuration: Algorithm 2 (s = 4) element by element,
    and two outer iterations of Algorithm 1 (literal form, nu = 3) against the oracle."""
    dims, csr, b = big_problem
    n = csr.n
    A = sstep.Stencil(*dims, points=7)
    s = 4
    with sstep.Solver(A, s=s, sweeps=3, rtol=0.0, max_outer=2, lambda_min=-1.0, power_iters=20,
                      power_tol=0.0, power_v0=dev(I.power_start(n))) as S:
        bi = S.get_basis_info()
        bd = dev(b)
        Z = torch.empty(s * n, dtype=torch.float64, device=DEV)
        AZ = torch.empty(s * n, dtype=torch.float64, device=DEV)
        S.mpk(bd, Z, AZ)
        Zg, AZg = host(Z).reshape(s, n), host(AZ).reshape(s, n)
        xd = dev(np.zeros(n))
        info = S.solve(bd, xd)
        x = host(xd)
    Zo, Po = O.mpk(csr, "jacobi", b, s, bi["c_alpha"], bi["c_sigma"], bi["c_gamma"])
    for j in range(s):
        assert np.max(np.abs(Zg[j] - Zo[j])) <= 1e-12 * (j + 1) * np.abs(Zo[j]).max()
        assert np.max(np.abs(AZg[j] - Po[j + 1])) <= 1e-12 * (j + 1) * np.abs(Po[j + 1]).max()
    del Zg, AZg, Zo, Po
    ref = O.pcgs(csr, b, s=s, nu=3, rtol=0.0, max_outer=2, algo="literal",
                 lambda_min=bi["lambda_min"], lambda_max=bi["lambda_max"])
    assert info.outer_iters == 2
    assert relerr(x, ref.x) <= 1e-9
