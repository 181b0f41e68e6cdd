"""The FP64 oracle checked against closed forms, the paper's theorems and dense solves."""
import numpy as np
import pytest

import oracle as O
from paper_2603_09790_gb300 import inputs as I

from . import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin()


def test_splitmix64_published_outputs():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")
    want = [int(l, 16) for l in open(path) if l.strip() and not l.startswith("#")]
    got = [int(v) for v in I.splitmix64(0, len(want))]
    assert got == want
    # stream offsets: outputs start.. of the same stream
    assert [int(v) for v in I.splitmix64(0, 2, start=2)] == want[2:4]
    u = I.uniform_pm1(0, 1000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.1


def test_csr_layout():
    rp, ci, v = I.poisson_csr((4, 3, 2), 7)
    assert rp.dtype == np.int64 and ci.dtype == np.int32
    for i in range(rp.size - 1):
        cols = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cols) > 0)
    A = O.CSR(rp, ci, v).dense()
    assert np.allclose(A, A.T)
    # nnz of the 64x64 5-point matrix quoted in the workload description
    rp, ci, v = I.poisson_csr((64, 64), 5)
    assert ci.size == 20224


def test_b_equals_A_xtrue():
    for dims, pts in [((6, 5), 5), ((4, 5, 3), 7), ((3, 4, 5), 27)]:
        xt, b = I.poisson_problem(dims, pts)
        A = O.CSR(*I.poisson_csr(dims, pts))
        assert np.allclose(O.spmv(A, xt), b, atol=1e-14)


def test_edge_cases():
    A = O.CSR(*I.poisson_csr((5, 5), 5))
    xt, b = I.poisson_problem((5, 5), 5)
    # b = 0 -> x = 0, no iterations
    r = O.pcgs(A, np.zeros(A.n), np.ones(A.n), s=3, nu=2, lambda_max=2.0)
    assert r.status == O.OK and r.iters == 0 and np.all(r.x == 0)
    r = O.pcg(A, np.zeros(A.n), np.ones(A.n))
    assert r.status == O.OK and r.iters == 0 and np.all(r.x == 0)
    # x0 already the solution -> zero iterations
    r = O.pcgs(A, b, xt, s=3, nu=2, rtol=1e-8, lambda_max=2.0)
    assert r.status == O.OK and r.iters == 0
    # iteration cap -> NOT_CONVERGED, x and info still filled
    r = O.pcgs(A, b, s=2, nu=2, rtol=1e-14, max_outer=2, lambda_max=2.0)
    assert r.status == O.NOT_CONVERGED and r.iters == 2 and r.relres < 1
    # non-finite right-hand side
    bb = b.copy()
    bb[3] = np.nan
    r = O.pcgs(A, bb, s=2, nu=2, lambda_max=2.0)
    assert r.status == O.ERR_NONFINITE
    # non-SPD Gram matrix in the reduced solve
    with pytest.raises(FloatingPointError):
        O.fgs(np.array([[1.0, 0.0], [0.0, -1.0]]), np.ones(2), 2)


def test_onesync_and_literal_share_the_first_steps_at_nu2():
    """At nu = 2 the two forms agree to rounding over the first outer iterations."""
    A = O.CSR(*I.poisson_csr((64, 64), 5))
    xt, b = I.poisson_problem((64, 64), 5)
    v0 = I.power_start(A.n)
    kw = dict(s=4, nu=2, rtol=0.0, max_outer=20, power_v0=v0, power_iters=20, power_tol=0.0)
    lit = O.pcgs(A, b, algo="literal", **kw)
    one = O.pcgs(A, b, algo="onesync", **kw)
    assert np.linalg.norm(lit.x - one.x) <= 1e-10 * np.linalg.norm(lit.x)


def _doubling_operator(W, nu):
    """P_nu = (I + M + ... + M^{nu-1}) T with T = (D + L)^{-1}, M = I - T W, formed from the
    binary digits of nu by doubling (S_2m = S_m + M^m S_m, S_{m+1} = I + M S_m): the operator
    form of the FGS sweeps, written here in numpy from the sweep's definition."""
    s = W.shape[0]
    T = np.linalg.inv(np.tril(W))
    M = np.eye(s) - T @ W
    if nu == 0:
        return np.zeros((s, s))
    S, Pw = np.eye(s), M.copy()
    for bit in bin(nu)[3:]:
        S, Pw = S + Pw @ S, Pw @ Pw
        if bit == "1":
            S, Pw = np.eye(s) + M @ S, Pw @ M
    return S @ T


@pytest.mark.parametrize("s,nu", [(1, 1), (2, 2), (3, 3), (4, 5), (4, 30), (5, 7), (8, 30), (8, 1),
                                  (6, 0), (7, 64)])
def test_fgs_sweeps_are_a_linear_operator(s, nu):
    """The reading behind the operator form of the reduced solves: nu FGS sweeps from 0 are a
    linear map of the right-hand side (the oracle's sweeps on a combination of right-hand sides
    equal the combination of its sweeps), and that map is P_nu formed by doubling.  A wrong
    splitting (D + U for D + L), a sweep miscounted in the binary digits or the factor T left
    out fails it."""
    rng = np.random.default_rng(50 + 10 * s + nu)
    Qm, _ = np.linalg.qr(rng.standard_normal((s, s)))
    W = Qm @ np.diag(np.geomspace(1.0, 40.0, s)) @ Qm.T
    d = rng.uniform(0.5, 2.0, s)
    W = (W * np.outer(d, d) + (W * np.outer(d, d)).T) / 2
    cols = np.column_stack([O.fgs(W, np.eye(s)[:, j], nu) for j in range(s)])
    b1, b2 = rng.standard_normal(s), rng.standard_normal(s)
    lin = O.fgs(W, 2.5 * b1 - 0.75 * b2, nu)
    assert np.allclose(lin, 2.5 * O.fgs(W, b1, nu) - 0.75 * O.fgs(W, b2, nu), rtol=1e-11, atol=1e-12)
    P = _doubling_operator(W, nu)
    scale = max(1.0, np.abs(cols).max())
    assert np.max(np.abs(P - cols)) <= 1e-11 * scale
    assert np.allclose(P @ b1, O.fgs(W, b1, nu), rtol=1e-10, atol=1e-12 * scale)
