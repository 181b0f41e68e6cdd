"""Pins of the oracle's aggregation AMG (oracle/amg.c) against closed forms and identities.

The paper uses an external AMG as the black-box preconditioner M (Section 5); amg.c defines
the concrete one (greedy pairwise matching twice per level, unsmoothed aggregation, Galerkin
coarse operators, l1-Jacobi smoothing, dense Cholesky coarse solve, V-cycle).  Nothing here
re-runs the oracle's own loops: the checks are closed-form matchings, the Galerkin identity,
exactness on one level, the two-level error-propagation identity, symmetry and definiteness.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_09790_gb300 import inputs as I


def dense_to_csr(M):
    rp, ci, v = [0], [], []
    for i in range(M.shape[0]):
        for j in np.flatnonzero(M[i]):
            ci.append(j)
            v.append(M[i, j])
        rp.append(len(ci))
    return O.CSR(np.array(rp, dtype=np.int64), np.array(ci, dtype=np.int32), np.array(v))


def q1_small(dims=(7, 6, 5), seed=3):
    (rp, ci, v), _, _, _ = I.q1_lognormal_problem(dims, sigma=1.0, corr=2.0, seed=seed)
    return O.CSR(rp, ci, v)


def test_match_chain_closed_form():
    n = 9
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    agg, nc = O.amg_match(dense_to_csr(T))
    assert nc == 5 and list(agg) == [0, 0, 1, 1, 2, 2, 3, 3, 4]


def test_match_grid_pairs_along_x():
    # 2D 5-point Poisson, all couplings equal: ties go to the lower index, i.e. the +x neighbour
    agg, nc = O.amg_match(O.CSR(*I.poisson_csr((6, 4), 5)))
    assert nc == 12 and np.array_equal(agg, np.arange(24) // 2)


def test_match_takes_the_strongest_coupling():
    M = np.array([[4.0, -1.0, -3.0], [-1.0, 4.0, 0.0], [-3.0, 0.0, 4.0]])
    agg, nc = O.amg_match(dense_to_csr(M))
    assert nc == 2 and list(agg) == [0, 1, 0]
    # a positive off-diagonal entry never pairs
    M = np.array([[4.0, 1.0], [1.0, 4.0]])
    agg, nc = O.amg_match(dense_to_csr(M))
    assert nc == 2 and list(agg) == [0, 1]


def test_match_is_a_maximal_matching():
    A = q1_small()
    agg, nc = O.amg_match(A)
    size = np.bincount(agg, minlength=nc)
    assert size.max() <= 2 and size.min() >= 1
    D = A.dense()
    single = np.flatnonzero(size[agg] == 1)
    # no two singletons are coupled by a negative entry (else greedy would have paired them)
    sub = D[np.ix_(single, single)] - np.diag(np.diag(D)[single])
    assert not np.any(sub < 0)
    # every pair is coupled by a negative entry
    for c in np.flatnonzero(size == 2):
        i, j = np.flatnonzero(agg == c)
        assert D[i, j] < 0
    # numbering follows the lowest row of each aggregate
    first = [np.flatnonzero(agg == c).min() for c in range(nc)]
    assert first == sorted(first)


def test_galerkin_identity():
    A = q1_small()
    agg, nc = O.amg_match(A)
    Ac = O.amg_galerkin(A, agg, nc)
    P = np.zeros((A.n, nc))
    P[np.arange(A.n), agg] = 1.0
    rng = np.random.default_rng(0)
    for _ in range(3):
        u, v = rng.standard_normal(nc), rng.standard_normal(nc)
        lhs = u @ O.spmv(Ac, v)
        rhs = (P @ u) @ O.spmv(A, P @ v)
        assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(A.dense()) * np.linalg.norm(u) * np.linalg.norm(v)
    D = Ac.dense()
    assert np.allclose(D, D.T, rtol=0, atol=1e-14 * np.abs(D).max())
    assert np.all(np.diff(Ac.rowptr) > 0)
    for i in range(nc):  # columns sorted within rows
        c = Ac.colind[Ac.rowptr[i]:Ac.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_single_level_is_an_exact_solve():
    A = q1_small((6, 5, 4))
    M = O.AMG(A, coarse_max=A.n)
    assert M.nlevels == 1
    b = I.uniform_pm1(4, A.n)
    x = M.apply(b)
    assert np.linalg.norm(O.spmv(A, x) - b) <= 1e-12 * np.linalg.norm(b)


def dense_inverse(M, n):
    return np.column_stack([M.apply(e) for e in np.eye(n)])


def test_two_level_error_propagation_identity():
    """With level 1 the coarsest, I - M^{-1}A = (I - D^{-1}A)(I - P A_c^{-1} P^T A)(I - D^{-1}A),
    D = diag(sum_j |a_ij|): the symmetric two-grid cycle with one l1-Jacobi sweep on each side."""
    A = q1_small((6, 5, 4))
    M = O.AMG(A, coarse_max=A.n // 3)
    assert M.nlevels == 2
    A0, agg = M.level(0)
    A1, _ = M.level(1)
    Ad = A.dense()
    n, nc = A.n, A1.n
    P = np.zeros((n, nc))
    P[np.arange(n), agg] = 1.0
    Dinv = np.diag(1.0 / np.abs(Ad).sum(axis=1))
    Ac = P.T @ Ad @ P
    assert np.allclose(A1.dense(), Ac, rtol=0, atol=1e-13 * np.abs(Ac).max())
    S = np.eye(n) - Dinv @ Ad
    E = S @ (np.eye(n) - P @ np.linalg.solve(Ac, P.T @ Ad)) @ S
    Minv = dense_inverse(M, n)
    assert np.abs((np.eye(n) - Minv @ Ad) - E).max() <= 1e-11


def test_vcycle_is_symmetric_positive_definite():
    A = q1_small((8, 7, 6))
    M = O.AMG(A, coarse_max=20)
    assert M.nlevels >= 3
    Minv = dense_inverse(M, A.n)
    assert np.abs(Minv - Minv.T).max() <= 1e-12 * np.abs(Minv).max()
    assert np.linalg.eigvalsh(0.5 * (Minv + Minv.T)).min() > 0
    # as a stationary iteration it converges: spectrum of M^{-1}A inside (0, 2)
    lam = np.linalg.eigvals(Minv @ A.dense()).real
    assert lam.min() > 0 and lam.max() < 2


def test_amg_preconditioning_beats_jacobi():
    dims = (16, 16, 16)
    A = O.CSR(*I.poisson_csr(dims, 7))
    xt, b = I.poisson_problem(dims, 7)
    M = O.AMG(A, coarse_max=64)
    ra = O.pcg(A, b, rtol=1e-8, prec="amg", amg=M)
    rj = O.pcg(A, b, rtol=1e-8, prec="jacobi")
    assert ra.status == O.OK and ra.iters < 0.6 * rj.iters
    rs = O.pcgs(A, b, s=4, nu=30, rtol=1e-8, prec="amg", amg=M, power_iters=20, power_tol=0.0)
    assert rs.status == O.OK and rs.relres_true <= 2e-8
    assert np.linalg.norm(rs.x - xt) <= 1e-5 * np.linalg.norm(xt)


def test_amg_rejects_bad_input():
    with pytest.raises(ValueError):
        O.AMG(dense_to_csr(np.array([[0.0, 1.0], [1.0, 0.0]])), coarse_max=1)
