"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each ``pin_*`` function raises AssertionError when the oracle disagrees with something
computed without the oracle's own code: closed-form spectra of the Dirichlet Poisson
matrices, Chebyshev polynomials evaluated by numpy on an eigendecomposition, the paper's
Theorem 1 / Corollary 1 / Corollary 2 (moment representation of the Chebyshev Gram
matrix), Proposition 1 (FGS residual), Theorem 2 (Ruhe's FGS/MGS equivalence), the
optimality of (block) conjugate gradients over a Krylov space built by QR, and dense
direct solves.  ``tests/test_oracle_pins.py`` runs them; ``tests/test_oracle_mutations.py``
plants mistakes in a copy of the oracle and checks that some pin fails.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import chebyshev as npcheb

import oracle as O
from paper_2603_09790_gb300 import inputs as I

# ---------------------------------------------------------------- closed-form spectra


def sine_basis(N: int) -> np.ndarray:
    """Orthonormal DST-I basis: row k is sqrt(2/(N+1)) sin((k+1)(i+1) pi/(N+1))."""
    k = np.arange(1, N + 1)[:, None]
    i = np.arange(1, N + 1)[None, :]
    return np.sqrt(2.0 / (N + 1)) * np.sin(k * i * np.pi / (N + 1))


def poisson_eig(dims, points):
    """Eigenvalues and orthonormal eigenvectors (rows) of the Dirichlet Poisson matrix.

    5/7-point: lambda = sum_d (2 - 2 cos theta_d); 27-point: lambda = 27 - prod_d (1 + 2 cos theta_d).
    """
    nx, ny, nz = (tuple(dims) + (1,))[:3]
    Sx, Sy, Sz = sine_basis(nx), sine_basis(ny), sine_basis(nz)
    cx = np.cos(np.arange(1, nx + 1) * np.pi / (nx + 1))
    cy = np.cos(np.arange(1, ny + 1) * np.pi / (ny + 1))
    cz = np.cos(np.arange(1, nz + 1) * np.pi / (nz + 1))
    lams, vecs = [], []
    for c in range(nz):
        for b in range(ny):
            for a in range(nx):
                if points == 27:
                    lam = 27.0 - (1 + 2 * cx[a]) * (1 + 2 * cy[b]) * (1 + 2 * cz[c])
                elif points == 7:
                    lam = (2 - 2 * cx[a]) + (2 - 2 * cy[b]) + (2 - 2 * cz[c])
                else:
                    lam = (2 - 2 * cx[a]) + (2 - 2 * cy[b])
                lams.append(lam)
                vecs.append(np.kron(Sz[c], np.kron(Sy[b], Sx[a])))
    return np.array(lams), np.array(vecs)


def csr_of(dims, points, diag_shift=None):
    rp, ci, v = I.poisson_csr(dims, points)
    v = v.copy()
    if diag_shift is not None:
        n = rp.size - 1
        for i in range(n):
            for k in range(rp[i], rp[i + 1]):
                if ci[k] == i:
                    v[k] += diag_shift[i]
    return O.CSR(rp, ci, v)


def cheb_T(j: int, x: np.ndarray) -> np.ndarray:
    return npcheb.chebval(x, [0.0] * j + [1.0])


def krylov_minimizer(Adense, Minv_diag, b, x0, m):
    """argmin over x0 + K_m(M^{-1}A, M^{-1}r0) of the A-norm error, with K built by QR."""
    r0 = b - Adense @ x0
    v = Minv_diag * r0
    K = np.zeros((b.size, 0))
    for _ in range(m):
        for _ in range(2):  # re-orthogonalise
            v = v - K @ (K.T @ v)
        v = v / np.linalg.norm(v)
        K = np.column_stack([K, v])
        v = Minv_diag * (Adense @ v)
    y = np.linalg.solve(K.T @ Adense @ K, K.T @ r0)
    return x0 + K @ y


# ---------------------------------------------------------------- pins


def pin_spmv_eigenpairs():
    """A v = lambda v for the sine modes of each stencil (catches weights, indices, transposes)."""
    for dims, pts in [((5, 4), 5), ((4, 3, 5), 7), ((3, 4, 3), 27)]:
        A = csr_of(dims, pts)
        lam, V = poisson_eig(dims, pts)
        for k in range(0, lam.size, max(1, lam.size // 7)):
            y = O.spmv(A, V[k])
            assert np.allclose(y, lam[k] * V[k], atol=1e-12), (dims, pts, k)


def pin_jacobi_and_prec():
    rng = np.random.default_rng(3)
    shift = rng.uniform(0.5, 3.0, 24)
    A = csr_of((4, 3, 2), 7, shift)
    d = O.jacobi_dinv(A)
    assert np.allclose(d, 1.0 / (6.0 + shift), rtol=1e-15)
    x = rng.standard_normal(24)
    assert np.allclose(O.prec_apply("jacobi", d, x), x / (6.0 + shift), rtol=1e-15)
    assert np.array_equal(O.prec_apply("none", None, x), x)


def pin_gershgorin():
    # interior rows of the Poisson matrices have zero row sum: the bound is exactly 0
    for dims, pts in [((6, 5), 5), ((4, 4, 4), 7), ((4, 4, 4), 27)]:
        assert O.gershgorin_lower(csr_of(dims, pts), "jacobi") == 0.0
    # strictly diagonally dominant rows: 1 - off/d with d = 6 + 2, off = 6 on every 7-point row
    A = csr_of((4, 4, 4), 7, np.full(64, 2.0))
    assert abs(O.gershgorin_lower(A, "jacobi") - (1.0 - 6.0 / 8.0)) < 1e-15


def pin_power_method():
    """lambda_max(D^{-1}A) = 1 + cos(pi/(N+1)) for 5/7-point Poisson; the norm estimator is a
    lower bound for a symmetric M^{-1}A and converges to it; the paper's stop rule is honoured."""
    for dims, pts in [((12, 12), 5), ((8, 8, 8), 7)]:
        A = csr_of(dims, pts)
        exact = 1.0 + np.cos(np.pi / (dims[0] + 1))
        v0 = I.power_start(A.n)
        lam20, it20 = O.power(A, "jacobi", v0, 20, 0.0)
        assert it20 == 20 and lam20 <= exact * (1 + 1e-14) and lam20 > 0.9 * exact
        lam_inf, _ = O.power(A, "jacobi", v0, 3000, 0.0)
        assert abs(lam_inf - exact) < 1e-6 * exact
        lam, it = O.power(A, "jacobi", v0, 50, 1e-3)
        assert 2 <= it <= 50
        prev, _ = O.power(A, "jacobi", v0, it - 1, 0.0)
        if it < 50:
            assert abs(lam - prev) < 1e-3 * abs(lam)
        if it > 2:
            prev2, _ = O.power(A, "jacobi", v0, it - 2, 0.0)
            assert abs(prev - prev2) >= 1e-3 * abs(prev)


def pin_cheb_scalars():
    """A_hat = c_alpha M^{-1}A - c_sigma I maps [lmin, lmax] onto [-1, 1]; c_gamma = 1."""
    for lmin, lmax in [(0.0, 2.0), (0.1, 1.9), (0.25, 7.5)]:
        a, s, g = O.cheb(lmin, lmax)
        assert abs(a * lmin - s + 1.0) < 1e-14 and abs(a * lmax - s - 1.0) < 1e-14 and g == 1.0


def pin_mpk_chebyshev_polynomials():
    """Z[:, j] = T_j(A_hat) M^{-1} r and P = [r, A Z] (Section 2, Algorithm 2), checked by
    evaluating T_j with numpy on the eigendecomposition of B = D^{-1/2} A D^{-1/2}."""
    rng = np.random.default_rng(5)
    for prec, shift, (lmin, lmax), s in [("jacobi", rng.uniform(0.2, 2.0, 36), (0.1, 1.9), 5),
                                         ("none", None, (0.0, 12.0), 4),
                                         ("jacobi", None, (0.0, 1.7), 6)]:
        A = csr_of((4, 3, 3), 7, shift)
        Ad = A.dense()
        d = np.diag(Ad) if prec == "jacobi" else np.ones(A.n)
        B = Ad / np.sqrt(np.outer(d, d))
        w, U = np.linalg.eigh(B)
        ca, cs, cg = O.cheb(lmin, lmax)
        r = rng.standard_normal(A.n)
        Z, P = O.mpk(A, prec, r, s, ca, cs, cg)
        y = U.T @ (r / np.sqrt(d))
        for j in range(s):
            zj = (U @ (cheb_T(j, ca * w - cs) * y)) / np.sqrt(d)
            assert np.allclose(Z[j], zj, rtol=1e-11, atol=1e-11 * np.abs(zj).max()), (prec, j)
        assert np.array_equal(P[0], r)
        for j in range(s):
            assert np.allclose(P[j + 1], Ad @ Z[j], rtol=1e-12, atol=1e-12 * np.abs(P[j + 1]).max())


def pin_gram_moments():
    """Theorem 1 (Eq. gram-moments), Corollary 1 and Corollary 2 for M = I, and the
    symmetric-representative remark for Jacobi, with moments from the closed-form spectrum."""
    dims, pts = (7, 6), 5
    A = csr_of(dims, pts)
    lam, V = poisson_eig(dims, pts)
    rng = np.random.default_rng(11)
    r = rng.standard_normal(A.n)
    for prec, scale in [("none", 1.0), ("jacobi", 4.0)]:
        # for Jacobi, B = D^{-1/2} A D^{-1/2} = A / 4 with the same eigenvectors
        lamB = lam / scale
        lmin, lmax = 0.0, lamB.max() * 1.05
        ca, cs, cg = O.cheb(lmin, lmax)
        s = 6
        Z, P = O.mpk(A, prec, r, s, ca, cs, cg)
        c = V @ (r / np.sqrt(scale))           # coefficients of D^{-1/2} r in the eigenbasis
        lhat = ca * lamB - cs
        mu0 = np.array([np.sum(c ** 2 * cheb_T(p, lhat)) for p in range(2 * s)])
        muA = np.array([np.sum(lamB * c ** 2 * cheb_T(p, lhat)) for p in range(2 * s)])
        Y = Z * np.sqrt(scale)                 # y_j = D^{1/2} z_j
        W0 = O.gram(Y, Y)
        WA = O.gram(Z, P[1:])                  # z_i^T A z_j
        for i in range(s):
            for j in range(s):
                e0 = 0.5 * (mu0[i + j] + mu0[abs(i - j)])
                eA = 0.5 * (muA[i + j] + muA[abs(i - j)])
                assert abs(W0[i, j] - e0) <= 1e-11 * abs(mu0[0]), (prec, i, j)
                assert abs(WA[i, j] - eA) <= 1e-11 * abs(muA[0]), (prec, i, j)
        rr = r / np.sqrt(scale)
        assert abs(mu0[0] - rr @ rr) < 1e-11 * mu0[0]
        assert abs(muA[0] - rr @ (A.dense() / scale) @ rr) < 1e-11 * muA[0]
        for W in (W0, WA):
            dW = np.sqrt(np.diag(W))
            Wc = W / np.outer(dW, dW)
            assert np.allclose(np.diag(Wc), 1.0, atol=1e-14) and np.all(np.abs(Wc) <= 1.0 + 1e-12)


def _spd(s, rng, cond=30.0):
    G = rng.standard_normal((s, s))
    Qm, _ = np.linalg.qr(G)
    ev = np.geomspace(1.0, cond, s)
    W = Qm @ np.diag(ev) @ Qm.T
    dd = rng.uniform(0.5, 4.0, s)
    return (W * np.outer(dd, dd) + (W * np.outer(dd, dd)).T) / 2


def pin_fgs_prop1():
    """Proposition 1: after nu sweeps from 0, the normalised residual equals
    (-1)^nu (L^T (I+L)^{-1})^nu m_tilde, with W_c = D^{-1/2} W D^{-1/2} = I + L + L^T."""
    rng = np.random.default_rng(17)
    for s in (2, 4, 7):
        W = _spd(s, rng)
        m = rng.standard_normal(s)
        d = np.sqrt(np.diag(W))
        Wc = W / np.outer(d, d)
        L = np.tril(Wc, -1)
        H = L.T @ np.linalg.inv(np.eye(s) + L)
        mt = m / d
        for nu in range(0, 6):
            a = O.fgs(W, m, nu)
            rho = mt - Wc @ (d * a)
            expect = ((-1) ** nu) * np.linalg.matrix_power(H, nu) @ mt
            assert np.allclose(rho, expect, atol=1e-12 * np.linalg.norm(mt)), (s, nu)


def _prop1_residual(W, M, nu):
    """m - W alpha^(nu) for each column m of M, from Proposition 1 alone: with
    D = diag(W), W_c = D^{-1/2} W D^{-1/2} = I + L + L^T and m_tilde = D^{-1/2} m, the
    normalised residual after nu sweeps from 0 is (-1)^nu (L^T (I+L)^{-1})^nu m_tilde, and
    m - W alpha = D^{1/2} times it."""
    s = W.shape[0]
    d = np.sqrt(np.diag(W))
    L = np.tril(W / np.outer(d, d), -1)
    H = L.T @ np.linalg.inv(np.eye(s) + L)
    Mt = np.asarray(M, dtype=np.float64).reshape(s, -1) / d[:, None]
    return d[:, None] * (((-1) ** nu) * np.linalg.matrix_power(H, nu) @ Mt)


def _eta_prop1(W, M, nu):
    """Section 3.3's eta (2-norm for one column, Frobenius for a block) from Proposition 1."""
    R = _prop1_residual(W, M, nu)
    return np.linalg.norm(R) / np.linalg.norm(np.asarray(M, dtype=np.float64))


def _fgs_splitting(W, m, nu):
    """nu forward Gauss-Seidel sweeps from 0 in matrix form, (D + L_W) a_new = m - L_W^T a."""
    DL = np.tril(W)
    U = np.triu(W, 1)
    a = np.zeros_like(m)
    for _ in range(nu):
        a = np.linalg.solve(DL, m - U @ a)
    return a


def pin_eta_closed_form():
    """eta_alpha and eta_beta (Section 3.3) after nu FGS sweeps equal the closed form of
    Proposition 1; nu = 0 gives 1; exact (Cholesky) solves give ~0."""
    rng = np.random.default_rng(41)
    for s in (2, 4, 7):
        W = _spd(s, rng, cond=50.0)
        m = rng.standard_normal(s)
        B = rng.standard_normal((s, s))
        for nu in (0, 1, 2, 3, 30):
            a = O.fgs(W, m, nu)
            e = O.reduced_relres(W, m, a)
            assert abs(e - _eta_prop1(W, m, nu)) <= 1e-12 * max(1.0, e), (s, nu)
            X = np.column_stack([O.fgs(W, B[:, c], nu) for c in range(s)])
            eb = O.reduced_relres(W, B, X)
            assert abs(eb - _eta_prop1(W, B, nu)) <= 1e-12 * max(1.0, eb), (s, nu)
        assert O.reduced_relres(W, m, np.zeros(s)) == 1.0
        assert O.reduced_relres(W, m, O.chol_solve(W, m)) < 1e-13
        X = np.column_stack([O.chol_solve(W, B[:, c]) for c in range(s)])
        assert O.reduced_relres(W, B, X) < 1e-13


def pin_eta_in_pcgs():
    """The eta_alpha_k, eta_beta_k that PCG-S records are Section 3.3's residuals of its own
    reduced systems: W_k = Q_k^T A Q_k with m_k = Q_k^T r^(k), and the conjugation system
    W_k beta_k = -Q_k^T A Z_{k+1} solved with the same W_k.  Everything on the right-hand side
    is built here from a dense A: the Chebyshev basis by numpy on the eigendecomposition of
    D^{-1/2} A D^{-1/2}, FGS in its matrix-splitting form, eta from Proposition 1."""
    A = csr_of((5, 4, 3), 7, np.linspace(0.1, 1.3, 60))
    Ad = A.dense()
    n = A.n
    dg = np.diag(Ad)
    w, U = np.linalg.eigh(Ad / np.sqrt(np.outer(dg, dg)))
    lmax = float(w.max()) * 1.01
    ca, cs, cg = O.cheb(0.0, lmax)
    rng = np.random.default_rng(43)
    b = rng.standard_normal(n)

    def basis(r, s):
        y = U.T @ (r / np.sqrt(dg))
        return np.column_stack([(U @ (cheb_T(j, ca * w - cs) * y)) / np.sqrt(dg) for j in range(s)])

    for s, nu in ((3, 2), (4, 3)):
        for algo in ("literal", "onesync"):
            res = O.pcgs(A, b, s=s, nu=nu, rtol=0.0, max_outer=3, algo=algo, lambda_max=lmax,
                         history=True)
            r = b.copy()
            Q = basis(r, s)
            for k in range(3):
                W = Q.T @ Ad @ Q
                m = Q.T @ r
                ea = _eta_prop1(W, m, nu)
                assert abs(res.eta_a[k] - ea) <= 1e-9 * ea, (s, nu, algo, k, res.eta_a[k], ea)
                a = _fgs_splitting(W, m, nu)
                r = r - Ad @ (Q @ a)
                if k == 2:
                    break
                Z = basis(r, s)
                B = -(Q.T @ Ad @ Z)
                eb = _eta_prop1(W, B, nu)
                assert abs(res.eta_b[k] - eb) <= 1e-9 * eb, (s, nu, algo, k, res.eta_b[k], eb)
                beta = np.column_stack([_fgs_splitting(W, B[:, c], nu) for c in range(s)])
                Q = Z + Q @ beta


def pin_fgs_limit_and_cholesky():
    """nu -> infinity: FGS converges to the dense solution (the Cholesky solve)."""
    rng = np.random.default_rng(19)
    for s in (3, 6, 10):
        W = _spd(s, rng, cond=8.0)
        m = rng.standard_normal(s)
        ref = np.linalg.solve(W, m)
        assert np.allclose(O.chol_solve(W, m), ref, rtol=1e-12, atol=1e-13)
        assert np.allclose(O.fgs(W, m, 600), ref, rtol=1e-9, atol=1e-10)


def pin_ruhe():
    """Theorem 2 (Ruhe): one sweep on W alpha = e1 (W = P^T P, unit columns) gives
    P alpha = MGS-type projection of p1 against p2..ps; also in the A-inner product."""
    rng = np.random.default_rng(23)
    n, s = 40, 6
    Pm = rng.standard_normal((n, s))
    Pm /= np.linalg.norm(Pm, axis=0)
    a = O.fgs(Pm.T @ Pm, np.eye(s)[0], 1)
    v = Pm[:, 0].copy()
    for j in range(1, s):
        v = v - (Pm[:, j] @ v) * Pm[:, j]
    assert np.allclose(Pm @ a, v, atol=1e-13)
    A = csr_of((5, 4, 2), 7)
    Ad = A.dense()
    Qm = rng.standard_normal((A.n, s))
    Qm /= np.sqrt(np.einsum("ij,ij->j", Qm, Ad @ Qm))
    a = O.fgs(Qm.T @ Ad @ Qm, np.eye(s)[0], 1)
    v = Qm[:, 0].copy()
    for j in range(1, s):
        v = v - (Qm[:, j] @ (Ad @ v)) * Qm[:, j]
    assert np.allclose(Qm @ a, v, atol=1e-12)


def pin_gram_products():
    """X^T Y on orthonormal sine vectors is the identity; on scaled ones it is diagonal."""
    S = sine_basis(9)
    G = O.gram(S[:4], S[:4])
    assert np.allclose(G, np.eye(4), atol=1e-14)
    G = O.gram(S[:3], 2.0 * S[2:6])
    expect = np.zeros((3, 4))
    expect[2, 0] = 2.0
    assert np.allclose(G, expect, atol=1e-14)


def pin_pcg_distinct_eigenvalues():
    """CG on a matrix with 3 distinct eigenvalues converges in 3 iterations."""
    rng = np.random.default_rng(29)
    n = 12
    U, _ = np.linalg.qr(rng.standard_normal((n, 2)))
    Ad = 2.0 * np.eye(n) + U @ np.diag([3.0, 7.0]) @ U.T
    rp = np.arange(0, n * n + 1, n, dtype=np.int64)
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    A = O.CSR(rp, ci, Ad.reshape(-1))
    b = rng.standard_normal(n)
    res = O.pcg(A, b, rtol=1e-10, prec="none")
    assert res.status == O.OK and res.iters == 3
    assert np.allclose(res.x, np.linalg.solve(Ad, b), rtol=1e-10)


def pin_pcg_krylov_optimality():
    """PCG iterate k is the A-norm minimiser over x0 + K_k(M^{-1}A, M^{-1}r0)."""
    rng = np.random.default_rng(31)
    A = csr_of((4, 3, 3), 7, rng.uniform(0.1, 2.0, 36))
    Ad = A.dense()
    b = rng.standard_normal(A.n)
    x0 = rng.standard_normal(A.n)
    dinv = 1.0 / np.diag(Ad)
    xs = np.linalg.solve(Ad, b)
    errs = []
    for k in range(1, 7):
        res = O.pcg(A, b, x0, rtol=0.0, max_iters=k, prec="jacobi")
        ref = krylov_minimizer(Ad, dinv, b, x0, k)
        assert np.allclose(res.x, ref, rtol=1e-8, atol=1e-9 * np.abs(ref).max()), k
        e = res.x - xs
        errs.append(e @ Ad @ e)
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))


def pin_pcgs_block_cg_optimality():
    """With exact (Cholesky) reduced solves, PCG-S outer iterate k is the A-norm minimiser
    over the Krylov space of dimension k*s (the alignment the paper uses in Section 3.3)."""
    rng = np.random.default_rng(37)
    A = csr_of((5, 4, 3), 7, rng.uniform(0.1, 2.0, 60))
    Ad = A.dense()
    b = rng.standard_normal(A.n)
    dinv = 1.0 / np.diag(Ad)
    lmax = float(np.max(np.linalg.eigvals(dinv[:, None] * Ad).real))
    for algo in ("literal", "onesync"):
        for s in (2, 3):
            for k in (1, 2):
                res = O.pcgs(A, b, s=s, nu=0, rtol=0.0, max_outer=k, algo=algo, gram="cholesky",
                             lambda_max=lmax)
                ref = krylov_minimizer(Ad, dinv, b, np.zeros(A.n), k * s)
                assert np.allclose(res.x, ref, rtol=1e-7, atol=1e-8 * np.abs(ref).max()), (algo, s, k)


def pin_pcgs_s1_is_pcg():
    """s = 1: the 1x1 FGS solve is exact and PCG-S reproduces classical PCG."""
    A = csr_of((9, 8), 5)
    xt, b = I.poisson_problem((9, 8), 5)
    ref = O.pcg(A, b, rtol=1e-10)
    for algo in ("literal", "onesync"):
        res = O.pcgs(A, b, s=1, nu=1, rtol=1e-10, algo=algo, lambda_max=2.0)
        assert abs(res.iters - ref.iters) <= 1
        assert np.linalg.norm(res.x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)


def pin_pcgs_forms_agree():
    """The one-reduction form is algebraically identical to Algorithm 1 (literal form)."""
    A = csr_of((12, 11), 5)
    xt, b = I.poisson_problem((12, 11), 5)
    v0 = I.power_start(A.n)
    for gram, nu in (("cholesky", 0), ("fgs", 30)):
        lit = O.pcgs(A, b, s=4, nu=nu, rtol=1e-9, algo="literal", gram=gram, power_v0=v0,
                     power_iters=20, power_tol=0.0)
        one = O.pcgs(A, b, s=4, nu=nu, rtol=1e-9, algo="onesync", gram=gram, power_v0=v0,
                     power_iters=20, power_tol=0.0)
        assert lit.status == O.OK and one.status == O.OK and abs(lit.iters - one.iters) <= 1
        assert np.linalg.norm(lit.x - one.x) <= 1e-9 * np.linalg.norm(lit.x)


def pin_pcgs_dense_solution():
    """On tiny grids the converged PCG-S solution matches a dense direct solve."""
    for dims, pts, s in [((4, 4, 4), 7, 3), ((5, 4), 5, 2), ((3, 3, 3), 27, 4)]:
        A = csr_of(dims, pts)
        xt, b = I.poisson_problem(dims, pts)
        xs = np.linalg.solve(A.dense(), b)
        res = O.pcgs(A, b, s=s, nu=30, rtol=1e-12, power_v0=I.power_start(A.n))
        assert res.status == O.OK
        assert np.linalg.norm(res.x - xs) <= 1e-9 * np.linalg.norm(xs), dims
        assert np.allclose(xs, xt, rtol=1e-10, atol=1e-10)


def pin_pcgs_reaches_tolerance():
    """Recursive and true residuals both reach rtol on a 2D and a 3D grid (nu = 2)."""
    for dims, pts in [((16, 16), 5), ((6, 6, 6), 7)]:
        A = csr_of(dims, pts)
        xt, b = I.poisson_problem(dims, pts)
        res = O.pcgs(A, b, s=4, nu=2, rtol=1e-8, power_v0=I.power_start(A.n), power_iters=20,
                     power_tol=0.0, algo="onesync")
        assert res.status == O.OK and res.relres <= 1e-8 and res.relres_true <= 2e-8


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
