"""FP64 CPU oracle for Chebyshev-basis s-step PCG with FGS Gram solves, and classical PCG.

TEST INFRASTRUCTURE ONLY.  Imported by the tests, by the smoke check and by the CPU
baseline leg of the benchmark; the CUDA library and its Python binding never import it.
It shares no code with the CUDA path: the arithmetic lives in ``oracle.c`` (plain C,
sequential loops, FP64), written from the paper:

* ``mpk``      -- the Chebyshev basis of Section 2 by its three-term recurrence (Algorithm 2)
* ``fgs``      -- Eq. (fgs-iteration), Section 3.1 (forward Gauss-Seidel on W)
* ``reduced_relres`` -- eta_alpha / eta_beta of Section 3.3
* ``pcgs``     -- PCG-S (Section 2, Algorithm 1), literal form and one-reduction form
* ``pcg``      -- classical Hestenes-Stiefel PCG (Section 1)
* ``power``    -- power method for lambda_max, Section 2
* ``cheb``     -- Chebyshev scalars alpha, sigma, gamma, Section 2
* ``AMG``      -- the aggregation AMG preconditioner ``amg.c`` defines (the paper's own AMG
                  is external; Section 5 treats M^{-1} as a black box)

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, NOT_CONVERGED, ERR_INVALID, ERR_BREAKDOWN, ERR_NONFINITE = 0, 1, 2, 3, 4
PREC = {"none": 0, "jacobi": 1, "amg": 2}
ALGO = {"literal": 0, "onesync": 1}
GRAM = {"fgs": 0, "cholesky": 1}


class _CSR(C.Structure):
    _fields_ = [("n", C.c_int64), ("rowptr", C.c_void_p), ("colind", C.c_void_p), ("vals", C.c_void_p)]


class _Info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("relres", C.c_double),
                ("relres_true", C.c_double), ("c_alpha", C.c_double), ("c_sigma", C.c_double),
                ("c_gamma", C.c_double)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = C.CDLL(path)
        P = C.c_void_p
        lib.or_spmv.argtypes = [P, P, P]
        lib.or_jacobi_dinv.argtypes = [P, P]
        lib.or_jacobi_dinv.restype = C.c_int
        lib.or_prec_apply.argtypes = [C.c_int, C.c_int64, P, P, P]
        lib.or_gershgorin_lower.argtypes = [P, C.c_int]
        lib.or_gershgorin_lower.restype = C.c_double
        lib.or_power_lambda_max.argtypes = [P, C.c_int, P, P, C.c_int, C.c_double, P]
        lib.or_power_lambda_max.restype = C.c_double
        lib.or_cheb_scalars.argtypes = [C.c_double, C.c_double, P, P, P]
        lib.or_mpk.argtypes = [P, C.c_int, P, P, C.c_int, C.c_double, C.c_double, C.c_double, P, P]
        lib.or_mpk.restype = C.c_int
        lib.or_fgs.argtypes = [C.c_int, P, P, C.c_int, P]
        lib.or_fgs.restype = C.c_int
        lib.or_chol_solve.argtypes = [C.c_int, P, P, P]
        lib.or_chol_solve.restype = C.c_int
        lib.or_gram.argtypes = [C.c_int64, C.c_int, P, C.c_int, P, P]
        lib.or_reduced_relres.argtypes = [C.c_int, C.c_int, P, P, P]
        lib.or_reduced_relres.restype = C.c_double
        lib.or_pcgs.argtypes = [P, C.c_int, P, P, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int,
                                C.c_int, C.c_double, C.c_double, P, C.c_int, C.c_double, P, P, P, P]
        lib.or_pcgs.restype = C.c_int
        lib.or_pcg.argtypes = [P, C.c_int, P, P, C.c_double, C.c_int, P, P]
        lib.or_pcg.restype = C.c_int
        I64 = C.c_int64
        lib.or_amg_match.argtypes = [P, P, P]
        lib.or_amg_match.restype = C.c_int
        lib.or_amg_galerkin.argtypes = [P, P, I64, P, P, P, P]
        lib.or_amg_galerkin.restype = C.c_int
        lib.or_amg_setup.argtypes = [P, I64, C.c_int, P]
        lib.or_amg_setup.restype = C.c_int
        lib.or_amg_free.argtypes = [P]
        lib.or_amg_apply.argtypes = [P, P, P]
        lib.or_amg_nlevels.argtypes = [P]
        lib.or_amg_nlevels.restype = C.c_int
        lib.or_amg_level.argtypes = [P, C.c_int, P, P, P, P, P, P]
        lib.or_amg_level.restype = C.c_int
        lib.or_use_amg.argtypes = [P]
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class CSR:
    """CSR operator handed to the oracle (rowptr int64, colind int32, vals float64)."""

    def __init__(self, rowptr, colind, vals):
        self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        self.colind = np.ascontiguousarray(colind, dtype=np.int32)
        self.vals = _f64(vals)
        self.n = self.rowptr.size - 1
        self._s = _CSR(self.n, self.rowptr.ctypes.data, self.colind.ctypes.data, self.vals.ctypes.data)

    @property
    def ref(self):
        return C.byref(self._s)

    def dense(self) -> np.ndarray:
        A = np.zeros((self.n, self.n))
        for i in range(self.n):
            for k in range(self.rowptr[i], self.rowptr[i + 1]):
                A[i, self.colind[k]] += self.vals[k]
        return A


def spmv(A: CSR, x) -> np.ndarray:
    x = _f64(x)
    y = np.empty(A.n)
    _load().or_spmv(A.ref, _ptr(x), _ptr(y))
    return y


def jacobi_dinv(A: CSR) -> np.ndarray:
    d = np.empty(A.n)
    st = _load().or_jacobi_dinv(A.ref, _ptr(d))
    if st != OK:
        raise ValueError("Jacobi needs a positive diagonal")
    return d


def prec_apply(prec: str, dinv, x) -> np.ndarray:
    x = _f64(x)
    y = np.empty_like(x)
    d = _f64(dinv) if dinv is not None else np.ones_like(x)
    _load().or_prec_apply(PREC[prec], x.size, _ptr(d), _ptr(x), _ptr(y))
    return y


def _use(prec, amg):
    if prec == "amg":
        if amg is None:
            raise ValueError("prec='amg' needs amg=AMG(A)")
        _load().or_use_amg(amg._h)


def gershgorin_lower(A: CSR, prec: str = "jacobi") -> float:
    return float(_load().or_gershgorin_lower(A.ref, PREC[prec]))


def power(A: CSR, prec: str, v0, max_iters: int = 50, tol: float = 1e-3, amg=None):
    """Power-method estimate of lambda_max(M^{-1}A) (Section 2); returns (lambda, iterations)."""
    _use(prec, amg)
    d = jacobi_dinv(A) if prec == "jacobi" else np.ones(A.n)
    v0 = _f64(v0)
    it = C.c_int(0)
    lam = _load().or_power_lambda_max(A.ref, PREC[prec], _ptr(d), _ptr(v0), int(max_iters),
                                      float(tol), C.byref(it))
    return float(lam), int(it.value)


def cheb(lmin: float, lmax: float):
    """(c_alpha, c_sigma, c_gamma) of Section 2."""
    a, s, g = C.c_double(), C.c_double(), C.c_double()
    _load().or_cheb_scalars(float(lmin), float(lmax), C.byref(a), C.byref(s), C.byref(g))
    return a.value, s.value, g.value


def mpk(A: CSR, prec: str, r, s: int, c_alpha: float, c_sigma: float, c_gamma: float = 1.0,
        amg=None):
    """Algorithm 2: returns Z (n x s) and P (n x (s+1)) as column arrays (shape (s, n), (s+1, n))."""
    _use(prec, amg)
    d = jacobi_dinv(A) if prec == "jacobi" else np.ones(A.n)
    r = _f64(r)
    Z = np.empty((s, A.n))
    P = np.empty((s + 1, A.n))
    st = _load().or_mpk(A.ref, PREC[prec], _ptr(d), _ptr(r), int(s), c_alpha, c_sigma, c_gamma,
                        _ptr(Z), _ptr(P))
    if st != OK:
        raise ValueError("invalid MPK arguments")
    return Z, P


def fgs(W, m, nu: int) -> np.ndarray:
    """nu FGS sweeps on W alpha = m from alpha = 0 (Eq. fgs-iteration)."""
    W = np.asfortranarray(W, dtype=np.float64)
    m = _f64(m)
    s = m.size
    out = np.empty(s)
    st = _load().or_fgs(s, W.ctypes.data_as(C.c_void_p), _ptr(m), int(nu), _ptr(out))
    if st != OK:
        raise FloatingPointError("FGS breakdown (W_ii <= 0 or non-finite)")
    return out


def chol_solve(W, m) -> np.ndarray:
    W = np.asfortranarray(W, dtype=np.float64)
    m = _f64(m)
    out = np.empty(m.size)
    st = _load().or_chol_solve(m.size, W.ctypes.data_as(C.c_void_p), _ptr(m), _ptr(out))
    if st != OK:
        raise FloatingPointError("Cholesky breakdown")
    return out


def gram(X, Y) -> np.ndarray:
    """X^T Y for column arrays X (a, n), Y (b, n) -> (a, b)."""
    X = _f64(X)
    Y = _f64(Y)
    a, n = X.shape
    b = Y.shape[0]
    G = np.empty((b, a))  # column-major a x b == row-major (b, a)
    _load().or_gram(n, a, _ptr(X), b, _ptr(Y), _ptr(G))
    return G.T.copy()


def reduced_relres(W, M, X) -> float:
    """||M - W X|| / ||M|| (Section 3.3: eta_alpha for one column, eta_beta as the Frobenius
    form for an s x ncol block).  M, X: (s,) or (s, ncol)."""
    W = np.asfortranarray(W, dtype=np.float64)
    M = np.asarray(M, dtype=np.float64)
    ncol = 1 if M.ndim == 1 else M.shape[1]
    Mf = np.asfortranarray(M.reshape(W.shape[0], ncol))
    Xf = np.asfortranarray(np.asarray(X, dtype=np.float64).reshape(W.shape[0], ncol))
    return float(_load().or_reduced_relres(W.shape[0], ncol, W.ctypes.data_as(C.c_void_p),
                                           Mf.ctypes.data_as(C.c_void_p),
                                           Xf.ctypes.data_as(C.c_void_p)))


class Result:
    def __init__(self, x, info, hist=None, eta_a=None, eta_b=None):
        self.x = x
        self.status = info.status
        self.iters = info.iters
        self.relres = info.relres
        self.relres_true = info.relres_true
        self.c_alpha, self.c_sigma, self.c_gamma = info.c_alpha, info.c_sigma, info.c_gamma
        n = self.iters
        self.hist = hist[: n + 1] if hist is not None else None
        self.eta_a = eta_a[:n] if eta_a is not None else None
        self.eta_b = eta_b[: max(n - 1, 0)] if eta_b is not None else None


def pcgs(A: CSR, b, x0=None, *, s=4, nu=2, rtol=1e-8, max_outer=10000, algo="literal",
         gram="fgs", prec="jacobi", lambda_min=0.0, lambda_max=0.0, power_v0=None,
         power_iters=50, power_tol=1e-3, history=False, amg=None) -> Result:
    """Algorithm 1 (PCG-S) on the CPU in FP64 (prec 'amg' applies the hierarchy amg)."""
    _use(prec, amg)
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    v0 = _f64(power_v0) if power_v0 is not None else np.ones(A.n)
    info = _Info()
    hist = np.zeros(max_outer + 1) if history else None
    ea = np.zeros(max(max_outer, 1)) if history else None
    eb = np.zeros(max(max_outer, 1)) if history else None
    _load().or_pcgs(A.ref, PREC[prec], _ptr(b), _ptr(x), int(s), int(nu), float(rtol),
                    int(max_outer), ALGO[algo], GRAM[gram], float(lambda_min), float(lambda_max),
                    _ptr(v0), int(power_iters), float(power_tol), C.byref(info), _ptr(hist),
                    _ptr(ea), _ptr(eb))
    return Result(x, info, hist, ea, eb)


def pcg(A: CSR, b, x0=None, *, rtol=1e-8, max_iters=100000, prec="jacobi", history=False,
        amg=None) -> Result:
    """Classical Hestenes-Stiefel PCG on the CPU in FP64."""
    _use(prec, amg)
    b = _f64(b)
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    info = _Info()
    hist = np.zeros(max_iters + 1) if history else None
    _load().or_pcg(A.ref, PREC[prec], _ptr(b), _ptr(x), float(rtol), int(max_iters),
                   C.byref(info), _ptr(hist))
    return Result(x, info, hist)


def _csr_from(n, nnz, rp, ci, v):
    rowptr = np.ctypeslib.as_array(C.cast(rp, C.POINTER(C.c_int64)), shape=(n + 1,)).copy()
    colind = np.ctypeslib.as_array(C.cast(ci, C.POINTER(C.c_int32)), shape=(max(nnz, 1),))[:nnz].copy()
    vals = np.ctypeslib.as_array(C.cast(v, C.POINTER(C.c_double)), shape=(max(nnz, 1),))[:nnz].copy()
    return CSR(rowptr, colind, vals)


def amg_match(A: CSR):
    """One greedy pairwise matching (amg.c): returns (agg, number of aggregates)."""
    agg = np.empty(A.n, dtype=np.int32)
    nc = C.c_int64(0)
    if _load().or_amg_match(A.ref, _ptr(agg), C.byref(nc)) != OK:
        raise ValueError("matching needs a positive diagonal")
    return agg, int(nc.value)


def amg_galerkin(A: CSR, agg, nc: int) -> CSR:
    """P^T A P for the piecewise-constant aggregation agg (amg.c's fixed summation order)."""
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    rp, ci, v = C.c_void_p(), C.c_void_p(), C.c_void_p()
    nnz = C.c_int64(0)
    lib = _load()
    if lib.or_amg_galerkin(A.ref, _ptr(agg), int(nc), C.byref(rp), C.byref(ci), C.byref(v),
                           C.byref(nnz)) != OK:
        raise ValueError("galerkin product failed")
    out = _csr_from(int(nc), int(nnz.value), rp, ci, v)
    libc = C.CDLL(None)
    libc.free.argtypes = [C.c_void_p]
    for ptr in (rp, ci, v):
        libc.free(ptr)
    return out


class AMG:
    """Aggregation AMG hierarchy of amg.c for A: levels until n <= coarse_max."""

    def __init__(self, A: CSR, coarse_max: int = 2048, max_levels: int = 25):
        self._lib = _load()
        h = C.c_void_p()
        st = self._lib.or_amg_setup(A.ref, int(coarse_max), int(max_levels), C.byref(h))
        if st != OK:
            raise ValueError(f"AMG set-up failed with status {st}")
        self._h = h
        self.nlevels = int(self._lib.or_amg_nlevels(h))

    def level(self, l: int):
        """(CSR of level l, its aggregation map or None on the coarsest level)."""
        n, nnz = C.c_int64(), C.c_int64()
        rp, ci, v, agg = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
        if self._lib.or_amg_level(self._h, int(l), C.byref(n), C.byref(nnz), C.byref(rp), C.byref(ci),
                                  C.byref(v), C.byref(agg)) != OK:
            raise IndexError(l)
        A = _csr_from(int(n.value), int(nnz.value), rp, ci, v)
        a = None
        if agg.value:
            a = np.ctypeslib.as_array(C.cast(agg, C.POINTER(C.c_int32)), shape=(int(n.value),)).copy()
        return A, a

    def apply(self, b) -> np.ndarray:
        """One V-cycle: M^{-1} b."""
        b = _f64(b)
        x = np.empty_like(b)
        self._lib.or_amg_apply(self._h, _ptr(b), _ptr(x))
        return x

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                self._lib.or_use_amg(None)
                self._lib.or_amg_free(self._h)
                self._h = None
        except Exception:
            pass


class _swapped_library:
    """Run the wrappers above against another build of oracle.c (used by the test that
    plants mistakes in a copy of the oracle and checks that the pins catch them)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self.saved = _lib
        lib = C.CDLL(self.path)
        for name in dir(self.saved):
            if name.startswith("or_"):
                f, g = getattr(self.saved, name), getattr(lib, name)
                g.argtypes, g.restype = f.argtypes, f.restype
        _lib = lib
        return lib

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def use_library(path):
    return _swapped_library(path)
