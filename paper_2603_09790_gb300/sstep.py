"""Python binding of libsstep.so (include/sstep.h): argument marshalling only.

Every numerical step runs in the CUDA library; this module converts torch tensors (CUDA or
CPU) and numpy arrays to raw pointers and sizes, calls the C ABI, and raises on error.  It
fails loudly when the library has not been built: there is no CPU fallback.

Names follow the C ABI: ``setup``/``solve``/``solve_batched``/``free`` (wrapped by
:class:`Solver`), ``mpk``, ``block_gram``, ``fgs``, ``block_update``, ``spmv``,
``get_basis_info``, ``get_history``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsstep.so")

(OK, NOT_CONVERGED, ERR_INVALID, ERR_BREAKDOWN, ERR_NONFINITE, ERR_CUDA, ERR_OOM, ERR_UNSUPPORTED,
 ERR_TIMEOUT) = range(9)
MATRIX_CSR, MATRIX_STENCIL, MATRIX_Q1 = 0, 1, 2
PREC = {"none": 0, "jacobi": 1, "amg": 2}
ALGO = {"onesync": 0, "literal": 1, "pcg": 2}
GRAM = {"fgs": 0, "cholesky": 1, "fgs_operator": 2}


class SstepError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sstep status {status}: {msg}")
        self.status = status


class _Matrix(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int64), ("rowptr", C.c_void_p), ("colind", C.c_void_p),
                ("vals", C.c_void_p), ("nnz", C.c_int64), ("nx", C.c_int), ("ny", C.c_int),
                ("nz", C.c_int), ("points", C.c_int), ("weights", C.c_void_p)]


class _Precond(C.Structure):
    _fields_ = [("kind", C.c_int), ("amg_coarse_max", C.c_int), ("amg_max_levels", C.c_int)]


class _Opts(C.Structure):
    _fields_ = [("s", C.c_int), ("sweeps", C.c_int), ("rtol", C.c_double), ("max_outer", C.c_int),
                ("algo", C.c_int), ("gram_solver", C.c_int), ("power_iters", C.c_int),
                ("power_tol", C.c_double), ("lambda_min", C.c_double), ("lambda_max", C.c_double),
                ("power_v0", C.c_void_p), ("check_every", C.c_int), ("gram_blocks", C.c_int),
                ("precision", C.c_int), ("rr_period", C.c_int), ("persistent", C.c_int),
                ("cluster", C.c_int), ("block_threads", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_iters", C.c_int), ("inner_equiv", C.c_int),
                ("relres", C.c_double), ("relres_true", C.c_double), ("lambda_max", C.c_double),
                ("lambda_min", C.c_double), ("ms_setup", C.c_double), ("ms_solve", C.c_double),
                ("launches", C.c_longlong)]


_lib = None


def load():
    """Load libsstep.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            "libsstep.so is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    P, I, D, I64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
    sig = {
        "sstep_default_opts": (None, [P]),
        "sstep_setup": (I, [P, I, P, P, P, P]),
        "sstep_solve": (I, [P, P, P, P]),
        "sstep_solve_batched": (I, [P, I, P, P, P]),
        "sstep_free": (I, [P]),
        "sstep_status_string": (C.c_char_p, [I]),
        "sstep_last_error": (C.c_char_p, []),
        "sstep_mpk": (I, [P, P, P, P, I]),
        "sstep_block_gram": (I, [I64, I, P, I, P, I, P, P, P]),
        "sstep_fgs": (I, [I, P, I, P, I, I, P, P, P]),
        "sstep_block_update": (I, [P, P, P, P, P, P, P, P, P, P, I]),
        "sstep_spmv": (I, [P, P, P]),
        "sstep_get_basis_info": (I, [P, P, P, P, P, P, P]),
        "sstep_get_history": (I, [P, P, I, P]),
        "sstep_profile": (I, [P, P, I, P]),
        "sstep_block_gram_noalloc": (I, [I64, I, P, I, P, I, P, P, P]),
        "sstep_pattern_grad": (I, [I64, P, P, P, P, P, D, I, P]),
        "sstep_update_values": (I, [P, P]),
        "sstep_get_batch_config": (I, [P, P, P, P, P, P]),
        "sstep_amg_levels": (I, [P, P]),
        "sstep_amg_level": (I, [P, I, P, P, P, P, P, P]),
        "sstep_amg_apply": (I, [P, P, P]),
        "sstep_get_diagnostics": (I, [P, P, P, I, P, P, I, P]),
        "sstep_q1_exp": (I, [I64, P, P, P]),
        "sstep_q1_assemble": (I, [I, I, I, P, P, P, P, P]),
        "sstep_q1_grad": (I, [I, I, I, P, P, P, P, I, I, P]),
        "sstep_stencil7_weight_grad": (I, [I, I, P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != OK:
        lib = load()
        msg = lib.sstep_last_error().decode() or lib.sstep_status_string(status).decode()
        raise SstepError(status, msg)


def _ptr(a) -> Optional[int]:
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data
    raise TypeError("expected a torch tensor or a numpy array")


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


@dataclass
class Stencil:
    """Matrix-free stencil operator on the interior of an nx x ny x nz grid."""
    nx: int
    ny: int
    nz: int = 1
    points: int = 7
    weights: Optional[Sequence[float]] = None

    @property
    def n(self):
        return self.nx * self.ny * self.nz


@dataclass
class CSR:
    """CSR operator: rowptr int64 (n+1), colind int32 (nnz), vals float64 (nnz); torch or numpy."""
    rowptr: object
    colind: object
    vals: object
    _keep: list = field(default_factory=list, repr=False)

    @property
    def n(self):
        return int(self.rowptr.shape[0]) - 1

    @property
    def nnz(self):
        return int(self.colind.shape[0])


@dataclass
class Q1:
    """Matrix-free Q1 finite-element diffusion operator on the nx x ny x nz interior vertices of
    a grid of (nx+1)(ny+1)(nz+1) unit cells; kappa: the cell conductivities, float64, shape
    (nz+1, ny+1, nx+1) or flat, torch (any device) or numpy."""
    nx: int
    ny: int
    nz: int
    kappa: object

    @property
    def n(self):
        return self.nx * self.ny * self.nz

    @property
    def ncell(self):
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)


@dataclass
class Info:
    status: int
    outer_iters: int
    inner_equiv: int
    relres: float
    relres_true: float
    lambda_max: float
    lambda_min: float
    ms_setup: float
    ms_solve: float
    launches: int


def _info(i: _Info) -> Info:
    return Info(i.status, i.outer_iters, i.inner_equiv, i.relres, i.relres_true, i.lambda_max,
                i.lambda_min, i.ms_setup, i.ms_solve, i.launches)


class Solver:
    """A handle of libsstep.so (sstep_setup ... sstep_free)."""

    def __init__(self, A, *, precond="jacobi", s=4, sweeps=2, rtol=1e-8, max_outer=10000,
                 algo="literal", gram="fgs", power_iters=50, power_tol=1e-3, lambda_min=0.0,
                 lambda_max=0.0, power_v0=None, check_every=0, gram_blocks="full", precision="fp64",
                 rr_period=0, persistent=False, cluster=0, block_threads=0, amg_coarse_max=0,
                 amg_max_levels=0, stream=None):
        """A: a Stencil, CSR or Q1 (one system), or a list of 7-point Stencils (the batched
        persistent solver; also used for a single Stencil when persistent=True)."""
        mats = list(A) if isinstance(A, (list, tuple)) else [A]
        if not mats:
            raise ValueError("no system given")
        marr = (_Matrix * len(mats))()
        self._weights = []
        for m, a in zip(marr, mats):
            if isinstance(a, Stencil):
                m.kind = MATRIX_STENCIL
                m.n = a.n
                m.nx, m.ny, m.nz, m.points = a.nx, a.ny, a.nz, a.points
                if a.weights is not None:
                    w = np.ascontiguousarray(a.weights, dtype=np.float64)
                    self._weights.append(w)
                    m.weights = w.ctypes.data
            elif isinstance(a, Q1):
                k = a.kappa
                numel = k.numel() if hasattr(k, "numel") else int(np.asarray(k).size)
                dt = str(getattr(k, "dtype", ""))
                if numel != a.ncell or "float64" not in dt:
                    raise ValueError("Q1 kappa must hold (nx+1)(ny+1)(nz+1) float64 values")
                m.kind = MATRIX_Q1
                m.n = a.n
                m.nx, m.ny, m.nz = a.nx, a.ny, a.nz
                m.weights = _ptr(k)
            elif isinstance(a, CSR):
                m.kind = MATRIX_CSR
                m.n = a.n
                m.nnz = a.nnz
                m.rowptr, m.colind, m.vals = _ptr(a.rowptr), _ptr(a.colind), _ptr(a.vals)
            else:
                raise TypeError("A must be a Stencil, a CSR or a Q1, or a list of Stencils")
        lib = load()
        self.nsys = len(mats)
        self.sizes = [int(m.n) for m in marr]
        self.batched = self.nsys > 1 or bool(persistent)
        self.n = int(marr[0].n)
        o = _Opts()
        lib.sstep_default_opts(C.byref(o))
        o.s, o.sweeps, o.rtol, o.max_outer = int(s), int(sweeps), float(rtol), int(max_outer)
        o.algo, o.gram_solver = ALGO[algo], GRAM[gram]
        o.power_iters, o.power_tol = int(power_iters), float(power_tol)
        o.lambda_min, o.lambda_max = float(lambda_min), float(lambda_max)
        o.power_v0 = _ptr(power_v0)
        o.check_every = int(check_every)
        o.gram_blocks = {"full": 0, "sym": 1}[gram_blocks]
        o.precision = {"fp64": 0, "fp32_rr": 1}[precision]
        o.rr_period = int(rr_period)
        o.persistent = int(bool(persistent))
        o.cluster, o.block_threads = int(cluster), int(block_threads)
        self.s = int(s)
        self.max_outer = int(max_outer)
        pc = _Precond(PREC[precond], int(amg_coarse_max), int(amg_max_levels))
        h = C.c_void_p()
        _check(lib.sstep_setup(C.cast(marr, C.c_void_p), self.nsys, C.byref(pc), C.byref(o), _stream_ptr(stream), C.byref(h)))
        self._h = h

    # -- lifecycle
    def free(self):
        if getattr(self, "_h", None):
            load().sstep_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    # -- solves
    def solve(self, b, x, check=True) -> Info:
        """sstep_solve: x (x^(0) on entry) receives the solution; device or host buffers."""
        info = _Info()
        st = load().sstep_solve(self._h, _ptr(b), _ptr(x), C.byref(info))
        if check and st not in (OK, NOT_CONVERGED):
            _check(st)
        return _info(info)

    def solve_batched(self, bs, xs, check=True):
        """Single-system handle: one right-hand side after another.  Batched handle: bs and xs
        hold nsys * nrhs device tensors, system-major (bs[sys * nrhs + j]); one launch."""
        n = len(bs)
        if len(xs) != n:
            raise ValueError("bs and xs differ in length")
        nrhs = n
        if self.batched:
            if n % self.nsys:
                raise ValueError("a batched handle takes nsys * nrhs right-hand sides")
            nrhs = n // self.nsys
        B = (C.c_void_p * n)(*[_ptr(b) for b in bs])
        X = (C.c_void_p * n)(*[_ptr(x) for x in xs])
        infos = (_Info * n)()
        st = load().sstep_solve_batched(self._h, nrhs, B, X, infos)
        if check and st not in (OK, NOT_CONVERGED):
            _check(st)
        return [_info(i) for i in infos]

    # -- hot-path steps
    def mpk(self, r, Z, AZ, s=0):
        _check(load().sstep_mpk(self._h, _ptr(r), _ptr(Z), _ptr(AZ), int(s)))

    def block_update(self, Z, AZ, Q, AQ, alpha, beta, x, r, rr_out, s=0):
        _check(load().sstep_block_update(self._h, _ptr(Z), _ptr(AZ), _ptr(Q), _ptr(AQ), _ptr(alpha),
                                         _ptr(beta), _ptr(x), _ptr(r), _ptr(rr_out), int(s)))

    def spmv(self, x, y):
        _check(load().sstep_spmv(self._h, _ptr(x), _ptr(y)))

    def amg_levels(self):
        """AMG handle: the hierarchy, one (CSR arrays, aggregation map or None) per level."""
        lib = load()
        nl = C.c_int()
        _check(lib.sstep_amg_levels(self._h, C.byref(nl)))
        out = []
        for l in range(nl.value):
            n, nnz = C.c_int64(), C.c_int64()
            _check(lib.sstep_amg_level(self._h, l, C.byref(n), C.byref(nnz), None, None, None, None))
            rp = np.empty(n.value + 1, dtype=np.int64)
            ci = np.empty(nnz.value, dtype=np.int32)
            v = np.empty(nnz.value)
            agg = np.full(n.value, -1, dtype=np.int32)
            _check(lib.sstep_amg_level(self._h, l, None, None, rp.ctypes.data, ci.ctypes.data,
                                       v.ctypes.data, agg.ctypes.data))
            out.append(((rp, ci, v), agg if l + 1 < nl.value else None))
        return out

    def amg_apply(self, b, x):
        """x = M^{-1} b (one V-cycle) on device tensors."""
        _check(load().sstep_amg_apply(self._h, _ptr(b), _ptr(x)))

    def get_diagnostics(self):
        """eta_alpha, eta_beta per outer iteration and the first W_k of the last solve."""
        m = self.max_outer + 2
        ea, eb = np.zeros(m), np.zeros(m)
        W = np.zeros((64, self.s, self.s))
        cnt, cw = C.c_int(), C.c_int()
        _check(load().sstep_get_diagnostics(self._h, ea.ctypes.data, eb.ctypes.data, m, C.byref(cnt),
                                            W.ctypes.data, 64, C.byref(cw)))
        n = cnt.value
        # W_k is column-major: W[k][j, i] holds entry (i, j)
        return dict(eta_a=ea[:n].copy(), eta_b=eb[:max(n - 1, 0)].copy(),
                    W=np.transpose(W[:cw.value], (0, 2, 1)).copy())

    def get_batch_config(self):
        """Batched handle: the configuration in use (autotuned where it was left open)."""
        v = [C.c_int() for _ in range(4)]
        t = C.c_double()
        _check(load().sstep_get_batch_config(self._h, *[C.byref(x) for x in v], C.byref(t)))
        return dict(s=v[0].value, cluster=v[1].value, threads=v[2].value, slots=v[3].value,
                    tune_ms=t.value)

    def get_basis_info(self):
        v = [C.c_double() for _ in range(5)]
        it = C.c_int()
        _check(load().sstep_get_basis_info(self._h, *[C.byref(t) for t in v], C.byref(it)))
        lmin, lmax, ca, cs, cg = (t.value for t in v)
        return dict(lambda_min=lmin, lambda_max=lmax, c_alpha=ca, c_sigma=cs, c_gamma=cg,
                    power_iters=it.value)

    def profile(self, b, iters=5):
        """sstep_profile: average device ms per phase of one outer iteration (4 values)."""
        ms = (C.c_double * 5)()
        _check(load().sstep_profile(self._h, _ptr(b), int(iters), ms))
        return list(ms)

    def update_values(self, vals):
        """sstep_update_values: new values for the handle's CSR operator (same pattern) or new
        Q1 cell conductivities; the Jacobi diagonal is recomputed, the Chebyshev interval is
        kept."""
        _check(load().sstep_update_values(self._h, _ptr(vals)))

    def get_history(self):
        buf = np.zeros(self.max_outer + 2)
        cnt = C.c_int()
        _check(load().sstep_get_history(self._h, buf.ctypes.data, buf.size, C.byref(cnt)))
        return buf[: cnt.value].copy()


def block_gram(L, R, pairs, out, stream=None):
    """sstep_block_gram: out[e] = L[pairs[e][0]] . R[pairs[e][1]] (device vectors of length n)."""
    n = int(L[0].numel())
    Lp = (C.c_void_p * len(L))(*[_ptr(v) for v in L])
    Rp = (C.c_void_p * len(R))(*[_ptr(v) for v in R])
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1))
    _check(load().sstep_block_gram(n, len(L), Lp, len(R), Rp, pr.size // 2, pr.ctypes.data,
                                   _ptr(out), _stream_ptr(stream)))


def block_gram_noalloc(L, R, pairs, out, stream=None):
    """sstep_block_gram_noalloc: the same products as block_gram for callers that cannot
    allocate device memory at call time; scratch is a fixed area inside the library (at most
    256 products per call; calls overlapping on the GPU race)."""
    n = int(L[0].numel())
    Lp = (C.c_void_p * len(L))(*[_ptr(v) for v in L])
    Rp = (C.c_void_p * len(R))(*[_ptr(v) for v in R])
    pr = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1))
    _check(load().sstep_block_gram_noalloc(n, len(L), Lp, len(R), Rp, pr.size // 2, pr.ctypes.data,
                                           _ptr(out), _stream_ptr(stream)))


def pattern_grad(rowptr, colind, lam, x, grad_vals, scale=1.0, accumulate=False, stream=None):
    """sstep_pattern_grad: grad_vals[k] (+)= -scale * lam[i] * x[colind[k]] for every stored
    entry k of row i (device tensors; rowptr int64, colind int32)."""
    n = int(rowptr.numel()) - 1
    _check(load().sstep_pattern_grad(n, _ptr(rowptr), _ptr(colind), _ptr(lam), _ptr(x), _ptr(grad_vals),
                                     float(scale), int(bool(accumulate)), _stream_ptr(stream)))


def q1_exp(theta, kappa, stream=None):
    """sstep_q1_exp: kappa = exp(theta) (device tensors of the cell count)."""
    _check(load().sstep_q1_exp(int(theta.numel()), _ptr(theta), _ptr(kappa), _stream_ptr(stream)))


def q1_assemble(dims, kappa, rowptr, colind, vals, stream=None):
    """sstep_q1_assemble: CSR values of the Q1 operator for cell conductivities kappa on the
    pattern (rowptr int64, colind int32) of the nx x ny x nz interior vertex grid."""
    nx, ny, nz = (int(d) for d in dims)
    _check(load().sstep_q1_assemble(nx, ny, nz, _ptr(kappa), _ptr(rowptr), _ptr(colind), _ptr(vals),
                                    _stream_ptr(stream)))


def q1_grad(dims, kappa, lam, x, grad, wrt_log=True, accumulate=False, stream=None):
    """sstep_q1_grad: grad[c] (+)= -lambda_c^T K_ref x_c per cell, times kappa_c when wrt_log."""
    nx, ny, nz = (int(d) for d in dims)
    _check(load().sstep_q1_grad(nx, ny, nz, _ptr(kappa), _ptr(lam), _ptr(x), _ptr(grad),
                                int(bool(wrt_log)), int(bool(accumulate)), _stream_ptr(stream)))


def stencil7_weight_grad(grids, nrhs, lam, x, grad, stream=None):
    """sstep_stencil7_weight_grad: grad[2 i] = -sum_r lam_ir^T x_ir, grad[2 i + 1] =
    -sum_r lam_ir^T N x_ir for systems with grids[i] = (nx, ny, nz) and nrhs right-hand sides
    each (lam, x: lists of device vectors, system-major; grad: device tensor of 2 nsys)."""
    nsys = len(grids)
    dims = np.ascontiguousarray(np.asarray(grids, dtype=np.int32).reshape(-1))
    L = (C.c_void_p * len(lam))(*[_ptr(v) for v in lam])
    X = (C.c_void_p * len(x))(*[_ptr(v) for v in x])
    _check(load().sstep_stencil7_weight_grad(nsys, int(nrhs), dims.ctypes.data, L, X, _ptr(grad),
                                             _stream_ptr(stream)))


def fgs(W, B, nu, X, solver="fgs", status=None, stream=None):
    """sstep_fgs: nu FGS sweeps (or Cholesky) on W X = B; W (s, s) and B (nrhs, s) device tensors
    in column-major order (row k of B is right-hand side k)."""
    s = int(W.shape[0])
    nrhs = int(B.shape[0])
    _check(load().sstep_fgs(s, _ptr(W), nrhs, _ptr(B), int(nu), GRAM[solver], _ptr(X), _ptr(status),
                            _stream_ptr(stream)))
