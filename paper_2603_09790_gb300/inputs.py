"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module draws random numbers and lays out test operators; it holds none of the
solver's arithmetic (no Krylov step, no Chebyshev recurrence, no Gram product).

* ``splitmix64`` / ``uniform_pm1``: SplitMix64 (Steele, Lea and Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014).  The k-th output of a stream with seed
  ``s`` mixes ``s + (k+1) * 0x9E3779B97F4A7C15``; a double in [-1, 1) is
  ``2 * (out >> 11) * 2**-53 - 1``.  x_true uses seed 0 and the power-method start vector
  seed 1, both in lexicographic grid order.
* ``poisson_csr``: the finite-difference Poisson matrices the paper's experiments use
  (27-point as in HPCG, Section 6) and their 5- and 7-point relatives, on the interior
  unknowns of an nx x ny x nz grid with Dirichlet neighbours dropped; row index
  ``i + nx*(j + ny*k)``; diagonal 4 / 6 / 26, off-diagonals -1; columns sorted.
* ``poisson_apply``: the same operator applied matrix-free, used only to form the
  right-hand side b = A x_true of a synthetic problem.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STENCIL_DIAG = {5: 4.0, 7: 6.0, 27: 26.0}


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+n-1`` of the SplitMix64 stream with the given seed (uint64)."""
    with np.errstate(over="ignore"):
        k = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_pm1(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Doubles in [-1, 1) from SplitMix64: 2*u - 1 with u = (next >> 11) * 2**-53."""
    u = (splitmix64(seed, n, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def stencil_offsets(points: int):
    """Neighbour offsets (dx, dy, dz) of a stencil, sorted by linear column offset."""
    if points == 5:
        offs = [(0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0)]
    elif points == 7:
        offs = [(0, 0, -1), (0, -1, 0), (-1, 0, 0), (0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    elif points == 27:
        offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    else:
        raise ValueError("points must be 5, 7 or 27")
    return offs


def _dims3(dims):
    dims = tuple(int(d) for d in dims)
    if len(dims) == 2:
        dims = dims + (1,)
    if len(dims) != 3 or min(dims) < 1:
        raise ValueError("dims must be (nx, ny) or (nx, ny, nz) with positive entries")
    return dims


def poisson_csr(dims, points: int):
    """CSR arrays (rowptr int64, colind int32, vals float64) of the Dirichlet Poisson matrix."""
    nx, ny, nz = _dims3(dims)
    if points == 5 and nz != 1:
        raise ValueError("the 5-point stencil is two-dimensional")
    n = nx * ny * nz
    diag = STENCIL_DIAG[points]
    idx = np.arange(n, dtype=np.int64)
    ix = idx % nx
    iy = (idx // nx) % ny
    iz = idx // (nx * ny)
    offs = stencil_offsets(points)
    masks = []
    for dx, dy, dz in offs:
        m = np.ones(n, dtype=bool)
        if dx:
            m &= (ix + dx >= 0) & (ix + dx < nx)
        if dy:
            m &= (iy + dy >= 0) & (iy + dy < ny)
        if dz:
            m &= (iz + dz >= 0) & (iz + dz < nz)
        masks.append(m)
    counts = np.zeros(n, dtype=np.int64)
    for m in masks:
        counts += m
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    if nnz >= 2 ** 31 or n >= 2 ** 31:
        raise ValueError("operator too large for int32 column indices")
    colind = np.empty(nnz, dtype=np.int32)
    vals = np.empty(nnz, dtype=np.float64)
    fill = rowptr[:-1].copy()
    for (dx, dy, dz), m in zip(offs, masks):
        rows = idx[m]
        pos = fill[m]
        colind[pos] = (rows + dx + nx * (dy + ny * dz)).astype(np.int32)
        vals[pos] = diag if (dx, dy, dz) == (0, 0, 0) else -1.0
        fill[m] += 1
    return rowptr, colind, vals


def poisson_apply(dims, points: int, x: np.ndarray) -> np.ndarray:
    """A x for the Dirichlet Poisson matrix, matrix-free (used to form b = A x_true)."""
    nx, ny, nz = _dims3(dims)
    u = np.asarray(x, dtype=np.float64).reshape(nz, ny, nx)
    pad = np.zeros((nz + 2, ny + 2, nx + 2))
    pad[1:-1, 1:-1, 1:-1] = u
    y = STENCIL_DIAG[points] * u
    for dx, dy, dz in stencil_offsets(points):
        if (dx, dy, dz) == (0, 0, 0):
            continue
        y = y - pad[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
    return y.reshape(-1)


def poisson_problem(dims, points: int, seed: int = 0):
    """x_true ~ U[-1,1) (SplitMix64, given seed, lexicographic) and b = A x_true."""
    nx, ny, nz = _dims3(dims)
    n = nx * ny * nz
    x_true = uniform_pm1(seed, n)
    b = poisson_apply((nx, ny, nz), points, x_true)
    return x_true, b


def power_start(n: int, seed: int = 1) -> np.ndarray:
    """Start vector of the power method: U[-1,1) with seed 1."""
    return uniform_pm1(seed, n)


# ---------------------------------------------------------------- variable-coefficient diffusion

def normal_pm(seed: int, n: int) -> np.ndarray:
    """Standard normal variates by Box-Muller from SplitMix64 outputs 2k, 2k+1 (k < n)."""
    u = (splitmix64(seed, 2 * n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def lognormal_conductivity(cells, sigma: float = 1.0, corr: float = 8.0, seed: int = 0):
    """Per-cell conductivity kappa = exp(sigma g): g is white noise (seed) convolved with a
    separable Gaussian of standard deviation corr / sqrt(2) cells (covariance
    exp(-d^2 / (2 corr^2))), renormalised to zero mean and unit variance.  Shape (cz, cy, cx)."""
    from scipy.ndimage import gaussian_filter

    cx, cy, cz = (int(c) for c in cells)
    g = normal_pm(seed, cx * cy * cz).reshape(cz, cy, cx)
    if corr > 0:
        g = gaussian_filter(g, sigma=corr / np.sqrt(2.0), mode="wrap")
    g = (g - g.mean()) / g.std()
    return np.exp(sigma * g)


def q1_reference_stiffness() -> np.ndarray:
    """8 x 8 stiffness of the trilinear (Q1) element on the unit cube, vertex (i, j, k) of the
    cell at local index i + 2 j + 4 k: K = K1 x M1 x M1 + M1 x K1 x M1 + M1 x M1 x K1 with the
    1D stiffness K1 = [[1, -1], [-1, 1]] and mass M1 = [[1/3, 1/6], [1/6, 1/3]]."""
    K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    M1 = np.array([[1.0, 0.5], [0.5, 1.0]]) / 3.0
    # index order of np.kron(a, b) is (a index) * 2 + b index: build z, y, x major -> i + 2j + 4k
    return (np.kron(np.kron(M1, M1), K1) + np.kron(np.kron(M1, K1), M1) +
            np.kron(np.kron(K1, M1), M1))


def q1_csr(dims, kappa):
    """CSR of the Q1 finite-element diffusion operator on the nx x ny x nz interior vertices of a
    grid of (nx+1)(ny+1)(nz+1) unit cells with conductivity kappa (shape (nz+1, ny+1, nx+1)),
    Dirichlet boundary vertices eliminated.  27-point pattern; the face-neighbour couplings
    of Q1 vanish identically and are not stored (21 entries on an interior row)."""
    nx, ny, nz = (int(d) for d in dims)
    kappa = np.asarray(kappa, dtype=np.float64)
    assert kappa.shape == (nz + 1, ny + 1, nx + 1)
    Kr = q1_reference_stiffness()
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    ix, iy, iz = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)
            if (dx != 0) + (dy != 0) + (dz != 0) != 1]
    coef = {}
    for d in offs:
        c = np.zeros(n)
        # cells around vertex v (grid coords v+1): lower corner v+1+o, o in {-1, 0}^3
        for ox in (-1, 0):
            for oy in (-1, 0):
                for oz in (-1, 0):
                    lv = (-ox, -oy, -oz)  # local coordinates of v in that cell
                    lw = (lv[0] + d[0], lv[1] + d[1], lv[2] + d[2])
                    if min(lw) < 0 or max(lw) > 1:
                        continue
                    kv = Kr[lv[0] + 2 * lv[1] + 4 * lv[2], lw[0] + 2 * lw[1] + 4 * lw[2]]
                    c += kv * kappa[iz + 1 + oz, iy + 1 + oy, ix + 1 + ox]
        coef[d] = c
    masks = []
    for dx, dy, dz in offs:
        m = (ix + dx >= 0) & (ix + dx < nx) & (iy + dy >= 0) & (iy + dy < ny) & \
            (iz + dz >= 0) & (iz + dz < nz)
        masks.append(m)
    counts = np.zeros(n, dtype=np.int64)
    for m in masks:
        counts += m
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    colind = np.empty(nnz, dtype=np.int32)
    vals = np.empty(nnz, dtype=np.float64)
    fill = rowptr[:-1].copy()
    for d, m in zip(offs, masks):
        rows = idx[m]
        pos = fill[m]
        colind[pos] = (rows + d[0] + nx * (d[1] + ny * d[2])).astype(np.int32)
        vals[pos] = coef[d][m]
        fill[m] += 1
    return rowptr, colind, vals


def csr_matvec(rowptr, colind, vals, x):
    """y = A x for CSR arrays (used to form b = A x_true of a synthetic problem)."""
    prod = vals * np.asarray(x)[colind]
    y = np.add.reduceat(prod, rowptr[:-1]) if prod.size else np.zeros(rowptr.size - 1)
    y[rowptr[1:] == rowptr[:-1]] = 0.0
    return y


def q1_lognormal_problem(dims, sigma: float = 1.0, corr: float = 8.0, seed: int = 0):
    """Operator (CSR), conductivity, x_true ~ U[-1,1) (seed) and b = A x_true."""
    nx, ny, nz = (int(d) for d in dims)
    kappa = lognormal_conductivity((nx + 1, ny + 1, nz + 1), sigma, corr, seed)
    rp, ci, v = q1_csr((nx, ny, nz), kappa)
    x_true = uniform_pm1(seed, nx * ny * nz)
    b = csr_matvec(rp, ci, v, x_true)
    return (rp, ci, v), kappa, x_true, b


def q1_assembly(dims):
    """The linear map from cell conductivities to the CSR values of q1_csr: vals[k] =
    sum_t S_vals[t] * kappa.flat[S_cells[t]] over the triplets t with S_rows[t] = k.
    Returns (rowptr, colind, S_rows, S_cells, S_vals); same pattern as q1_csr."""
    nx, ny, nz = (int(d) for d in dims)
    ones = np.ones((nz + 1, ny + 1, nx + 1))
    rowptr, colind, _ = q1_csr((nx, ny, nz), ones)
    Kr = q1_reference_stiffness()
    n = nx * ny * nz
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))
    ix, iy, iz = rows % nx, (rows // nx) % ny, rows // (nx * ny)
    jx, jy, jz = colind % nx, (colind // nx) % ny, colind // (nx * ny)
    dx, dy, dz = jx - ix, jy - iy, jz - iz
    tr, tc, tv = [], [], []
    k_all = np.arange(colind.size, dtype=np.int64)
    for ox in (-1, 0):
        for oy in (-1, 0):
            for oz in (-1, 0):
                lvx, lvy, lvz = -ox, -oy, -oz
                lwx, lwy, lwz = lvx + dx, lvy + dy, lvz + dz
                ok = (lwx >= 0) & (lwx <= 1) & (lwy >= 0) & (lwy <= 1) & (lwz >= 0) & (lwz <= 1)
                kv = Kr[lvx + 2 * lvy + 4 * lvz, (lwx + 2 * lwy + 4 * lwz)[ok]]
                cell = ((iz[ok] + 1 + oz) * (ny + 1) + (iy[ok] + 1 + oy)) * (nx + 1) + (ix[ok] + 1 + ox)
                tr.append(k_all[ok])
                tc.append(cell)
                tv.append(kv)
    S_rows, S_cells, S_vals = np.concatenate(tr), np.concatenate(tc), np.concatenate(tv)
    keep = S_vals != 0.0
    return rowptr, colind, S_rows[keep], S_cells[keep], S_vals[keep]


def batch_grids(nsys: int = 64, lo: int = 32, hi: int = 96, seed: int = 0):
    """Grid edges of a batch of 3D systems: each of nx, ny, nz drawn independently and
    uniformly from {lo, ..., hi} with SplitMix64 (seed), in the order sys0 (nx, ny, nz),
    sys1 (nx, ny, nz), ...  Returns a list of (nx, ny, nz)."""
    u = (uniform_pm1(seed, 3 * nsys) + 1.0) * 0.5  # exact: U[0, 1) on the 2^-53 grid
    e = lo + np.minimum(np.floor(u * (hi - lo + 1)).astype(np.int64), hi - lo)
    return [tuple(int(v) for v in e[3 * i:3 * i + 3]) for i in range(nsys)]


def batch_rhs(sys: int, n: int, nrhs: int) -> np.ndarray:
    """Right-hand sides of system `sys` of a batch: U[-1, 1) from SplitMix64 seed 1 + sys,
    right-hand side j taking elements j*n .. (j+1)*n - 1 of the stream.  Shape (nrhs, n)."""
    return uniform_pm1(1 + sys, nrhs * n).reshape(nrhs, n)
