"""The Q1 variable-coefficient diffusion generator against closed forms and its definition."""
import numpy as np

import oracle as O
from paper_2603_09790_gb300 import inputs as I


def test_reference_element():
    K = I.q1_reference_stiffness()
    assert np.allclose(K, K.T) and np.allclose(K.sum(axis=1), 0.0, atol=1e-15)
    # diagonal 1/3; vertices sharing an edge: 0; a face or the body diagonal: -1/12
    for a in range(8):
        for b in range(8):
            d = bin(a ^ b).count("1")
            want = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[d]
            assert abs(K[a, b] - want) < 1e-15
    w = np.linalg.eigvalsh(K)
    assert abs(w[0]) < 1e-14 and w[1] > 0


def test_unit_conductivity_spectrum():
    """kappa = 1: sine modes are eigenvectors with lambda = sum_d k(t_d) m(t_e) m(t_f),
    k(t) = 2 - 2 cos t (1D stiffness), m(t) = (2 + cos t) / 3 (1D mass)."""
    dims = (5, 4, 3)
    nx, ny, nz = dims
    rp, ci, v = I.q1_csr(dims, np.ones((nz + 1, ny + 1, nx + 1)))
    A = O.CSR(rp, ci, v)
    for a, b, c in [(1, 1, 1), (2, 3, 1), (5, 4, 3), (3, 1, 2)]:
        tx, ty, tz = a * np.pi / (nx + 1), b * np.pi / (ny + 1), c * np.pi / (nz + 1)
        k = lambda t: 2 - 2 * np.cos(t)  # noqa: E731
        m = lambda t: (2 + np.cos(t)) / 3  # noqa: E731
        lam = k(tx) * m(ty) * m(tz) + m(tx) * k(ty) * m(tz) + m(tx) * m(ty) * k(tz)
        i = np.arange(nx)[None, None, :] + 1
        j = np.arange(ny)[None, :, None] + 1
        l = np.arange(nz)[:, None, None] + 1
        vec = (np.sin(a * i * np.pi / (nx + 1)) * np.sin(b * j * np.pi / (ny + 1)) *
               np.sin(c * l * np.pi / (nz + 1))).reshape(-1)
        assert np.allclose(O.spmv(A, vec), lam * vec, atol=1e-12)


def test_energy_is_sum_of_cell_energies():
    """u^T A u = sum over cells of kappa_c u_c^T K_ref u_c (u = 0 on the boundary)."""
    dims = (4, 3, 5)
    nx, ny, nz = dims
    kappa = I.lognormal_conductivity((nx + 1, ny + 1, nz + 1), 1.0, 2.0, seed=3)
    rp, ci, v = I.q1_csr(dims, kappa)
    u = I.uniform_pm1(5, nx * ny * nz)
    full = np.zeros((nz + 2, ny + 2, nx + 2))
    full[1:-1, 1:-1, 1:-1] = u.reshape(nz, ny, nx)
    K = I.q1_reference_stiffness()
    e = 0.0
    for cz in range(nz + 1):
        for cy in range(ny + 1):
            for cx in range(nx + 1):
                uc = np.array([full[cz + (q >> 2), cy + ((q >> 1) & 1), cx + (q & 1)] for q in range(8)])
                e += kappa[cz, cy, cx] * uc @ K @ uc
    A = O.CSR(rp, ci, v)
    assert abs(u @ O.spmv(A, u) - e) < 1e-12 * abs(e)


def test_lognormal_field_statistics():
    k = I.lognormal_conductivity((40, 40, 40), sigma=1.0, corr=8.0, seed=0)
    g = np.log(k)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    # neighbouring cells are strongly correlated at correlation length 8
    c = np.corrcoef(g[:, :, :-1].ravel(), g[:, :, 1:].ravel())[0, 1]
    assert c > 0.9
    z = I.normal_pm(0, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_assembly_map_reproduces_csr():
    """The linear map kappa -> vals (used to differentiate through assembly) reproduces q1_csr
    exactly, and is linear: a cell's unit conductivity gives that cell's 8x8 element matrix."""
    dims = (6, 5, 4)
    nx, ny, nz = dims
    kappa = I.lognormal_conductivity((nx + 1, ny + 1, nz + 1), 1.0, 2.0, seed=1)
    rp, ci, v = I.q1_csr(dims, kappa)
    rp2, ci2, sr, sc, sv = I.q1_assembly(dims)
    assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2)
    vals = np.zeros(ci.size)
    np.add.at(vals, sr, sv * kappa.reshape(-1)[sc])
    assert np.abs(vals - v).max() <= 1e-15 * np.abs(v).max()
    # one interior cell switched on: its 8 vertices couple through K_ref and nothing else does
    cx, cy, cz = 2, 2, 2
    e = np.zeros_like(kappa)
    e[cz, cy, cx] = 1.0
    _, _, ve = I.q1_csr(dims, e)
    A = O.CSR(rp, ci, ve).dense()
    K = I.q1_reference_stiffness()
    verts = [((cz - 1 + (q >> 2)) * ny + (cy - 1 + ((q >> 1) & 1))) * nx + (cx - 1 + (q & 1)) for q in range(8)]
    B = np.zeros_like(A)
    for a in range(8):
        for b in range(8):
            B[verts[a], verts[b]] += K[a, b]
    assert np.abs(A - B).max() < 1e-15
