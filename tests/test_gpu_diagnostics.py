"""Reduced-solve diagnostics (Section 3.3 experiments): eta_alpha, eta_beta and the Gram
matrices W_k recorded by the CUDA path, against the oracle's own eta on the same solve.

eta is the relative residual of an s x s solve; both sides form it in FP64 from Gram sums that
agree to ~1e-12 relative, so eta agrees to 1e-6 relative (it divides a residual that is a few
percent of its right-hand side).  Exact (Cholesky) reduced solves give eta at rounding level.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2603_09790_gb300 import inputs as I
from paper_2603_09790_gb300 import sstep

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def run(A, b, **kw):
    with sstep.Solver(A, **kw) as S:
        x = torch.zeros(b.size, dtype=torch.float64, device=DEV)
        info = S.solve(torch.from_numpy(b).to(DEV), x)
        d = S.get_diagnostics()
        bi = S.get_basis_info()
    return info, d, bi


@pytest.mark.parametrize("dims,points,algo,s,nu,K,gram", [
    ((24, 22, 20), 27, "literal", 4, 30, 10, "fgs"), ((24, 22, 20), 27, "onesync", 6, 30, 6, "fgs"),
    ((30, 26, 22), 7, "literal", 8, 60, 4, "fgs"), ((30, 26, 22), 7, "literal", 10, 30, 3, "fgs"),
    ((24, 22, 20), 27, "literal", 4, 3, 10, "fgs_operator"),
    ((24, 22, 20), 27, "onesync", 5, 4, 8, "fgs_operator")])
def test_eta_matches_oracle(dims, points, algo, s, nu, K, gram):
    csr = O.CSR(*I.poisson_csr(dims, points))
    b = np.ones(csr.n)  # the unit right-hand side of the paper's 27-point benchmark
    info, d, bi = run(sstep.Stencil(*dims, points=points), b, s=s, sweeps=nu, rtol=0.0,
                      max_outer=K, algo=algo, gram=gram, power_iters=20, power_tol=0.0)
    assert info.outer_iters == K
    ref = O.pcgs(csr, b, s=s, nu=nu, rtol=0.0, max_outer=K, algo=algo,
                 lambda_min=bi["lambda_min"], lambda_max=bi["lambda_max"], history=True)
    assert d["eta_a"].size == K and d["eta_b"].size == K - 1
    assert np.allclose(d["eta_a"], ref.eta_a, rtol=1e-6, atol=1e-14)
    assert np.allclose(d["eta_b"], ref.eta_b, rtol=1e-6, atol=1e-14)
    assert np.all(d["eta_a"] < 1.0) and np.all(d["eta_b"] < 1.0)


def test_exact_reduced_solves_have_rounding_level_eta():
    dims = (20, 18, 16)
    b = np.ones(int(np.prod(dims)))
    info, d, _ = run(sstep.Stencil(*dims, points=27), b, s=4, gram="cholesky", rtol=0.0,
                     max_outer=8, algo="onesync", lambda_max=2.0)
    assert d["eta_a"].max() < 1e-10 and d["eta_b"].max() < 1e-10


def test_gram_history_is_a_gram_matrix():
    dims = (24, 22, 20)
    b = np.ones(int(np.prod(dims)))
    info, d, _ = run(sstep.Stencil(*dims, points=27), b, s=10, sweeps=30, rtol=0.0, max_outer=9,
                     power_iters=20, power_tol=0.0)
    W = d["W"]
    assert W.shape == (9, 10, 10)
    for Wk in W:
        assert np.allclose(Wk, Wk.T, rtol=1e-10, atol=1e-12 * np.abs(Wk).max())
        dg = np.sqrt(np.diag(Wk))
        Wn = np.abs(Wk) / np.outer(dg, dg)
        assert np.all(np.diag(Wk) > 0) and Wn.max() <= 1.0 + 1e-12   # Cauchy-Schwarz


def test_pcg_has_no_reduced_solves():
    dims = (10, 9, 8)
    b = np.ones(int(np.prod(dims)))
    info, d, _ = run(sstep.Stencil(*dims, points=7), b, algo="pcg", lambda_max=2.0)
    assert d["eta_a"].size == 0 and d["W"].shape[0] == 0
