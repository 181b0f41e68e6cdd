"""Plant plausible mistakes in a copy of the oracle's C source and check that a pin fails.

Each mutation is a one-token slip of the kind a restatement of Algorithm 1, Algorithm 2,
the FGS iteration or textbook PCG could contain.  The mutated copy is compiled into a
temporary directory; the committed oracle is never modified.
"""
import os
import subprocess

import pytest

import oracle as O

from . import oracle_pins as P

SRC = os.path.join(os.path.dirname(O.__file__), "oracle.c")

MUTATIONS = {
    "spmv_reads_own_row": ("s += A->vals[k] * x[A->colind[k]];", "s += A->vals[k] * x[i];"),
    "jacobi_multiplies_by_diag": ("y[i] = dinv[i] * x[i];", "y[i] = x[i] / dinv[i];"),
    "cheb_sigma_inverted": ("*c_sigma = (lmax + lmin) / (lmax - lmin);", "*c_sigma = (lmax - lmin) / (lmax + lmin);"),
    "mpk_first_step_doubled": ("ZPC(1)[i] = c_alpha * PC(1)[i] - c_sigma * ZPC(0)[i];",
                               "ZPC(1)[i] = 2.0 * c_alpha * PC(1)[i] - c_sigma * ZPC(0)[i];"),
    "mpk_recurrence_drops_2": ("ZPC(q)[i] = 2.0 * c_alpha * pq1[i]", "ZPC(q)[i] = c_alpha * pq1[i]"),
    "mpk_recurrence_sign": ("- 2.0 * c_sigma * ZPC(q - 1)[i]", "+ 2.0 * c_sigma * ZPC(q - 1)[i]"),
    "mpk_recurrence_index": ("c_gamma * ZPC(q - 2)[i]", "c_gamma * ZPC(q - 1)[i]"),
    "mpk_missing_precond": ("or_prec_apply(prec, n, dinv, ZPC(q), ZC(q));", "memcpy(ZC(q), ZPC(q), sizeof(double) * n);"),
    "fgs_backward_sweep": ("for (int i = 0; i < s; ++i) {\n      double acc = m[i];",
                           "for (int i = s - 1; i >= 0; --i) {\n      double acc = m[i];"),
    "fgs_warm_start_ones": ("for (int i = 0; i < s; ++i) alpha[i] = 0.0;", "for (int i = 0; i < s; ++i) alpha[i] = 1.0;"),
    "power_no_normalise": ("for (int64_t i = 0; i < n; ++i) v[i] = y[i] / lam;", "for (int64_t i = 0; i < n; ++i) v[i] = y[i];"),
    "pcg_beta_inverted": ("double be = rz_new / rz;", "double be = rz / rz_new;"),
    "pcgs_residual_sign": ("r[i] -= dr;", "r[i] += dr;"),
    "pcgs_beta_transposed": ("vq += Q[i + (size_t)l * n] * beta[l + (size_t)j * s];",
                             "vq += Q[i + (size_t)l * n] * beta[j + (size_t)l * s];"),
    "pcgs_aq_not_updated": ("va += AQ[i + (size_t)l * n] * beta[l + (size_t)j * s];", "va += 0.0;"),
    "onesync_quadratic_sign": ("v += beta[l + (size_t)i * s] * T[l + (size_t)j * s];",
                               "v -= beta[l + (size_t)i * s] * T[l + (size_t)j * s];"),
    "onesync_b1_drops_term": ("v += beta[l + (size_t)i * s] * g5[l];", "v += 0.0 * g5[l];"),
    "literal_b2_sign": ("for (int i = 0; i < s * s; ++i) B2[i] = -B2[i];", "for (int i = 0; i < s * s; ++i) B2[i] = B2[i];"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor must occur exactly once"
    mutated = tmp_path / "oracle.c"
    mutated.write_text(src.replace(old, new))
    (tmp_path / "oracle.h").write_text(open(SRC[:-1] + "h").read())
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", str(lib), str(mutated), "-lm"])
    failed = []
    with O.use_library(str(lib)):
        for pin in P.ALL_PINS:
            try:
                pin()
            except (AssertionError, FloatingPointError, ValueError, np_linalg_error()):
                failed.append(pin.__name__)
    assert failed, f"no pin caught mutation {name}"


def np_linalg_error():
    import numpy as np
    return np.linalg.LinAlgError
