"""Plant plausible mistakes in a copy of the oracle's C source and check that a pin fails.

Each mutation is a one-token slip of the kind a restatement of the PCG-S outer iteration,
the Chebyshev basis recurrence, the FGS iteration, the reduced-solve residuals or textbook PCG
could contain.  The mutated copy is compiled into a
temporary directory; the committed oracle is never modified.
"""
import os
import subprocess

import pytest

import oracle as O

from . import oracle_pins as P
from . import test_oracle_amg as AMG_PINS

SRC = os.path.join(os.path.dirname(O.__file__), "oracle.c")
AMG_SRC = os.path.join(os.path.dirname(O.__file__), "amg.c")

# Slips in amg.c, caught by the AMG pins (tests/test_oracle_amg.py).
AMG_MUTATIONS = {
    "amg_match_takes_weakest": ("if (w > wbest || (w == wbest && best >= 0 && j < best)) {",
                                "if (best < 0 || w < wbest) {"),
    "amg_galerkin_drops_repeat": ("          acc[pos[Jc]] += A->vals[k];", "          acc[pos[Jc]] += 0.0;"),
    "amg_no_post_smoothing": ("  for (int64_t i = 0; i < n; ++i) x[i] += r[i] / L->dl1[i];\n}",
                              "  for (int64_t i = 0; i < n; ++i) x[i] += 0.0 * r[i];\n}"),
    "amg_restriction_sign": ("C->b[L->agg[i]] += r[i];", "C->b[L->agg[i]] -= r[i];"),
    "amg_l1_uses_diagonal_only": ("for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k) s += fabs(L->vals[k]);",
                                  "for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k) s += (L->colind[k] == i) ? L->vals[k] : 0.0;"),
    "amg_prolongation_missing": ("x[i] += C->x[L->agg[i]];", "x[i] += 0.0 * C->x[L->agg[i]];"),
}

MUTATIONS = {
    "spmv_reads_own_row": ("s += A->vals[k] * x[A->colind[k]];", "s += A->vals[k] * x[i];"),
    "jacobi_multiplies_by_diag": ("y[i] = dinv[i] * x[i];", "y[i] = x[i] / dinv[i];"),
    "cheb_sigma_inverted": ("*c_sigma = (lmax + lmin) / (lmax - lmin);", "*c_sigma = (lmax - lmin) / (lmax + lmin);"),
    "mpk_first_step_doubled": ("wj[i] = c_alpha * az[i] - c_sigma * wm1[i];",
                               "wj[i] = 2.0 * c_alpha * az[i] - c_sigma * wm1[i];"),
    "mpk_recurrence_drops_2": ("wj[i] = 2.0 * c_alpha * az[i] - 2.0", "wj[i] = c_alpha * az[i] - 2.0"),
    "mpk_recurrence_sign": ("- 2.0 * c_sigma * wm1[i] - c_gamma", "+ 2.0 * c_sigma * wm1[i] - c_gamma"),
    "mpk_recurrence_index": ("const double* wm2 = W_(j - 2);", "const double* wm2 = W_(j - 1);"),
    "mpk_missing_precond": ("or_prec_apply(prec, n, dinv, wj, Z_(j));", "memcpy(Z_(j), wj, sizeof(double) * n);"),
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
    "literal_b2_sign": ("for (int i = 0; i < s * s; ++i) B[i] = -B[i];", "for (int i = 0; i < s * s; ++i) B[i] = B[i];"),
    "eta_divides_by_product": ("den += M[i + (size_t)c * s] * M[i + (size_t)c * s];",
                               "den += (M[i + (size_t)c * s] - v) * (M[i + (size_t)c * s] - v);"),
    "eta_beta_last_column_only": ("num += v * v;", "num = v * v;"),
    "eta_alpha_before_solve": ("if (eta_a) eta_a[k] = or_reduced_relres(s, 1, W, m, alpha);",
                               "if (eta_a) eta_a[k] = or_reduced_relres(s, 1, W, m, m);"),
}


def build_mutant(tmp_path, target, old, new):
    """Compile oracle.c + amg.c with one replacement in `target` (a source path)."""
    srcs = []
    for path in (SRC, AMG_SRC):
        text = open(path).read()
        if path == target:
            assert text.count(old) == 1, "mutation anchor must occur exactly once"
            text = text.replace(old, new)
        out = tmp_path / os.path.basename(path)
        out.write_text(text)
        srcs.append(str(out))
    (tmp_path / "oracle.h").write_text(open(SRC[:-1] + "h").read())
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", str(lib)] + srcs + ["-lm"])
    return lib


def run_pins(lib, pins):
    failed = []
    with O.use_library(str(lib)):
        for pin in pins:
            try:
                pin()
            except (AssertionError, FloatingPointError, ValueError, IndexError, np_linalg_error()):
                failed.append(pin.__name__)
    return failed


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    lib = build_mutant(tmp_path, SRC, old, new)
    assert run_pins(lib, P.ALL_PINS), f"no pin caught mutation {name}"


AMG_PIN_FUNCS = [getattr(AMG_PINS, k) for k in sorted(dir(AMG_PINS))
                 if k.startswith("test_") and k != "test_amg_rejects_bad_input"]


@pytest.mark.parametrize("name", sorted(AMG_MUTATIONS))
def test_planted_amg_mistake_is_caught(name, tmp_path):
    old, new = AMG_MUTATIONS[name]
    lib = build_mutant(tmp_path, AMG_SRC, old, new)
    assert run_pins(lib, AMG_PIN_FUNCS), f"no AMG pin caught mutation {name}"


def np_linalg_error():
    import numpy as np
    return np.linalg.LinAlgError
