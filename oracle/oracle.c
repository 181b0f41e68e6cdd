/*
 * oracle.c -- plain sequential FP64 restatement of PCG-S (Algorithm 1 + Algorithm 2 of
 * "Scalable s-step Preconditioned Conjugate Gradient with Chebyshev Basis and Gauss-Seidel
 * Gram Solve") and of classical PCG.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark; never by the CUDA library.  Loops are the definitions written out,
 * in the order the paper states them; no blocking, fusion or reordering.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- small helpers */

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double nrm2(int64_t n, const double* a) { return sqrt(dot(n, a, a)); }

/* ---------------------------------------------------------------- operator, preconditioner */

/* y = A x, row by row in CSR order. */
void or_spmv(const or_csr* A, const double* x, double* y) {
  for (int64_t i = 0; i < A->n; ++i) {
    double s = 0.0;
    for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) s += A->vals[k] * x[A->colind[k]];
    y[i] = s;
  }
}

/* Jacobi preconditioner M = diag(A) (Section 1: any SPD M; the tested configurations use
 * Jacobi).  dinv_i = 1 / a_ii. */
int or_jacobi_dinv(const or_csr* A, double* dinv) {
  for (int64_t i = 0; i < A->n; ++i) {
    double d = 0.0;
    int found = 0;
    for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k)
      if (A->colind[k] == i) { d += A->vals[k]; found = 1; }
    if (!found || !(d > 0.0)) return OR_ERR_INVALID;
    dinv[i] = 1.0 / d;
  }
  return OR_OK;
}

/* y = M^{-1} x. */
void or_prec_apply(int prec, int64_t n, const double* dinv, const double* x, double* y) {
  if (prec == OR_PREC_AMG) {
    or_amg_apply(or_current_amg(), x, y);
    return;
  }
  if (prec == OR_PREC_JACOBI) {
    for (int64_t i = 0; i < n; ++i) y[i] = dinv[i] * x[i];
  } else {
    for (int64_t i = 0; i < n; ++i) y[i] = x[i];
  }
}

/* Gershgorin lower bound of spec(M^{-1}A), clamped at 0 (Section 2 sets lambda_min = 0;
 * for the Poisson matrices used here both readings give 0). */
double or_gershgorin_lower(const or_csr* A, int prec) {
  if (prec == OR_PREC_AMG) return 0.0;  /* no cheap bound for a V-cycle: Section 2's 0 */
  double lo = INFINITY;
  for (int64_t i = 0; i < A->n; ++i) {
    double d = 0.0, off = 0.0;
    for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
      if (A->colind[k] == i) d += A->vals[k];
      else off += fabs(A->vals[k]);
    }
    double b = (prec == OR_PREC_JACOBI) ? 1.0 - off / d : d - off;
    if (b < lo) lo = b;
  }
  return lo > 0.0 ? lo : 0.0;
}

/* Power method of Section 2 on M^{-1}A. */
double or_power_lambda_max(const or_csr* A, int prec, const double* dinv, const double* v0,
                           int max_iters, double tol, int* iters_out) {
  int64_t n = A->n;
  double* v = (double*)malloc(sizeof(double) * n);
  double* t = (double*)malloc(sizeof(double) * n);
  double* y = (double*)malloc(sizeof(double) * n);
  double nv = nrm2(n, v0);
  for (int64_t i = 0; i < n; ++i) v[i] = v0[i] / nv;
  double lam = 0.0, lam_prev = 0.0;
  int it = 0;
  for (it = 1; it <= max_iters; ++it) {
    or_spmv(A, v, t);                 /* one SpMV with A ...              */
    or_prec_apply(prec, n, dinv, t, y); /* ... and one application of M^{-1} */
    lam = nrm2(n, y);
    for (int64_t i = 0; i < n; ++i) v[i] = y[i] / lam;
    if (it > 1 && tol > 0.0 && fabs(lam - lam_prev) < tol * fabs(lam)) break;
    lam_prev = lam;
  }
  if (it > max_iters) it = max_iters;
  if (iters_out) *iters_out = it;
  free(v); free(t); free(y);
  return lam;
}

/* Chebyshev scalars of Section 2 (shifted and scaled operator
 * A_hat = c_alpha M^{-1}A - c_sigma I). */
void or_cheb_scalars(double lmin, double lmax, double* c_alpha, double* c_sigma, double* c_gamma) {
  *c_alpha = 2.0 / (lmax - lmin);
  *c_sigma = (lmax + lmin) / (lmax - lmin);
  *c_gamma = 1.0;
}

/* ---------------------------------------------------------------- Algorithm 2 (MPK) */

int or_mpk(const or_csr* A, int prec, const double* dinv, const double* r, int s,
           double c_alpha, double c_sigma, double c_gamma, double* Z, double* P) {
  if (s < 1) return OR_ERR_INVALID;
  int64_t n = A->n;
  double* zp = (double*)malloc(sizeof(double) * n * (size_t)s); /* zp_1 .. zp_s */
#define ZC(j) (Z + (size_t)(j) * n)
#define PC(j) (P + (size_t)(j) * n)
#define ZPC(j) (zp + (size_t)(j) * n)
  /* p_1 = r; zp_1 = p_1; z_1 = M^{-1} zp_1 */
  memcpy(PC(0), r, sizeof(double) * n);
  memcpy(ZPC(0), PC(0), sizeof(double) * n);
  or_prec_apply(prec, n, dinv, ZPC(0), ZC(0));
  if (s > 1) {
    /* p_2 = A z_1; zp_2 = c_alpha p_2 - c_sigma zp_1; z_2 = M^{-1} zp_2 */
    or_spmv(A, ZC(0), PC(1));
    for (int64_t i = 0; i < n; ++i) ZPC(1)[i] = c_alpha * PC(1)[i] - c_sigma * ZPC(0)[i];
    or_prec_apply(prec, n, dinv, ZPC(1), ZC(1));
    /* q = 2 .. s-1 (1-based): three-term Chebyshev recurrence */
    for (int q = 2; q <= s - 1; ++q) {
      double* pq1 = PC(q);          /* p_{q+1} */
      or_spmv(A, ZC(q - 1), pq1);   /* p_{q+1} = A z_q */
      for (int64_t i = 0; i < n; ++i)
        ZPC(q)[i] = 2.0 * c_alpha * pq1[i] - 2.0 * c_sigma * ZPC(q - 1)[i] - c_gamma * ZPC(q - 2)[i];
      or_prec_apply(prec, n, dinv, ZPC(q), ZC(q));
    }
  }
  /* p_{s+1} = A z_s */
  or_spmv(A, ZC(s - 1), PC(s));
#undef ZC
#undef PC
#undef ZPC
  free(zp);
  return OR_OK;
}

/* ---------------------------------------------------------------- reduced (Gram) solves */

/* nu forward Gauss-Seidel sweeps on W alpha = m from alpha^(0) = 0 (Section 3.1,
 * Eq. fgs-iteration, in its plain form on W: (D + L_W) alpha^(l+1) = m - L_W^T alpha^(l)).
 * Entries above the diagonal are read from W itself. */
int or_fgs(int s, const double* W, const double* m, int nu, double* alpha) {
  for (int i = 0; i < s; ++i) {
    double d = W[i + (size_t)i * s];
    if (!(d > 0.0) || !isfinite(d)) return OR_ERR_BREAKDOWN;
  }
  for (int i = 0; i < s; ++i) alpha[i] = 0.0;
  for (int sweep = 0; sweep < nu; ++sweep) {
    for (int i = 0; i < s; ++i) {
      double acc = m[i];
      for (int j = 0; j < s; ++j)
        if (j != i) acc -= W[i + (size_t)j * s] * alpha[j];
      alpha[i] = acc / W[i + (size_t)i * s];
    }
  }
  for (int i = 0; i < s; ++i)
    if (!isfinite(alpha[i])) return OR_ERR_BREAKDOWN;
  return OR_OK;
}

/* Dense Cholesky W = L L^T, then forward and back substitution (the exact Gram solve the
 * paper compares FGS against in Section 3.3). */
int or_chol_solve(int s, const double* W, const double* m, double* alpha) {
  double* L = (double*)calloc((size_t)s * s, sizeof(double));
  double* y = (double*)malloc(sizeof(double) * s);
  int st = OR_OK;
  for (int j = 0; j < s && st == OR_OK; ++j) {
    double d = W[j + (size_t)j * s];
    for (int k = 0; k < j; ++k) d -= L[j + (size_t)k * s] * L[j + (size_t)k * s];
    if (!(d > 0.0) || !isfinite(d)) { st = OR_ERR_BREAKDOWN; break; }
    L[j + (size_t)j * s] = sqrt(d);
    for (int i = j + 1; i < s; ++i) {
      double v = W[i + (size_t)j * s];
      for (int k = 0; k < j; ++k) v -= L[i + (size_t)k * s] * L[j + (size_t)k * s];
      L[i + (size_t)j * s] = v / L[j + (size_t)j * s];
    }
  }
  if (st == OR_OK) {
    for (int i = 0; i < s; ++i) {
      double v = m[i];
      for (int k = 0; k < i; ++k) v -= L[i + (size_t)k * s] * y[k];
      y[i] = v / L[i + (size_t)i * s];
    }
    for (int i = s - 1; i >= 0; --i) {
      double v = y[i];
      for (int k = i + 1; k < s; ++k) v -= L[k + (size_t)i * s] * alpha[k];
      alpha[i] = v / L[i + (size_t)i * s];
    }
  }
  free(L); free(y);
  return st;
}

/* G = X^T Y  (X: n x a, Y: n x b, G: a x b; all column-major). */
void or_gram(int64_t n, int a, const double* X, int b, const double* Y, double* G) {
  for (int j = 0; j < b; ++j)
    for (int i = 0; i < a; ++i)
      G[i + (size_t)j * a] = dot(n, X + (size_t)i * n, Y + (size_t)j * n);
}

static int reduced_solve(int gram, int s, const double* W, const double* m, int nu, double* out) {
  return gram == OR_GRAM_CHOLESKY ? or_chol_solve(s, W, m, out) : or_fgs(s, W, m, nu, out);
}

/* Solve W X = R column by column (the multiple-right-hand-side system defining beta). */
static int reduced_solve_block(int gram, int s, const double* W, const double* R, int nu, double* X) {
  for (int j = 0; j < s; ++j) {
    int st = reduced_solve(gram, s, W, R + (size_t)j * s, nu, X + (size_t)j * s);
    if (st != OR_OK) return st;
  }
  return OR_OK;
}

/* Relative residual ||m - W a|| / ||m|| (Section 3.3, eta_alpha); block version uses the
 * Frobenius norm over all columns (eta_beta). */
static double reduced_relres(int s, int ncol, const double* W, const double* M, const double* X) {
  double num = 0.0, den = 0.0;
  for (int c = 0; c < ncol; ++c)
    for (int i = 0; i < s; ++i) {
      double v = M[i + (size_t)c * s];
      for (int j = 0; j < s; ++j) v -= W[i + (size_t)j * s] * X[j + (size_t)c * s];
      num += v * v;
      den += M[i + (size_t)c * s] * M[i + (size_t)c * s];
    }
  return den > 0.0 ? sqrt(num / den) : 0.0;
}

static int check_gram(int s, const double* W) {
  for (int i = 0; i < s * s; ++i)
    if (!isfinite(W[i])) return OR_ERR_BREAKDOWN;
  for (int i = 0; i < s; ++i)
    if (!(W[i + (size_t)i * s] > 0.0)) return OR_ERR_BREAKDOWN;
  return OR_OK;
}

/* ---------------------------------------------------------------- Algorithm 1 (PCG-S) */

int or_pcgs(const or_csr* A, int prec, const double* b, double* x,
            int s, int nu, double rtol, int max_outer, int algo, int gram,
            double lambda_min, double lambda_max, const double* power_v0, int power_iters,
            double power_tol, or_info* info, double* hist, double* eta_a, double* eta_b) {
  int64_t n = A->n;
  or_info inf;
  memset(&inf, 0, sizeof(inf));
  if (s < 1 || n < 1 || nu < 0 || max_outer < 0) { inf.status = OR_ERR_INVALID; if (info) *info = inf; return OR_ERR_INVALID; }

  double* dinv = (double*)malloc(sizeof(double) * n);
  double* r = (double*)malloc(sizeof(double) * n);
  double* t = (double*)malloc(sizeof(double) * n);
  double* Z = (double*)malloc(sizeof(double) * n * (size_t)s);
  double* P = (double*)malloc(sizeof(double) * n * (size_t)(s + 1));
  double* Q = (double*)malloc(sizeof(double) * n * (size_t)s);
  double* AQ = (double*)malloc(sizeof(double) * n * (size_t)s);
  double* Qn = (double*)malloc(sizeof(double) * n * (size_t)s);
  double* AQn = (double*)malloc(sizeof(double) * n * (size_t)s);
  double* W = (double*)malloc(sizeof(double) * s * s);
  double* G1 = (double*)malloc(sizeof(double) * s * s);
  double* G2 = (double*)malloc(sizeof(double) * s * s);
  double* G3 = (double*)malloc(sizeof(double) * s * s);
  double* G4 = (double*)malloc(sizeof(double) * s * s);
  double* B2 = (double*)malloc(sizeof(double) * s * s);
  double* beta = (double*)malloc(sizeof(double) * s * s);
  double* T = (double*)malloc(sizeof(double) * s * s);
  double* b1 = (double*)malloc(sizeof(double) * s);
  double* g5 = (double*)malloc(sizeof(double) * s);
  double* g6 = (double*)malloc(sizeof(double) * s);
  double* alpha = (double*)malloc(sizeof(double) * s);
  int st = OR_OK;

  if (prec == OR_PREC_JACOBI) {
    st = or_jacobi_dinv(A, dinv);
    if (st != OR_OK) goto done;
  }

  /* Chebyshev interval (Section 2): lambda_min given (Gershgorin or 0), lambda_max from
   * the power method unless given. */
  if (!(lambda_max > 0.0)) {
    int pit = 0;
    lambda_max = or_power_lambda_max(A, prec, dinv, power_v0, power_iters, power_tol, &pit);
  }
  or_cheb_scalars(lambda_min, lambda_max, &inf.c_alpha, &inf.c_sigma, &inf.c_gamma);

  double nb = nrm2(n, b);
  if (nb == 0.0) { /* b = 0: the solution is x = 0 */
    memset(x, 0, sizeof(double) * n);
    inf.status = OR_OK; inf.iters = 0; inf.relres = 0.0; inf.relres_true = 0.0;
    if (hist) hist[0] = 0.0;
    goto done;
  }

  /* line 1: r^(0) = b - A x^(0) */
  or_spmv(A, x, t);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
  double nr = nrm2(n, r);
  if (hist) hist[0] = nr / nb;
  if (!isfinite(nr)) { st = OR_ERR_NONFINITE; goto done; }
  if (nr <= rtol * nb) { inf.iters = 0; inf.relres = nr / nb; st = OR_OK; goto finish; }

  /* line 2-3: [Z, P] = MPK(r^(0)); Q = Z; AQ = P(:, 2:end) */
  or_mpk(A, prec, dinv, r, s, inf.c_alpha, inf.c_sigma, inf.c_gamma, Z, P);
  memcpy(Q, Z, sizeof(double) * n * s);
  memcpy(AQ, P + n, sizeof(double) * n * s);
  /* one-sync form, first pass: W_0 = Z^T AZ, b1 = Z^T r */
  if (algo == OR_ALGO_ONESYNC) {
    or_gram(n, s, Z, s, P + n, W);
    or_gram(n, s, Z, 1, r, b1);
  }

  st = OR_NOT_CONVERGED;
  for (int k = 0; k < max_outer; ++k) {
    if (algo == OR_ALGO_LITERAL) {
      /* line 5: W = Q^T AQ, b1 = Q^T P(:,1), where P(:,1) = r^(k) (Algorithm 2, first line) */
      or_gram(n, s, Q, s, AQ, W);
      or_gram(n, s, Q, 1, r, b1);
    }
    int cs = check_gram(s, W);
    if (cs != OR_OK) { st = cs; break; }
    /* line 6: alpha = FGS(W, b1, nu) */
    cs = reduced_solve(gram, s, W, b1, nu, alpha);
    if (cs != OR_OK) { st = cs; break; }
    if (eta_a) eta_a[k] = reduced_relres(s, 1, W, b1, alpha);
    /* line 7-8: x += Q alpha; r -= AQ alpha */
    for (int64_t i = 0; i < n; ++i) {
      double dx = 0.0, dr = 0.0;
      for (int j = 0; j < s; ++j) { dx += Q[i + (size_t)j * n] * alpha[j]; dr += AQ[i + (size_t)j * n] * alpha[j]; }
      x[i] += dx;
      r[i] -= dr;
    }
    inf.iters = k + 1;
    nr = nrm2(n, r);
    if (hist) hist[k + 1] = nr / nb;
    /* line 9: stop test on the recursively updated residual */
    if (!isfinite(nr)) { st = OR_ERR_NONFINITE; break; }
    if (nr <= rtol * nb) { st = OR_OK; break; }
    if (k + 1 == max_outer) break;

    /* line 10-11: [Z, P] = MPK(r^(k+1)); AQ_new = P(:, 2:end) */
    or_mpk(A, prec, dinv, r, s, inf.c_alpha, inf.c_sigma, inf.c_gamma, Z, P);
    const double* AZ = P + n;
    if (algo == OR_ALGO_LITERAL) {
      /* line 12-13: b2 = -Q^T AQ_new; beta = FGS(W, b2, nu) */
      or_gram(n, s, Q, s, AZ, B2);
      for (int i = 0; i < s * s; ++i) B2[i] = -B2[i];
      cs = reduced_solve_block(gram, s, W, B2, nu, beta);
      if (cs != OR_OK) { st = cs; break; }
      if (eta_b) eta_b[k] = reduced_relres(s, s, W, B2, beta);
    } else {
      /* one reduction over [Q_k, Z_{k+1}] against [AQ_k, AZ_{k+1}, r^(k+1)] */
      or_gram(n, s, Q, s, AQ, G1);   /* Q_k^T AQ_k       */
      or_gram(n, s, Q, s, AZ, G2);   /* Q_k^T AZ_{k+1}   */
      or_gram(n, s, Z, s, AQ, G3);   /* Z_{k+1}^T AQ_k   */
      or_gram(n, s, Z, s, AZ, G4);   /* Z_{k+1}^T AZ_{k+1} */
      or_gram(n, s, Q, 1, r, g5);    /* Q_k^T r^(k+1)    */
      or_gram(n, s, Z, 1, r, g6);    /* Z_{k+1}^T r^(k+1) */
      for (int i = 0; i < s * s; ++i) B2[i] = -G2[i];
      cs = reduced_solve_block(gram, s, W, B2, nu, beta); /* W = W_k, as in line 13 */
      if (cs != OR_OK) { st = cs; break; }
      if (eta_b) eta_b[k] = reduced_relres(s, s, W, B2, beta);
      /* W_{k+1} = (Z + Q beta)^T (AZ + AQ beta) = G4 + G3 beta + beta^T G2 + beta^T G1 beta */
      for (int j = 0; j < s; ++j)       /* T = G1 beta */
        for (int i = 0; i < s; ++i) {
          double v = 0.0;
          for (int l = 0; l < s; ++l) v += G1[i + (size_t)l * s] * beta[l + (size_t)j * s];
          T[i + (size_t)j * s] = v;
        }
      for (int j = 0; j < s; ++j)
        for (int i = 0; i < s; ++i) {
          double v = G4[i + (size_t)j * s];
          for (int l = 0; l < s; ++l) {
            v += G3[i + (size_t)l * s] * beta[l + (size_t)j * s];
            v += beta[l + (size_t)i * s] * G2[l + (size_t)j * s];
            v += beta[l + (size_t)i * s] * T[l + (size_t)j * s];
          }
          W[i + (size_t)j * s] = v;
        }
      /* b1 = Q_{k+1}^T r^(k+1) = g6 + beta^T g5 */
      for (int i = 0; i < s; ++i) {
        double v = g6[i];
        for (int l = 0; l < s; ++l) v += beta[l + (size_t)i * s] * g5[l];
        b1[i] = v;
      }
    }
    /* line 15: Q = Z + Q beta; AQ = AQ_new + AQ beta */
    for (int64_t i = 0; i < n; ++i)
      for (int j = 0; j < s; ++j) {
        double vq = Z[i + (size_t)j * n], va = AZ[i + (size_t)j * n];
        for (int l = 0; l < s; ++l) {
          vq += Q[i + (size_t)l * n] * beta[l + (size_t)j * s];
          va += AQ[i + (size_t)l * n] * beta[l + (size_t)j * s];
        }
        Qn[i + (size_t)j * n] = vq;
        AQn[i + (size_t)j * n] = va;
      }
    memcpy(Q, Qn, sizeof(double) * n * s);
    memcpy(AQ, AQn, sizeof(double) * n * s);
  }

finish:
  inf.relres = nr / nb;
  or_spmv(A, x, t);
  {
    double s2 = 0.0;
    for (int64_t i = 0; i < n; ++i) { double d = b[i] - t[i]; s2 += d * d; }
    inf.relres_true = sqrt(s2) / nb;
  }
done:
  inf.status = st;
  if (info) *info = inf;
  free(dinv); free(r); free(t); free(Z); free(P); free(Q); free(AQ); free(Qn); free(AQn);
  free(W); free(G1); free(G2); free(G3); free(G4); free(B2); free(beta); free(T);
  free(b1); free(g5); free(g6); free(alpha);
  return st;
}

/* ---------------------------------------------------------------- classical PCG */

/* Hestenes-Stiefel preconditioned CG (Section 1; e.g. Saad, Iterative Methods for Sparse
 * Linear Systems, Alg. 9.1).  Same stop test as PCG-S: ||r|| <= rtol ||b|| after each update. */
int or_pcg(const or_csr* A, int prec, const double* b, double* x, double rtol, int max_iters,
           or_info* info, double* hist) {
  int64_t n = A->n;
  or_info inf;
  memset(&inf, 0, sizeof(inf));
  double* dinv = (double*)malloc(sizeof(double) * n);
  double* r = (double*)malloc(sizeof(double) * n);
  double* z = (double*)malloc(sizeof(double) * n);
  double* p = (double*)malloc(sizeof(double) * n);
  double* Ap = (double*)malloc(sizeof(double) * n);
  int st = OR_OK;
  double nr = 0.0;
  if (prec == OR_PREC_JACOBI) {
    st = or_jacobi_dinv(A, dinv);
    if (st != OR_OK) goto done;
  }
  double nb = nrm2(n, b);
  if (nb == 0.0) {
    memset(x, 0, sizeof(double) * n);
    if (hist) hist[0] = 0.0;
    goto done;
  }
  or_spmv(A, x, Ap);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - Ap[i];
  nr = nrm2(n, r);
  if (hist) hist[0] = nr / nb;
  if (!isfinite(nr)) { st = OR_ERR_NONFINITE; goto finish; }
  if (nr <= rtol * nb) goto finish;
  or_prec_apply(prec, n, dinv, r, z);
  memcpy(p, z, sizeof(double) * n);
  double rz = dot(n, r, z);
  st = OR_NOT_CONVERGED;
  for (int j = 0; j < max_iters; ++j) {
    or_spmv(A, p, Ap);
    double pAp = dot(n, p, Ap);
    if (!(pAp > 0.0) || !isfinite(pAp)) { st = OR_ERR_BREAKDOWN; break; }
    double a = rz / pAp;
    for (int64_t i = 0; i < n; ++i) { x[i] += a * p[i]; r[i] -= a * Ap[i]; }
    inf.iters = j + 1;
    nr = nrm2(n, r);
    if (hist) hist[j + 1] = nr / nb;
    if (!isfinite(nr)) { st = OR_ERR_NONFINITE; break; }
    if (nr <= rtol * nb) { st = OR_OK; break; }
    or_prec_apply(prec, n, dinv, r, z);
    double rz_new = dot(n, r, z);
    double be = rz_new / rz;
    rz = rz_new;
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + be * p[i];
  }
finish:
  inf.relres = nr / nb;
  or_spmv(A, x, Ap);
  {
    double s2 = 0.0;
    for (int64_t i = 0; i < n; ++i) { double d = b[i] - Ap[i]; s2 += d * d; }
    inf.relres_true = sqrt(s2) / nb;
  }
done:
  inf.status = st;
  if (info) *info = inf;
  free(dinv); free(r); free(z); free(p); free(Ap);
  return st;
}
