/*
 * oracle.c -- plain sequential FP64 restatement of PCG-S (the s-step PCG of Section 2 of
 * "Scalable s-step Preconditioned Conjugate Gradient with Chebyshev Basis and Gauss-Seidel
 * Gram Solve": Chebyshev basis, reduced Gram systems, FGS of Section 3.1, block updates) and
 * of classical PCG.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark; never by the CUDA library.  Each operation is its defining formula
 * written out as a loop, taken in the order the method states them; no blocking, fusion or
 * reordering.
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

/* ---------------------------------------------------------------- Chebyshev basis (Section 2) */

/* The s-column Chebyshev basis of Section 2, z_j = T_{j-1}(A_hat) M^{-1} r (j = 1..s) with
 * A_hat = c_alpha M^{-1}A - c_sigma I, and its products with A.
 *
 * T_0 = 1, T_1(t) = t and T_{j+1}(t) = 2t T_j(t) - T_{j-1}(t) give, multiplied through by M,
 * a recurrence on w_j = M z_j that needs one product with A and one application of M^{-1}
 * per new column (the form of Algorithm 2, whose name for w_j is zp_j):
 *   w_1     = r
 *   w_2     = c_alpha (A z_1) - c_sigma w_1
 *   w_{j+1} = 2 c_alpha (A z_j) - 2 c_sigma w_j - c_gamma w_{j-1}       (j >= 2)
 *   z_j     = M^{-1} w_j.
 * Outputs Z = [z_1 .. z_s] and P = [r, A z_1, .., A z_s] (n x (s+1)), as Algorithm 2 does. */
int or_mpk(const or_csr* A, int prec, const double* dinv, const double* r, int s,
           double c_alpha, double c_sigma, double c_gamma, double* Z, double* P) {
  if (s < 1) return OR_ERR_INVALID;
  int64_t n = A->n;
  double* w = (double*)malloc(sizeof(double) * n * (size_t)s); /* w_1 .. w_s */
  /* columns are 1-based: Z_(j) = z_j, AZ_(j) = A z_j = P(:, j+1), W_(j) = w_j */
#define Z_(j) (Z + (size_t)((j) - 1) * n)
#define AZ_(j) (P + (size_t)(j) * n)
#define W_(j) (w + (size_t)((j) - 1) * n)
  memcpy(P, r, sizeof(double) * n);
  for (int j = 1; j <= s; ++j) {
    double* wj = W_(j);
    if (j == 1) {
      memcpy(wj, r, sizeof(double) * n);
    } else if (j == 2) {  /* T_1(t) = t: no doubling, no c_gamma term */
      const double* az = AZ_(1);
      const double* wm1 = W_(1);
      for (int64_t i = 0; i < n; ++i) wj[i] = c_alpha * az[i] - c_sigma * wm1[i];
    } else {              /* three-term recurrence */
      const double* az = AZ_(j - 1);
      const double* wm1 = W_(j - 1);
      const double* wm2 = W_(j - 2);
      for (int64_t i = 0; i < n; ++i) wj[i] = 2.0 * c_alpha * az[i] - 2.0 * c_sigma * wm1[i] - c_gamma * wm2[i];
    }
    or_prec_apply(prec, n, dinv, wj, Z_(j));  /* z_j = M^{-1} w_j */
    or_spmv(A, Z_(j), AZ_(j));                /* A z_j            */
  }
#undef Z_
#undef AZ_
#undef W_
  free(w);
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

/* Relative residual of a reduced solve (Section 3.3): ||M - W X|| / ||M||, the 2-norm for one
 * right-hand side (eta_alpha) and the Frobenius norm over the ncol columns of a block
 * (eta_beta).  0 when M = 0. */
double or_reduced_relres(int s, int ncol, const double* W, const double* M, const double* X) {
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

/* ---------------------------------------------------------------- PCG-S (Section 2, Algorithm 1) */

/* The operations of one outer iteration, each as Section 2 defines it.  Blocks are n x s,
 * column-major; s x s matrices are column-major. */

/* Reduced system for the step (Section 2): W_k = Q_k^T A Q_k, m_k = Q_k^T r^(k). */
static void step_system(int64_t n, int s, const double* Q, const double* AQ, const double* r,
                        double* W, double* m) {
  or_gram(n, s, Q, s, AQ, W);
  or_gram(n, s, Q, 1, r, m);
}

/* New iterate and residual (Section 2): x^(k+1) = x^(k) + Q_k alpha_k,
 * r^(k+1) = r^(k) - (A Q_k) alpha_k. */
static void advance_iterate(int64_t n, int s, const double* Q, const double* AQ,
                            const double* alpha, double* x, double* r) {
  for (int64_t i = 0; i < n; ++i) {
    double dx = 0.0, dr = 0.0;
    for (int j = 0; j < s; ++j) { dx += Q[i + (size_t)j * n] * alpha[j]; dr += AQ[i + (size_t)j * n] * alpha[j]; }
    x[i] += dx;
    r[i] -= dr;
  }
}

/* Right-hand sides of the conjugation system W_k beta_k = -Q_k^T A Z_{k+1} (Section 2: the
 * condition Q_{k+1}^T A Q_k = 0 with Q_{k+1} = Z_{k+1} + Q_k beta_k and W_k symmetric). */
static void conjugation_rhs(int64_t n, int s, const double* Q, const double* AZ, double* B) {
  or_gram(n, s, Q, s, AZ, B);
  for (int i = 0; i < s * s; ++i) B[i] = -B[i];
}

/* Next direction block, Eq. (blockdirupdate), and its product with A without a new SpMV
 * (Section 2): Q_{k+1} = Z_{k+1} + Q_k beta_k, A Q_{k+1} = A Z_{k+1} + (A Q_k) beta_k.
 * Qn, AQn: n x s work blocks; the result is copied back into Q, AQ. */
static void next_directions(int64_t n, int s, const double* Z, const double* AZ, const double* beta,
                            double* Q, double* AQ, double* Qn, double* AQn) {
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

/* One-reduction form: every product the next step needs, taken in one pass over the current
 * vectors Q_k, Z_{k+1}, AQ_k, AZ_{k+1}, r^(k+1):
 *   G1 = Q_k^T AQ_k, G2 = Q_k^T AZ_{k+1}, G3 = Z_{k+1}^T AQ_k, G4 = Z_{k+1}^T AZ_{k+1},
 *   g5 = Q_k^T r^(k+1), g6 = Z_{k+1}^T r^(k+1).
 * With Q_{k+1} = Z_{k+1} + Q_k beta_k (Eq. blockdirupdate) the next reduced system follows on
 * s x s data:
 *   W_{k+1} = Q_{k+1}^T A Q_{k+1} = G4 + G3 beta + beta^T G2 + beta^T G1 beta,
 *   m_{k+1} = Q_{k+1}^T r^(k+1)   = g6 + beta^T g5. */
static void onesync_products(int64_t n, int s, const double* Q, const double* AQ, const double* Z,
                             const double* AZ, const double* r, double* G1, double* G2,
                             double* G3, double* G4, double* g5, double* g6) {
  or_gram(n, s, Q, s, AQ, G1);
  or_gram(n, s, Q, s, AZ, G2);
  or_gram(n, s, Z, s, AQ, G3);
  or_gram(n, s, Z, s, AZ, G4);
  or_gram(n, s, Q, 1, r, g5);
  or_gram(n, s, Z, 1, r, g6);
}

static void onesync_next_system(int s, const double* G1, const double* G2, const double* G3,
                                const double* G4, const double* g5, const double* g6,
                                const double* beta, double* T, double* W, double* m) {
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
  for (int i = 0; i < s; ++i) {
    double v = g6[i];
    for (int l = 0; l < s; ++l) v += beta[l + (size_t)i * s] * g5[l];
    m[i] = v;
  }
}

/* PCG-S: the outer iteration of Section 2 in the order Algorithm 1 takes it.  Per outer
 * iteration k: the step alpha_k from the reduced system (W_k, m_k) by nu FGS sweeps or
 * exactly; x and r advanced; the stop test ||r^(k+1)|| <= rtol ||b||; the Chebyshev basis
 * Z_{k+1} of r^(k+1); beta_k from W_k beta_k = -Q_k^T A Z_{k+1} with the same W_k; the next
 * direction block.  The first block is the basis itself, Q_0 = Z_0. */
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
  double* m = (double*)malloc(sizeof(double) * s);
  double* g5 = (double*)malloc(sizeof(double) * s);
  double* g6 = (double*)malloc(sizeof(double) * s);
  double* alpha = (double*)malloc(sizeof(double) * s);
  const double* AZ = P + n;  /* A Z = P(:, 2:s+1) */
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

  /* initial residual r^(0) = b - A x^(0) */
  or_spmv(A, x, t);
  for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
  double nr = nrm2(n, r);
  if (hist) hist[0] = nr / nb;
  if (!isfinite(nr)) { st = OR_ERR_NONFINITE; goto done; }
  if (nr <= rtol * nb) { inf.iters = 0; inf.relres = nr / nb; st = OR_OK; goto finish; }

  /* first block: Q_0 = Z_0, the Chebyshev basis of r^(0) */
  or_mpk(A, prec, dinv, r, s, inf.c_alpha, inf.c_sigma, inf.c_gamma, Z, P);
  memcpy(Q, Z, sizeof(double) * n * s);
  memcpy(AQ, AZ, sizeof(double) * n * s);
  if (algo == OR_ALGO_ONESYNC) step_system(n, s, Z, AZ, r, W, m);

  st = OR_NOT_CONVERGED;
  for (int k = 0; k < max_outer; ++k) {
    /* step: alpha_k ~ W_k^{-1} m_k */
    if (algo == OR_ALGO_LITERAL) step_system(n, s, Q, AQ, r, W, m);
    int cs = check_gram(s, W);
    if (cs != OR_OK) { st = cs; break; }
    cs = reduced_solve(gram, s, W, m, nu, alpha);
    if (cs != OR_OK) { st = cs; break; }
    if (eta_a) eta_a[k] = or_reduced_relres(s, 1, W, m, alpha);

    advance_iterate(n, s, Q, AQ, alpha, x, r);
    inf.iters = k + 1;
    nr = nrm2(n, r);
    if (hist) hist[k + 1] = nr / nb;
    /* stop test on the recursively updated residual */
    if (!isfinite(nr)) { st = OR_ERR_NONFINITE; break; }
    if (nr <= rtol * nb) { st = OR_OK; break; }
    if (k + 1 == max_outer) break;

    /* Chebyshev basis of r^(k+1): Z_{k+1}, A Z_{k+1} */
    or_mpk(A, prec, dinv, r, s, inf.c_alpha, inf.c_sigma, inf.c_gamma, Z, P);

    /* conjugation: W_k beta_k = -Q_k^T A Z_{k+1} */
    if (algo == OR_ALGO_LITERAL) {
      conjugation_rhs(n, s, Q, AZ, B2);
    } else {
      onesync_products(n, s, Q, AQ, Z, AZ, r, G1, G2, G3, G4, g5, g6);
      for (int i = 0; i < s * s; ++i) B2[i] = -G2[i];
    }
    cs = reduced_solve_block(gram, s, W, B2, nu, beta);
    if (cs != OR_OK) { st = cs; break; }
    if (eta_b) eta_b[k] = or_reduced_relres(s, s, W, B2, beta);
    if (algo == OR_ALGO_ONESYNC) onesync_next_system(s, G1, G2, G3, G4, g5, g6, beta, T, W, m);

    next_directions(n, s, Z, AZ, beta, Q, AQ, Qn, AQn);
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
  free(m); free(g5); free(g6); free(alpha);
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
