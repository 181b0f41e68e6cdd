/*
 * oracle.h -- plain, sequential, FP64 CPU restatement of Chebyshev-basis s-step PCG
 * (PCG-S) with Forward Gauss-Seidel (FGS) Gram solves, and of classical PCG.
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path: only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark load it.  It shares no
 * code, header, helper or constant with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Every routine is written as the paper states it ("Scalable s-step Preconditioned
 * Conjugate Gradient with Chebyshev Basis and Gauss-Seidel Gram Solve"):
 *   - Section 2: the PCG-S outer iteration (Algorithm 1) and the Chebyshev basis built by
 *     its three-term recurrence (Algorithm 2),
 *   - Section 2, Chebyshev scalars alpha, sigma, gamma and the power method for lambda_max,
 *   - Section 3.1, Eq. (fgs-iteration): FGS on the Gram system (plain splitting of W),
 *   - Section 1 (PCG), textbook Hestenes-Stiefel preconditioned CG.
 * The paper reuses the letter alpha for the Chebyshev scale and for the step vector; this
 * code names the Chebyshev scalars c_alpha, c_sigma, c_gamma.
 *
 * Conventions: vectors are plain double arrays of length n; blocks are column-major
 * n x k arrays with leading dimension n; the operator is CSR with int64 row pointers and
 * int32 column indices.  No routine allocates more than O(n s) doubles.  Status codes are
 * the integers listed below.
 */
#ifndef SSTEP_ORACLE_H
#define SSTEP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  OR_OK = 0,
  OR_NOT_CONVERGED = 1,
  OR_ERR_INVALID = 2,
  OR_ERR_BREAKDOWN = 3,   /* W_ii <= 0 or non-finite Gram entry */
  OR_ERR_NONFINITE = 4    /* non-finite residual norm */
};

enum { OR_PREC_NONE = 0, OR_PREC_JACOBI = 1, OR_PREC_AMG = 2 };
enum { OR_ALGO_LITERAL = 0, OR_ALGO_ONESYNC = 1 };
enum { OR_GRAM_FGS = 0, OR_GRAM_CHOLESKY = 1 };

typedef struct {
  int64_t n;
  const int64_t* rowptr;  /* n+1 */
  const int32_t* colind;  /* nnz */
  const double* vals;     /* nnz */
} or_csr;

typedef struct {
  int status;
  int iters;              /* outer iterations (PCG-S) or iterations (PCG) = executed x/r updates */
  double relres;          /* ||r_rec|| / ||b|| at exit (recursively updated residual) */
  double relres_true;     /* ||b - A x|| / ||b|| at exit */
  double c_alpha, c_sigma, c_gamma;
} or_info;

/* y = A x. */
void or_spmv(const or_csr* A, const double* x, double* y);
/* dinv_i = 1 / a_ii  (Jacobi, M = diag(A)). Returns OR_ERR_INVALID if a diagonal is missing or <= 0. */
int or_jacobi_dinv(const or_csr* A, double* dinv);
/* y = M^{-1} x for M = I (dinv ignored) or M = diag(A). */
void or_prec_apply(int prec, int64_t n, const double* dinv, const double* x, double* y);
/* Gershgorin lower bound of the spectrum of M^{-1}A, clamped at 0. */
double or_gershgorin_lower(const or_csr* A, int prec);
/* Power method on M^{-1}A (Section 2): lambda^(l) = ||M^{-1}A v_{l-1}||, ||v_{l-1}|| = 1.
 * Stops when |lambda^(l) - lambda^(l-1)| < tol |lambda^(l)| or after max_iters iterations
 * (tol <= 0: exactly max_iters).  v0 need not be normalised.  Returns lambda, *iters_out. */
double or_power_lambda_max(const or_csr* A, int prec, const double* dinv, const double* v0,
                           int max_iters, double tol, int* iters_out);
/* Chebyshev scalars of Section 2: c_alpha = 2/(lmax-lmin), c_sigma = (lmax+lmin)/(lmax-lmin), c_gamma = 1. */
void or_cheb_scalars(double lmin, double lmax, double* c_alpha, double* c_sigma, double* c_gamma);
/* Algorithm 2: Z (n x s) and P (n x (s+1)) for residual r. zp workspace is internal. */
int or_mpk(const or_csr* A, int prec, const double* dinv, const double* r, int s,
           double c_alpha, double c_sigma, double c_gamma, double* Z, double* P);
/* Eq. (fgs-iteration) written on W itself (plain Gauss-Seidel splitting W = D + L_W + L_W^T):
 * nu forward sweeps from alpha^(0) = 0 on W alpha = m.  W is s x s column-major. */
int or_fgs(int s, const double* W, const double* m, int nu, double* alpha);
/* Dense Cholesky solve of W alpha = m (W SPD, s x s column-major). */
int or_chol_solve(int s, const double* W, const double* m, double* alpha);
/* Gram products: G = X^T Y with X n x a, Y n x b (column-major), G a x b column-major. */
void or_gram(int64_t n, int a, const double* X, int b, const double* Y, double* G);

/* Relative residual of a reduced solve (Section 3.3): ||M - W X|| / ||M|| over ncol columns
 * (2-norm for ncol = 1: eta_alpha; Frobenius norm for a block: eta_beta).  W s x s, M and X
 * s x ncol, column-major. */
double or_reduced_relres(int s, int ncol, const double* W, const double* M, const double* X);

/* PCG-S (Section 2, Algorithm 1).  x holds x^(0) on entry and the solution on exit.
 * algo: OR_ALGO_LITERAL forms W_k = Q_k^T A Q_k and m_k = Q_k^T r^(k) after each direction
 *       update and -Q_k^T A Z_{k+1} after each basis (two reductions per outer iteration),
 *       as Algorithm 1 prints it;
 *       OR_ALGO_ONESYNC forms W_{k+1} from the Gram blocks of [Q_k, Z_{k+1}] and beta_k
 *       (algebraically identical; one reduction per outer iteration).
 * gram: OR_GRAM_FGS (nu sweeps) or OR_GRAM_CHOLESKY (exact reduced solves).
 * lambda_max > 0 is used as given; otherwise it is estimated by the power method.
 * hist (optional, length max_outer+1): ||r^(k)|| / ||b||.  eta_a, eta_b (optional, length
 * max_outer): reduced-solve relative residuals of Section 3.3. */
int or_pcgs(const or_csr* A, int prec, const double* b, double* x,
            int s, int nu, double rtol, int max_outer, int algo, int gram,
            double lambda_min, double lambda_max, const double* power_v0, int power_iters,
            double power_tol, or_info* info, double* hist, double* eta_a, double* eta_b);

/* Classical preconditioned CG (Hestenes-Stiefel).  hist optional, length max_iters+1. */
int or_pcg(const or_csr* A, int prec, const double* b, double* x, double rtol, int max_iters,
           or_info* info, double* hist);

/* ---- aggregation AMG (amg.c): the preconditioner OR_PREC_AMG.  The paper uses an external
 * AMG as a black box M (Section 5); amg.c states the concrete one: double pairwise greedy
 * matching on w_ij = -a_ij / sqrt(a_ii a_jj), unsmoothed aggregation, Galerkin coarse
 * operators, l1-Jacobi pre/post smoothing, dense Cholesky on the coarsest level, V-cycle. */
#define OR_AMG_MAX_LEVELS 32
typedef struct or_amg or_amg;
/* One pairwise matching of A's rows: agg[i] = aggregate of row i (aggregates of 1 or 2 rows,
 * numbered by their lowest row); *nc = number of aggregates. */
int or_amg_match(const or_csr* A, int32_t* agg, int64_t* nc);
/* A_c = P^T A P for the aggregation agg (nc aggregates); allocates *rowptr, *colind, *vals
 * (free with free()). */
int or_amg_galerkin(const or_csr* A, const int32_t* agg, int64_t nc, int64_t** rowptr,
                    int32_t** colind, double** vals, int64_t* nnz);
/* Hierarchy for A: levels until n <= coarse_max or max_levels. */
int or_amg_setup(const or_csr* A, int64_t coarse_max, int max_levels, or_amg** out);
void or_amg_free(or_amg* M);
/* x = M^{-1} b: one V-cycle. */
void or_amg_apply(const or_amg* M, const double* b, double* x);
int or_amg_nlevels(const or_amg* M);
/* Level l's matrix and aggregation map (agg is NULL on the coarsest level); pointers owned by M. */
int or_amg_level(const or_amg* M, int l, int64_t* n, int64_t* nnz, const int64_t** rowptr,
                 const int32_t** colind, const double** vals, const int32_t** agg);
/* The hierarchy that OR_PREC_AMG applies in or_prec_apply, or_pcgs and or_pcg. */
void or_use_amg(const or_amg* M);
const or_amg* or_current_amg(void);

#ifdef __cplusplus
}
#endif
#endif
