/*
 * amg.c -- plain FP64 aggregation AMG used as the preconditioner M of the differentiated
 * diffusion workload.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper treats M^{-1} as a black box and uses an external AMG (Section 5, BootCMatchGX's
 * matching-based aggregation); this file defines the concrete AMG that the CUDA library
 * reproduces, written out in its plainest form:
 *
 *  - Strength of the coupling i-j: w_ij = -a_ij / sqrt(a_ii a_jj) (positive for the negative
 *    off-diagonal entries of an M-matrix-like operator; entries with w_ij <= 0 never pair).
 *  - Pairwise matching: rows in increasing order; an unmatched row i pairs with the unmatched
 *    neighbour j != i of largest w_ij > 0 (ties: the lower j); a row without such a neighbour
 *    stays a singleton.  Aggregates are numbered in increasing order of their lowest row.
 *  - One level applies the matching twice (pairs of pairs: aggregates of at most 4 rows):
 *    B = P1^T A P1, second matching on B, P = P1 P2 (unsmoothed, piecewise constant).
 *  - Galerkin coarse operator A_c = P^T A P, summed in a fixed order: coarse row J visits the
 *    fine rows of aggregate J in increasing order and each row's entries in stored order;
 *    the first contribution to an entry initialises it, later ones are added.  Coarse rows are
 *    stored with increasing column indices.
 *  - Smoother: l1-Jacobi, D_l1 = diag(sum_j |a_ij|), one sweep before and one after the coarse
 *    correction (same D on both sides, so the V-cycle is symmetric; l1-Jacobi makes 2 D_l1 - A
 *    SPD, so it is positive definite).
 *  - Coarsening stops at n <= coarse_max (or max_levels); the coarsest system is solved by
 *    dense Cholesky.
 *
 * V-cycle on level l for right-hand side b (x = M_l^{-1} b):
 *   coarsest: x = A_l^{-1} b;
 *   else: x = D^{-1} b; r = b - A_l x; x_c = M_{l+1}^{-1} (P^T r); x = x + P x_c;
 *         x = x + D^{-1} (b - A_l x).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

typedef struct {
  int64_t n, nnz;
  int64_t* rowptr;
  int32_t* colind;
  double* vals;
  double* dl1;    /* l1 row sums */
  int32_t* agg;   /* fine row -> coarse index (not on the coarsest level) */
  int64_t nc;     /* number of aggregates */
  double* chol;   /* coarsest level: lower Cholesky factor, n x n column-major */
  double *x, *b, *r;  /* V-cycle work vectors */
} amg_level;

struct or_amg {
  int nlev;
  amg_level lev[OR_AMG_MAX_LEVELS];
};

static const or_amg* g_current = NULL;

void or_use_amg(const or_amg* M) { g_current = M; }
const or_amg* or_current_amg(void) { return g_current; }

int or_amg_match(const or_csr* A, int32_t* agg, int64_t* nc_out) {
  const int64_t n = A->n;
  int64_t* mate = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  double* diag = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!mate || !diag) {
    free(mate);
    free(diag);
    return OR_ERR_INVALID;
  }
  for (int64_t i = 0; i < n; ++i) {
    mate[i] = -1;
    diag[i] = 0.0;
    for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k)
      if (A->colind[k] == i) diag[i] = A->vals[k];
    if (!(diag[i] > 0.0)) {
      free(mate);
      free(diag);
      return OR_ERR_INVALID;
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    if (mate[i] >= 0) continue;
    int64_t best = -1;
    double wbest = 0.0;
    for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
      const int64_t j = A->colind[k];
      if (j == i || mate[j] >= 0) continue;
      const double w = -A->vals[k] / sqrt(diag[i] * diag[j]);
      if (w > wbest || (w == wbest && best >= 0 && j < best)) {
        best = j;
        wbest = w;
      }
    }
    if (best >= 0) {
      mate[i] = best;
      mate[best] = i;
    } else {
      mate[i] = i;
    }
  }
  int64_t nc = 0;
  for (int64_t i = 0; i < n; ++i)
    if (i <= mate[i]) {  /* the lowest row of its aggregate */
      agg[i] = (int32_t)nc;
      agg[mate[i]] = (int32_t)nc;
      ++nc;
    }
  *nc_out = nc;
  free(mate);
  free(diag);
  return OR_OK;
}

/* A_c = P^T A P for the piecewise-constant P of agg (nc aggregates), in the fixed order above.
 * Allocates the three arrays of the result. */
int or_amg_galerkin(const or_csr* A, const int32_t* agg, int64_t nc, int64_t** rp_out,
                    int32_t** ci_out, double** v_out, int64_t* nnz_out) {
  const int64_t n = A->n;
  /* members of every aggregate in increasing row order (counting sort) */
  int64_t* mptr = (int64_t*)calloc((size_t)nc + 1, sizeof(int64_t));
  int64_t* mem = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
  int64_t* rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc + 1));
  if (!mptr || !mem || !fill || !pos || !rp) return OR_ERR_INVALID;
  for (int64_t i = 0; i < n; ++i) mptr[agg[i] + 1] += 1;
  for (int64_t J = 0; J < nc; ++J) mptr[J + 1] += mptr[J];
  for (int64_t J = 0; J < nc; ++J) fill[J] = mptr[J];
  for (int64_t i = 0; i < n; ++i) mem[fill[agg[i]]++] = i;
  for (int64_t J = 0; J < nc; ++J) pos[J] = -1;
  /* pass 1: count the distinct coarse columns of every coarse row */
  int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
  rp[0] = 0;
  for (int64_t J = 0; J < nc; ++J) {
    int64_t cnt = 0;
    for (int64_t m = mptr[J]; m < mptr[J + 1]; ++m) {
      const int64_t i = mem[m];
      for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
        const int64_t Jc = agg[A->colind[k]];
        if (pos[Jc] < 0) {
          pos[Jc] = cnt;
          cols[cnt++] = Jc;
        }
      }
    }
    for (int64_t t = 0; t < cnt; ++t) pos[cols[t]] = -1;
    rp[J + 1] = rp[J] + cnt;
  }
  const int64_t nnz = rp[nc];
  int32_t* ci = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  double* v = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  double* acc = (double*)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
  /* pass 2: sums in the fixed order, then the row sorted by column */
  for (int64_t J = 0; J < nc; ++J) {
    int64_t cnt = 0;
    for (int64_t m = mptr[J]; m < mptr[J + 1]; ++m) {
      const int64_t i = mem[m];
      for (int64_t k = A->rowptr[i]; k < A->rowptr[i + 1]; ++k) {
        const int64_t Jc = agg[A->colind[k]];
        if (pos[Jc] < 0) {
          pos[Jc] = cnt;
          cols[cnt] = Jc;
          acc[cnt] = A->vals[k];
          ++cnt;
        } else {
          acc[pos[Jc]] += A->vals[k];
        }
      }
    }
    /* insertion sort of (cols, acc) by column: rows are short */
    for (int64_t t = 1; t < cnt; ++t) {
      const int64_t c = cols[t];
      const double a = acc[t];
      int64_t u = t - 1;
      while (u >= 0 && cols[u] > c) {
        cols[u + 1] = cols[u];
        acc[u + 1] = acc[u];
        --u;
      }
      cols[u + 1] = c;
      acc[u + 1] = a;
    }
    for (int64_t t = 0; t < cnt; ++t) {
      ci[rp[J] + t] = (int32_t)cols[t];
      v[rp[J] + t] = acc[t];
      pos[cols[t]] = -1;
    }
  }
  free(mptr);
  free(mem);
  free(fill);
  free(pos);
  free(cols);
  free(acc);
  *rp_out = rp;
  *ci_out = ci;
  *v_out = v;
  *nnz_out = nnz;
  return OR_OK;
}

static void level_free(amg_level* L) {
  free(L->rowptr);
  free(L->colind);
  free(L->vals);
  free(L->dl1);
  free(L->agg);
  free(L->chol);
  free(L->x);
  free(L->b);
  free(L->r);
  memset(L, 0, sizeof(*L));
}

void or_amg_free(or_amg* M) {
  if (!M) return;
  for (int l = 0; l < M->nlev; ++l) level_free(&M->lev[l]);
  free(M);
}

static int copy_csr(const or_csr* A, amg_level* L) {
  const int64_t n = A->n, nnz = A->rowptr[n];
  L->n = n;
  L->nnz = nnz;
  L->rowptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  L->colind = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  L->vals = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!L->rowptr || !L->colind || !L->vals) return OR_ERR_INVALID;
  memcpy(L->rowptr, A->rowptr, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(L->colind, A->colind, sizeof(int32_t) * (size_t)nnz);
  memcpy(L->vals, A->vals, sizeof(double) * (size_t)nnz);
  return OR_OK;
}

static or_csr level_csr(const amg_level* L) {
  or_csr A = {L->n, L->rowptr, L->colind, L->vals};
  return A;
}

/* Dense Cholesky factor of the level's matrix (lower, column-major). */
static int coarse_factor(amg_level* L) {
  const int64_t n = L->n;
  double* a = (double*)calloc((size_t)(n * n > 0 ? n * n : 1), sizeof(double));
  if (!a) return OR_ERR_INVALID;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k) a[i + n * L->colind[k]] = L->vals[k];
  for (int64_t j = 0; j < n; ++j) {
    double d = a[j + n * j];
    for (int64_t k = 0; k < j; ++k) d -= a[j + n * k] * a[j + n * k];
    if (!(d > 0.0)) {
      free(a);
      return OR_ERR_BREAKDOWN;
    }
    const double ljj = sqrt(d);
    a[j + n * j] = ljj;
    for (int64_t i = j + 1; i < n; ++i) {
      double v = a[i + n * j];
      for (int64_t k = 0; k < j; ++k) v -= a[i + n * k] * a[j + n * k];
      a[i + n * j] = v / ljj;
    }
    for (int64_t i = 0; i < j; ++i) a[i + n * j] = 0.0;  /* keep only the lower triangle */
  }
  L->chol = a;
  return OR_OK;
}

int or_amg_setup(const or_csr* A, int64_t coarse_max, int max_levels, or_amg** out) {
  *out = NULL;
  if (max_levels < 1 || max_levels > OR_AMG_MAX_LEVELS || coarse_max < 1) return OR_ERR_INVALID;
  or_amg* M = (or_amg*)calloc(1, sizeof(or_amg));
  if (!M) return OR_ERR_INVALID;
  int st = copy_csr(A, &M->lev[0]);
  M->nlev = 1;
  for (int l = 0; st == OR_OK; ++l) {
    amg_level* L = &M->lev[l];
    const int64_t n = L->n;
    L->dl1 = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    L->x = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    L->b = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    L->r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k) s += fabs(L->vals[k]);
      L->dl1[i] = s;
    }
    if (n <= coarse_max || l + 1 >= max_levels) {
      st = coarse_factor(L);
      break;
    }
    /* two pairwise matchings: aggregates of at most four rows */
    const or_csr Al = level_csr(L);
    int32_t* agg1 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int64_t nc1 = 0, nc = 0, nnzb = 0, nnzc = 0;
    st = or_amg_match(&Al, agg1, &nc1);
    int64_t* rpb = NULL;
    int32_t* cib = NULL;
    double* vb = NULL;
    if (st == OR_OK) st = or_amg_galerkin(&Al, agg1, nc1, &rpb, &cib, &vb, &nnzb);
    int32_t* agg2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nc1 > 0 ? nc1 : 1));
    if (st == OR_OK) {
      const or_csr B = {nc1, rpb, cib, vb};
      st = or_amg_match(&B, agg2, &nc);
    }
    free(rpb);
    free(cib);
    free(vb);
    if (st != OR_OK) {
      free(agg1);
      free(agg2);
      break;
    }
    L->agg = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) L->agg[i] = agg2[agg1[i]];
    L->nc = nc;
    free(agg1);
    free(agg2);
    if (nc == n) {  /* nothing aggregated: this level is the coarsest */
      free(L->agg);
      L->agg = NULL;
      L->nc = 0;
      st = n <= 8 * coarse_max ? coarse_factor(L) : OR_ERR_INVALID;
      break;
    }
    amg_level* C = &M->lev[l + 1];
    C->n = nc;
    st = or_amg_galerkin(&Al, L->agg, nc, &C->rowptr, &C->colind, &C->vals, &nnzc);
    C->nnz = nnzc;
    M->nlev = l + 2;
  }
  if (st != OR_OK) {
    or_amg_free(M);
    return st;
  }
  *out = M;
  return OR_OK;
}

static void vcycle(const or_amg* M, int l, const double* b, double* x) {
  const amg_level* L = &M->lev[l];
  const int64_t n = L->n;
  if (l == M->nlev - 1) {  /* dense Cholesky: L y = b, L^T x = y */
    const double* a = L->chol;
    for (int64_t i = 0; i < n; ++i) {
      double v = b[i];
      for (int64_t k = 0; k < i; ++k) v -= a[i + n * k] * x[k];
      x[i] = v / a[i + n * i];
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double v = x[i];
      for (int64_t k = i + 1; k < n; ++k) v -= a[k + n * i] * x[k];
      x[i] = v / a[i + n * i];
    }
    return;
  }
  const amg_level* C = &M->lev[l + 1];
  double* r = L->r;
  for (int64_t i = 0; i < n; ++i) x[i] = b[i] / L->dl1[i];        /* pre-smoothing from 0 */
  for (int64_t i = 0; i < n; ++i) {                               /* r = b - A x */
    double ax = 0.0;
    for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k) ax += L->vals[k] * x[L->colind[k]];
    r[i] = b[i] - ax;
  }
  for (int64_t J = 0; J < C->n; ++J) C->b[J] = 0.0;               /* b_c = P^T r */
  for (int64_t i = 0; i < n; ++i) C->b[L->agg[i]] += r[i];
  vcycle(M, l + 1, C->b, C->x);                                    /* coarse correction */
  for (int64_t i = 0; i < n; ++i) x[i] += C->x[L->agg[i]];        /* x = x + P x_c */
  for (int64_t i = 0; i < n; ++i) {                               /* post-smoothing */
    double ax = 0.0;
    for (int64_t k = L->rowptr[i]; k < L->rowptr[i + 1]; ++k) ax += L->vals[k] * x[L->colind[k]];
    r[i] = b[i] - ax;
  }
  for (int64_t i = 0; i < n; ++i) x[i] += r[i] / L->dl1[i];
}

void or_amg_apply(const or_amg* M, const double* b, double* x) { vcycle(M, 0, b, x); }

int or_amg_nlevels(const or_amg* M) { return M->nlev; }

int or_amg_level(const or_amg* M, int l, int64_t* n, int64_t* nnz, const int64_t** rowptr,
                 const int32_t** colind, const double** vals, const int32_t** agg) {
  if (!M || l < 0 || l >= M->nlev) return OR_ERR_INVALID;
  const amg_level* L = &M->lev[l];
  if (n) *n = L->n;
  if (nnz) *nnz = L->nnz;
  if (rowptr) *rowptr = L->rowptr;
  if (colind) *colind = L->colind;
  if (vals) *vals = L->vals;
  if (agg) *agg = L->agg;
  return OR_OK;
}
