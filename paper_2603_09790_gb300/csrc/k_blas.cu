// k_blas.cu -- tall-skinny block kernels of PCG-S and the PCG comparator.
//
//  * k_gram: one pass over n rows forms every requested dot product L_a^T R_b (Algorithm 1
//    step system W, b1 and the conjugation right-hand sides -Q^T AZ of Section 2; in the
//    one-reduction form, all blocks of [Q_k Z_{k+1}]^T
//    [AQ_k AZ_{k+1} r]).  Rows are staged in shared memory in tiles of 256; each thread owns a
//    few (entry, row-phase) slots, so every FP64 multiply-add of the product is issued once.
//    Per-CTA partials are summed in a fixed order by the last CTA to finish (no grid barrier,
//    bit-reproducible), and that same CTA then solves the reduced systems: FGS sweeps of
//    Section 3.1 (Eq. fgs-iteration) for beta and alpha, and the assembly of W_{k+1}.
//  * k_update: the block updates of Section 2 in one pass: Q <- Z + Q beta, AQ <- AZ + AQ beta
//    (Eq. blockdirupdate), x <- x + Q alpha, r <- r - AQ alpha, ||r||^2 and Algorithm 1's stop test.
//  * PCG vector kernels (x/r/z update with r^T z and ||r||^2; direction update).
#include <algorithm>
#include <cstdlib>

#include "common.cuh"

namespace sstep {

namespace {

constexpr int kGramRows = 256;  // rows per shared-memory tile

// SM count of the current device, cached per device ordinal.
int sm_count() {
  constexpr int kDevs = 64;
  static int sms[kDevs] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= kDevs) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }
  if (!sms[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    sms[dev] = v > 0 ? v : 1;
  }
  return sms[dev];
}

// ---------------------------------------------------------------- reduced-system tail

// nu forward Gauss-Seidel sweeps from x = 0 on W x = b (W: s x s column-major in shared memory),
// Eq. (fgs-iteration) in its plain form on W: x_i <- (b_i - sum_{j != i} W_ij x_j) / W_ii, rows
// in increasing order, the rows above i taking this sweep's values.  One warp per right-hand
// side, lane i owning row i.  The part of row i above the diagonal uses the previous sweep's x
// and is formed by all lanes at once; each new x_k is then passed down the warp, so the
// sequential chain per row is one multiply, one shuffle and one FMA instead of a dot product of
// s terms.  The terms above the diagonal are added first, then those below it in increasing
// order.  Executed by the whole CTA.
__device__ void fgs_warp(int s, const double* W, const double* rinv, const double* B, int nrhs,
                         int nu, double* X) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool row = lane < s;
  double wr[kMaxS];
#pragma unroll
  for (int j = 0; j < kMaxS; ++j) wr[j] = (row && j < s) ? W[lane + j * s] : 0.0;
  const double ri = row ? rinv[lane] : 0.0;
  for (int c = warp; c < nrhs; c += nw) {
    const double bi = row ? B[lane + c * s] : 0.0;
    double x = 0.0;
    for (int sw = 0; sw < nu; ++sw) {
      double up = 0.0;
#pragma unroll
      for (int j = 1; j < kMaxS; ++j) {
        const double xj = __shfl_sync(0xffffffffu, x, j);
        if (j > lane && j < s) up = fma(-wr[j], xj, up);
      }
      double acc = bi + up, xn = x;
#pragma unroll
      for (int k = 0; k < kMaxS; ++k) {
        if (k < s) {  // warp-uniform
          if (lane == k) xn = acc * ri;
          const double xk = __shfl_sync(0xffffffffu, xn, k);
          if (lane > k && row) acc = fma(-wr[k], xk, acc);
        }
      }
      x = xn;
    }
    if (row) X[lane + c * s] = x;
  }
}

// fgs_warp with the step size known at compile time: the same operations in the same order
// (bit-identical results), with every loop over the rows exactly s long, so that the chain of
// dependent FP64 operations per sweep is s - 1 multiply-adds (above the diagonal) and s
// (multiply, shuffle, multiply-add) steps, not kMaxS of each.
template <int S>
__device__ void fgs_warp_s(const double* W, const double* rinv, const double* B, int nrhs, int nu,
                           double* X) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const bool row = lane < S;
  double wr[S];
#pragma unroll
  for (int j = 0; j < S; ++j) wr[j] = row ? W[lane + j * S] : 0.0;
  const double ri = row ? rinv[lane] : 0.0;
  for (int c = warp; c < nrhs; c += nw) {
    const double bi = row ? B[lane + c * S] : 0.0;
    double x = 0.0;
    for (int sw = 0; sw < nu; ++sw) {
      double up = 0.0;
#pragma unroll
      for (int j = 1; j < S; ++j) {
        const double xj = __shfl_sync(0xffffffffu, x, j);
        if (j > lane) up = fma(-wr[j], xj, up);
      }
      double acc = bi + up, xn = x;
#pragma unroll
      for (int k = 0; k < S; ++k) {
        if (lane == k) xn = acc * ri;
        const double xk = __shfl_sync(0xffffffffu, xn, k);
        if (lane > k && row) acc = fma(-wr[k], xk, acc);
      }
      x = xn;
    }
    if (row) X[lane + c * S] = x;
  }
}

__device__ void fgs_warp_dispatch(int s, const double* W, const double* rinv, const double* B,
                                  int nrhs, int nu, double* X) {
  switch (s) {
    case 1: fgs_warp_s<1>(W, rinv, B, nrhs, nu, X); return;
    case 2: fgs_warp_s<2>(W, rinv, B, nrhs, nu, X); return;
    case 3: fgs_warp_s<3>(W, rinv, B, nrhs, nu, X); return;
    case 4: fgs_warp_s<4>(W, rinv, B, nrhs, nu, X); return;
    case 8: fgs_warp_s<8>(W, rinv, B, nrhs, nu, X); return;
    default: fgs_warp(s, W, rinv, B, nrhs, nu, X); return;
  }
}

// ---- the FGS operator (solver SSTEP_GRAM_FGS_OPERATOR)
//
// nu sweeps from x = 0 are linear in the right-hand side: with W = D + L + U (diagonal, strictly
// lower, strictly upper), one sweep is x <- T (b - U x), T = (D + L)^{-1}, so
//   x_nu = P_nu b,   P_nu = (I + M + ... + M^{nu-1}) T,   M = -T U = I - T W.
// For s^2 <= 32 one warp holds an s x s matrix one entry per lane (lane i + j s: entry (i, j),
// the column-major index), and P_nu is formed from the binary digits of nu by doubling,
// S_{2m} = S_m + M^m S_m, M^{2m} = M^m M^m, and stepping, S_{m+1} = I + M S_m,
// M^{m+1} = M^m M (S_m = I + ... + M^{m-1}): about 2 log2(nu) + 3 products, each a chain of s
// FP64 multiply-adds, where nu sequential sweeps chain about 3 s dependent operations each.

// (A B)_ij for the s x s matrices held one entry per lane (a = A_ij, b = B_ij in lane i + j s);
// the s products are summed in increasing k by a chain of multiply-adds from 0.
template <int S>
__device__ __forceinline__ double lane_mm(double a, double b, int i, int j) {
  double ak[S], bk[S];
#pragma unroll
  for (int k = 0; k < S; ++k) {
    ak[k] = __shfl_sync(0xffffffffu, a, i + k * S);
    bk[k] = __shfl_sync(0xffffffffu, b, k + j * S);
  }
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < S; ++k) acc = fma(ak[k], bk[k], acc);
  return acc;
}

// P = P_nu(W) into P (s x s column-major, shared memory); rinv[i] = 1 / W_ii.  Executed by all
// 32 lanes of one warp.
template <int S>
__device__ void fgs_operator_s(const double* W, const double* rinv, int nu, double* P) {
  static_assert(S * S <= 32, "one entry per lane");
  const int lane = threadIdx.x & 31;
  const bool in = lane < S * S;
  const int i = in ? lane % S : 0, j = in ? lane / S : 0;
  const double eye = (in && i == j) ? 1.0 : 0.0;
  // T = (D + L)^{-1}, column j by forward substitution: row r is final after step r
  double wl[S];
#pragma unroll
  for (int r = 0; r < S; ++r) wl[r] = W[i + r * S];
  const double ri = rinv[i];
  double t = 0.0, acc = eye;
#pragma unroll
  for (int r = 0; r < S; ++r) {
    if (i == r) t = acc * ri;
    const double tr = __shfl_sync(0xffffffffu, t, r + j * S);
    if (i > r) acc = fma(-wl[r], tr, acc);
  }
  if (nu <= 0) {
    if (in) P[lane] = 0.0;
    return;
  }
  const double m1 = eye - lane_mm<S>(t, in ? W[lane] : 0.0, i, j);  // M = I - T W
  double sum = eye, pw = m1;                                        // S_1 = I, M^1
  for (int bit = 30 - __clz(nu); bit >= 0; --bit) {
    const double ps = lane_mm<S>(pw, sum, i, j);
    const double pp = lane_mm<S>(pw, pw, i, j);
    sum += ps;
    pw = pp;
    if ((nu >> bit) & 1) {
      const double ms = lane_mm<S>(m1, sum, i, j);
      const double pm = lane_mm<S>(pw, m1, i, j);
      sum = eye + ms;
      pw = pm;
    }
  }
  const double p = lane_mm<S>(sum, t, i, j);
  if (in) P[lane] = p;
}

// C = A B for s x s matrices in shared memory (column-major), one entry per thread of the CTA's
// first s^2 threads starting at thread `first`, products summed in increasing k from 0 (the
// order of lane_mm).
__device__ __forceinline__ void smem_mm(int s, const double* A, const double* B, double* C,
                                        int first) {
  const int e = (int)threadIdx.x - first;
  if (e < 0 || e >= s * s) return;
  const int i = e % s, j = e / s;
  double acc = 0.0;
  for (int k = 0; k < s; ++k) acc = fma(A[i + k * s], B[k + j * s], acc);
  C[e] = acc;
}

constexpr int kOpMaxS = 8;  // largest s of the operator form

// fgs_operator_s for 6 <= s <= 8: the same products in the same order, one matrix entry per
// thread through shared memory.  Executed by the whole CTA (blockDim >= 2 s^2).
__device__ void fgs_operator_cta(int s, const double* W, const double* rinv, int nu, double* P) {
  constexpr int Q = kOpMaxS * kOpMaxS;
  __shared__ double T[Q], M1[Q], Sm[Q], Pw[Q], X1[Q], X2[Q];
  const int e = threadIdx.x, ss = s * s;
  const bool in = e < ss;
  const int i = in ? e % s : 0, j = in ? e / s : 0;
  const double eye = (in && i == j) ? 1.0 : 0.0;
  // T = (D + L)^{-1}: row r of every column final after step r
  double acc = eye;
  for (int r = 0; r < s; ++r) {
    if (in && i == r) T[e] = acc * rinv[i];
    __syncthreads();
    if (in && i > r) acc = fma(-W[i + r * s], T[r + j * s], acc);
  }
  __syncthreads();
  if (nu <= 0) {
    if (in) P[e] = 0.0;
    __syncthreads();
    return;
  }
  smem_mm(s, T, W, X1, 0);
  __syncthreads();
  if (in) {
    M1[e] = eye - X1[e];
    Sm[e] = eye;
  }
  __syncthreads();
  if (in) Pw[e] = M1[e];
  __syncthreads();
  for (int bit = 30 - __clz(nu); bit >= 0; --bit) {
    smem_mm(s, Pw, Sm, X1, 0);   // M^m S_m
    smem_mm(s, Pw, Pw, X2, ss);  // (M^m)^2, on the next s^2 threads
    __syncthreads();
    if (in) {
      Sm[e] += X1[e];
      Pw[e] = X2[e];
    }
    __syncthreads();
    if ((nu >> bit) & 1) {
      smem_mm(s, M1, Sm, X1, 0);   // M S_m
      smem_mm(s, Pw, M1, X2, ss);  // M^m M
      __syncthreads();
      if (in) {
        Sm[e] = eye + X1[e];
        Pw[e] = X2[e];
      }
      __syncthreads();
    }
  }
  smem_mm(s, Sm, T, P, 0);
  __syncthreads();
}

// P = P_nu(W) for s <= kOpMaxS; executed by the whole CTA (blockDim >= 2 kOpMaxS^2); ends with
// __syncthreads().  Returns false for larger s.
__device__ bool fgs_operator(int s, const double* W, const double* rinv, int nu, double* P) {
  if (s > kOpMaxS) return false;
  if (s > 5) {
    fgs_operator_cta(s, W, rinv, nu, P);
    return true;
  }
  if (threadIdx.x < 32) {
    switch (s) {
      case 1: fgs_operator_s<1>(W, rinv, nu, P); break;
      case 2: fgs_operator_s<2>(W, rinv, nu, P); break;
      case 3: fgs_operator_s<3>(W, rinv, nu, P); break;
      case 4: fgs_operator_s<4>(W, rinv, nu, P); break;
      default: fgs_operator_s<5>(W, rinv, nu, P); break;
    }
  }
  __syncthreads();
  return true;
}

// X = P B (P: s x s, B and X: s x nrhs, column-major), one entry per thread, the products
// summed in increasing k by a chain of multiply-adds from 0 (the order of lane_mm).
__device__ __forceinline__ void apply_operator(int s, const double* P, const double* B, int nrhs,
                                               double* X) {
  for (int e = threadIdx.x; e < s * nrhs; e += blockDim.x) {
    const int i = e % s, j = e / s;
    double acc = 0.0;
    for (int k = 0; k < s; ++k) acc = fma(P[i + k * s], B[k + j * s], acc);
    X[e] = acc;
  }
}

// Bit tests equivalent to the floating-point checks of the reduced solve, on the integer pipe:
// finite_ok(w) <=> !(w != w) && |w| <= 1.79e308;  diag_ok(d) <=> d > 0 && d <= 1.79e308.
// (Non-negative doubles order like their bit patterns; NaN patterns lie above infinity's.)
__device__ __forceinline__ unsigned long long dbits(double v) {
  return static_cast<unsigned long long>(__double_as_longlong(v));
}
__device__ __forceinline__ bool finite_ok(double w) {
  return (dbits(w) & 0x7FFFFFFFFFFFFFFFull) <= dbits(1.79e308);
}
__device__ __forceinline__ bool diag_ok(double d) {
  return dbits(d) != 0ull && dbits(d) <= dbits(1.79e308);  // sign clear, not +0, not too large
}

// Dense Cholesky factorisation in place (lower triangle of L, column-major), one thread.
__device__ bool chol_factor(int s, const double* W, double* L) {
  for (int j = 0; j < s; ++j) {
    double d = W[j + j * s];
    for (int k = 0; k < j; ++k) d -= L[j + k * s] * L[j + k * s];
    if (!(d > 0.0) || d > 1.79e308) return false;
    const double ljj = sqrt(d);
    L[j + j * s] = ljj;
    for (int i = j + 1; i < s; ++i) {
      double v = W[i + j * s];
      for (int k = 0; k < j; ++k) v -= L[i + k * s] * L[j + k * s];
      L[i + j * s] = v / ljj;
    }
  }
  return true;
}

__device__ void chol_column(int s, const double* L, const double* b, double* x, int stride) {
  double y[kMaxS];
  for (int i = 0; i < s; ++i) {
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= L[i + k * s] * y[k];
    y[i] = v / L[i + i * s];
  }
  for (int i = s - 1; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < s; ++k) v -= L[k + i * s] * x[k * stride];
    x[i * stride] = v / L[i + i * s];
  }
}

// Solve W X = B for nrhs columns (B, X column-major s x nrhs in shared memory) with nu FGS
// sweeps or exactly (Cholesky).  Executed by the whole CTA; returns false on breakdown.
//
// The FP64 pipe of this part is narrow: a warp's FP64 instruction occupies its SM sub-partition
// for tens of cycles whether one lane or thirty-two are active, so this serial tail is written
// lane-parallel.  Warp 0 checks the entries and forms the s reciprocals of the diagonal with one
// instruction sequence (lane i: row i); the FGS sweeps run one warp per right-hand side
// (fgs_warp: lane i owns row i, successive right-hand sides on successive warps, which the SM
// schedules on different sub-partitions).
//
// solver SSTEP_GRAM_FGS_OPERATOR (s <= 8; larger s take the sweeps): P_nu(W) is formed into
// scratch[0 .. s*s) (fgs_operator) and X = P_nu B; the caller may keep P for a later system
// with the same W.
__device__ bool reduced_solve(int s, const double* W, const double* B, int nrhs, int nu,
                              int solver, double* X, double* scratch /* s*s + s */) {
  __shared__ int ok;
  const int tid = threadIdx.x;
  if (solver == SSTEP_GRAM_FGS_OPERATOR && s > kOpMaxS) solver = SSTEP_GRAM_FGS;
  if (solver == SSTEP_GRAM_CHOLESKY) {
    if (tid == 0) {
      ok = 1;
      for (int i = 0; i < s; ++i) {
        const double d = W[i + i * s];
        if (!(d > 0.0) || d > 1.79e308) ok = 0;
      }
      for (int i = 0; i < s * s; ++i)
        if (!(W[i] == W[i]) || fabs(W[i]) > 1.79e308) ok = 0;
      if (ok && !chol_factor(s, W, scratch)) ok = 0;
    }
  } else if (tid < 32) {
    // the same predicates as the Cholesky branch's, on the integer pipe
    bool good = true;
    for (int e = tid; e < s * s; e += 32)
      if (!finite_ok(W[e])) good = false;
    if (tid < s) {
      const double d = W[tid + tid * s];
      if (!diag_ok(d)) good = false;
      else scratch[s * s + tid] = 1.0 / d;
    }
    good = __all_sync(0xffffffffu, good);
    if (tid == 0) ok = good ? 1 : 0;
  }
  __syncthreads();
  if (!ok) return false;
  if (solver == SSTEP_GRAM_FGS_OPERATOR) {
    fgs_operator(s, W, scratch + s * s, nu, scratch);
    apply_operator(s, scratch, B, nrhs, X);
  } else if (solver != SSTEP_GRAM_CHOLESKY) {
    fgs_warp_dispatch(s, W, scratch + s * s, B, nrhs, nu, X);
  } else if (tid < nrhs) {
    chol_column(s, scratch, B + tid * s, X + tid * s, 1);
  }
  __syncthreads();
  return true;
}

// Entry layout of the Gram reductions (shared by the host, which lists the pairs, and by the
// tail, which reads them back).  Blocks are s x s; symmetric blocks keep i <= j only unless
// `full` is set.
struct Layout {
  int s, full;
  __host__ __device__ int nsym() const { return full ? s * s : s * (s + 1) / 2; }
  __host__ __device__ int sym(int i, int j) const {  // index inside a symmetric block
    if (full) return i + j * s;
    if (i > j) { int t = i; i = j; j = t; }
    return j * (j + 1) / 2 + i;  // packed upper triangle, column by column
  }
};

// GM_ONESYNC entry order: G1 = Q^T AQ (sym), G2 = Q^T AZ (s^2), [G3 = Z^T AQ (s^2) if full],
// G4 = Z^T AZ (sym), g5 = Q^T r (s), g6 = Z^T r (s).
struct OneSyncIdx {
  Layout L;
  __host__ __device__ int g1(int i, int j) const { return L.sym(i, j); }
  __host__ __device__ int g2(int i, int j) const { return L.nsym() + i + j * L.s; }
  __host__ __device__ int g3(int i, int j) const {  // Z^T AQ, or (Q^T AZ)^T when not full
    return L.full ? L.nsym() + L.s * L.s + i + j * L.s : g2(j, i);
  }
  __host__ __device__ int g4base() const { return L.nsym() + L.s * L.s * (L.full ? 2 : 1); }
  __host__ __device__ int g4(int i, int j) const { return g4base() + L.sym(i, j); }
  __host__ __device__ int g5(int i) const { return g4base() + L.nsym() + i; }
  __host__ __device__ int g6(int i) const { return g5(L.s) + i; }
  __host__ __device__ int count() const { return g6(L.s); }
};

// Keeps W_k, b1_k and alpha_k of outer iteration k = updates so far (executed by the whole CTA;
// plain stores).
__device__ void record_alpha(Ctrl* c, int s, const double* W, const double* b1, const double* a) {
  const int k = c->iters;
  if (!c->red || k > c->red_max) return;
  double* r = c->red + (size_t)k * c->red_stride;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) r[e] = W[e];
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    r[s * s + i] = b1[i];
    r[s * s + s + i] = a[i];
  }
}

// Keeps B2_k and beta_k, formed after update k + 1 (executed by the whole CTA; plain stores).
__device__ void record_beta(Ctrl* c, int s, const double* B, const double* X) {
  const int k = c->iters - 1;
  if (!c->red || k < 0 || k > c->red_max) return;
  double* r = c->red + (size_t)k * c->red_stride + s * s + 2 * s;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
    r[e] = B[e];
    r[s * s + e] = X[e];
  }
}

// Operator form: keeps P_nu(W) (left in scr[0 .. s*s) by reduced_solve) for the next system
// with the same W.
__device__ __forceinline__ void keep_operator(Ctrl* c, int s, const double* scr) {
  if (c->solver != SSTEP_GRAM_FGS_OPERATOR || s > kOpMaxS) return;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) c->P[e] = scr[e];
  if (threadIdx.x == 0) c->p_valid = 1;
}

// Operator form: whether a kept P_nu(W) can serve the next system with the same W.
__device__ __forceinline__ bool can_reuse_operator(const Ctrl* c, int s) {
  return c->solver == SSTEP_GRAM_FGS_OPERATOR && s <= kOpMaxS && c->p_valid;
}

// X = P B with the kept P for the s right-hand sides of the conjugation system (no new checks:
// W passed them when P was formed).  pre: a copy of c->P the kernel loaded into shared memory
// at its start, or null.  Executed by the whole CTA.
__device__ __forceinline__ void reuse_operator(const Ctrl* c, int s, const double* B, double* X,
                                               double* scr, const double* pre) {
  if (!pre) {
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) scr[e] = c->P[e];
    __syncthreads();
    pre = scr;
  }
  apply_operator(s, pre, B, s, X);
  __syncthreads();
}

// Loads c->P into shared memory (all CTAs of a conjugation-system kernel, at its start: the
// last CTA then finds it there).  Executed by the whole CTA; the caller synchronises.
__device__ __forceinline__ void preload_operator(const Ctrl* c, double* pre) {
  if (c->solver != SSTEP_GRAM_FGS_OPERATOR || c->s > kOpMaxS || !c->p_valid) return;
  for (int e = threadIdx.x; e < c->s * c->s; e += blockDim.x) pre[e] = c->P[e];
}

// The tail: executed by the last CTA after the reduction, with the sums in shared memory.
// pre: c->P loaded into shared memory by the kernel (GM_LITERAL_B2 with a kept operator), or null.
__device__ void gram_tail(int mode, Ctrl* c, const double* sums, double* sh,
                          const double* pre = nullptr) {
  const int s = c->s, nu = c->nu, solver = c->solver;
  const Layout L{s, c->full_gram};
  double* W = sh;               // s*s
  double* Bm = W + s * s;       // s*s  right-hand sides
  double* X = Bm + s * s;       // s*s  solutions
  double* T = X + s * s;        // s*s
  double* G1 = T + s * s;       // s*s
  double* G2 = G1 + s * s;      // s*s
  double* G3 = G2 + s * s;      // s*s
  double* b1 = G3 + s * s;      // s
  double* scr = b1 + s;         // s*s + s
  const int tid = threadIdx.x;
  bool ok = true;
  if (mode == GM_ONESYNC_FIRST || mode == GM_LITERAL_W) {
    // the direction update before this reduction added the pending x step (FP32 forms)
    if (tid == 0) c->x_pending = 0;
    // W = V^T AV (V = Z_0 or Q_k), b1 = V^T r;  alpha = FGS(W, b1)       (step system)
    for (int e = tid; e < s * s; e += blockDim.x) {
      const int i = e % s, j = e / s;
      W[e] = sums[L.sym(i, j)];
    }
    for (int i = tid; i < s; i += blockDim.x) b1[i] = sums[L.nsym() + i];
    __syncthreads();
    ok = reduced_solve(s, W, b1, 1, nu, solver, X, scr);
    if (ok) {
      for (int i = tid; i < s; i += blockDim.x) c->alpha[i] = X[i];
      for (int e = tid; e < s * s; e += blockDim.x) c->W[e] = W[e];
      keep_operator(c, s, scr);
      record_alpha(c, s, W, b1, X);
    }
  } else if (mode == GM_LITERAL_B2) {
    // b2 = -Q^T AQ_new; beta = FGS(W, b2)                                    (conjugation)
    const bool reuse = can_reuse_operator(c, s);
    for (int e = tid; e < s * s; e += blockDim.x) {
      if (!reuse) W[e] = c->W[e];
      Bm[e] = -sums[e];  // entry e = i + j*s is q_i^T az_j
    }
    __syncthreads();
    if (reuse) reuse_operator(c, s, Bm, X, scr, pre);
    else ok = reduced_solve(s, W, Bm, s, nu, solver, X, scr);
    if (ok) {
      for (int e = tid; e < s * s; e += blockDim.x) c->beta[e] = X[e];
      record_beta(c, s, Bm, X);
    }
  } else if (mode == GM_ONESYNC) {
    const OneSyncIdx I{L};
    for (int e = tid; e < s * s; e += blockDim.x) {
      const int i = e % s, j = e / s;
      W[e] = c->W[e];                 // W_k (the matrix alpha_k was computed with)
      G1[e] = sums[I.g1(i, j)];       // Q_k^T AQ_k
      G2[e] = sums[I.g2(i, j)];       // Q_k^T AZ_{k+1}
      G3[e] = sums[I.g3(i, j)];       // Z_{k+1}^T AQ_k
      Bm[e] = -G2[e];
    }
    __syncthreads();
    // beta_k = FGS(W_k, -Q_k^T AZ_{k+1})                                   (conjugation)
    if (can_reuse_operator(c, s)) reuse_operator(c, s, Bm, X, scr, nullptr);
    else ok = reduced_solve(s, W, Bm, s, nu, solver, X, scr);
    if (ok) {
      for (int e = tid; e < s * s; e += blockDim.x) c->beta[e] = X[e];
      record_beta(c, s, Bm, X);
      __syncthreads();
      // T = G1 beta
      for (int e = tid; e < s * s; e += blockDim.x) {
        const int i = e % s, j = e / s;
        double v = 0.0;
        for (int l = 0; l < s; ++l) v = fma(G1[i + l * s], X[l + j * s], v);
        T[e] = v;
      }
      __syncthreads();
      // W_{k+1} = (Z + Q beta)^T (AZ + AQ beta) = G4 + G3 beta + beta^T G2 + beta^T G1 beta
      for (int e = tid; e < s * s; e += blockDim.x) {
        const int i = e % s, j = e / s;
        double v = sums[I.g4(i, j)];
        for (int l = 0; l < s; ++l) {
          v = fma(G3[i + l * s], X[l + j * s], v);
          v = fma(X[l + i * s], G2[l + j * s], v);
          v = fma(X[l + i * s], T[l + j * s], v);
        }
        Bm[e] = v;  // reuse as W_{k+1}
      }
      // b1 = Q_{k+1}^T r = Z^T r + beta^T Q^T r
      for (int i = tid; i < s; i += blockDim.x) {
        double v = sums[I.g6(i)];
        for (int l = 0; l < s; ++l) v = fma(X[l + i * s], sums[I.g5(l)], v);
        b1[i] = v;
      }
      __syncthreads();
      for (int e = tid; e < s * s; e += blockDim.x) W[e] = Bm[e];
      __syncthreads();
      // alpha_{k+1} = FGS(W_{k+1}, b1)                                     (step system)
      ok = reduced_solve(s, W, b1, 1, nu, solver, T, scr);
      if (ok) {
        for (int i = tid; i < s; i += blockDim.x) c->alpha[i] = T[i];
        for (int e = tid; e < s * s; e += blockDim.x) c->W[e] = W[e];
        keep_operator(c, s, scr);
        record_alpha(c, s, W, b1, T);
      }
    }
  }
  __syncthreads();
  if (tid == 0 && !ok) {
    c->status = SSTEP_ERR_BREAKDOWN;
    c->done = 1;
  }
}

// ---------------------------------------------------------------- Gram kernel

template <int EPT>
__global__ void __launch_bounds__(kThreads) k_gram(GramArgs g, int nch, int rp) {
  if (g.ctrl && g.ctrl->done) return;
  extern __shared__ double sm[];
  const int ldS = kGramRows + 1;  // odd stride: columns fall in different banks
  const int ncols = g.nl + g.nr;
  const int tid = threadIdx.x;
  const int ch = tid % nch, ph = tid / nch;
  const bool active = ph < rp;
  int la[EPT], ra[EPT];
  double acc[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = ch * EPT + k;
    acc[k] = 0.0;
    if (e < g.ne) {
      la[k] = g.pairs[e] >> 8;
      ra[k] = g.nl + (g.pairs[e] & 255);
    } else {
      la[k] = ra[k] = -1;
    }
  }
  for (int64_t tile = blockIdx.x; tile * kGramRows < g.n; tile += gridDim.x) {
    const int64_t p0 = tile * kGramRows;
    const int rows = (int)(g.n - p0 < kGramRows ? g.n - p0 : kGramRows);
    for (int cix = 0; cix < ncols; ++cix) {
      const double* v = cix < g.nl ? g.L[cix] : g.R[cix - g.nl];
      for (int p = tid; p < kGramRows; p += blockDim.x)
        sm[cix * ldS + p] = p < rows ? __ldg(v + p0 + p) : 0.0;
    }
    __syncthreads();
    if (active) {
      for (int p = ph; p < rows; p += rp) {
#pragma unroll
        for (int k = 0; k < EPT; ++k)
          if (la[k] >= 0) acc[k] = fma(sm[la[k] * ldS + p], sm[ra[k] * ldS + p], acc[k]);
      }
    }
    __syncthreads();
  }
  // CTA reduction over row phases, in phase order.
  double* red = sm;  // rp * ne doubles
  if (active) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = ch * EPT + k;
      if (e < g.ne) red[ph * g.ne + e] = acc[k];
    }
  }
  __syncthreads();
  for (int e = tid; e < g.ne; e += blockDim.x) {
    double v = 0.0;
    for (int q = 0; q < rp; ++q) v += red[q * g.ne + e];
    g.partials[(size_t)blockIdx.x * g.ne + e] = v;
  }
  __shared__ bool last;
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(&g.ctrl->ticket[TK_GRAM], 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // Fixed-order sum over CTAs: entry e is summed by threads e, e+ne, ... over CTA slices,
  // then the slices are added: in slice order by one thread when there are at most 32, else by
  // one warp per entry (lane l: slices l, l + 32, ... in order, then a fixed butterfly).
  const int per = max(1, (int)blockDim.x / g.ne);  // threads per entry
  double* part = sm;                                // per * ne
  double* sums = sm + per * g.ne;                   // ne
  for (int idx = tid; idx < per * g.ne; idx += blockDim.x) {  // ne may exceed blockDim.x
    const int e = idx % g.ne, sl = idx / g.ne;
    const int nb = gridDim.x;
    const int b0 = (int)((int64_t)nb * sl / per), b1 = (int)((int64_t)nb * (sl + 1) / per);
    double v = 0.0;
    for (int b = b0; b < b1; ++b) v += __ldcg(g.partials + (size_t)b * g.ne + e);
    part[sl * g.ne + e] = v;
  }
  __syncthreads();
  if (per <= 32) {
    for (int e = tid; e < g.ne; e += blockDim.x) {
      double v = 0.0;
      for (int sl = 0; sl < per; ++sl) v += part[sl * g.ne + e];
      sums[e] = v;
    }
  } else {
    const int lane = tid & 31, w = tid >> 5, nw = blockDim.x >> 5;
    for (int e = w; e < g.ne; e += nw) {
      double v = 0.0;
      for (int sl = lane; sl < per; sl += 32) v += part[sl * g.ne + e];
      v = warp_sum(v);
      if (lane == 0) sums[e] = v;
    }
  }
  __syncthreads();
  if (tid == 0) g.ctrl->ticket[TK_GRAM] = 0u;
  for (int e = tid; e < g.ne; e += blockDim.x) {
    g.ctrl->sums[e] = sums[e];
    if (g.out) g.out[e] = sums[e];
  }
  if (g.mode != GM_SUMS) gram_tail(g.mode, g.ctrl, sums, sums + g.ne);
}

// ---------------------------------------------------------------- register-tiled Gram kernel

// Tall-skinny products X^T Y with every product of an NR x NC tile accumulated in registers:
// a thread streams rows (points) p with a grid stride, loads NR + NC values per row and
// issues NR * NC independent FP64 FMAs, so the FP64 pipe is fed without shared memory or
// barriers in the main loop.  blockIdx.y selects the tile; all tiles of a launch have the
// same shape.  Partials per CTA are written in a fixed order and the last CTA to finish sums
// them (fixed order), then solves the reduced systems exactly as k_gram does.
template <int NR, int NC>
__global__ void __launch_bounds__(kThreads, 1) k_gram_tiled(GramTiles g) {
  if (g.ctrl->done) return;
  constexpr int K = NR * NC;
  const int t = blockIdx.y;
  const double* xp[NR];
  const double* yp[NC];
#pragma unroll
  for (int i = 0; i < NR; ++i) xp[i] = g.x[t][i];
#pragma unroll
  for (int j = 0; j < NC; ++j) yp[j] = g.y[t][j];
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < g.n; p += stride) {
    double xv[NR], yv[NC];
#pragma unroll
    for (int i = 0; i < NR; ++i) xv[i] = __ldg(xp[i] + p);
#pragma unroll
    for (int j = 0; j < NC; ++j) yv[j] = __ldg(yp[j] + p);
#pragma unroll
    for (int i = 0; i < NR; ++i)
#pragma unroll
      for (int j = 0; j < NC; ++j) acc[i * NC + j] = fma(xv[i], yv[j], acc[i * NC + j]);
  }
  // CTA reduction: warp shuffles, then the warps in order.
  __shared__ double buf[kTiledSmem];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) buf[wid * K + k] = v;
  }
  __syncthreads();
  const unsigned int cta = blockIdx.x + gridDim.x * blockIdx.y;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v += buf[w * K + k];
    g.partials[(size_t)cta * K + k] = v;
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int tk = atomicAdd(&g.ctrl->ticket[TK_GRAM], 1u);
    last = (tk == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double* sums = buf;  // ne entries, then the tail's scratch
  {
    __shared__ double tot[kMaxTiles * kTileMaxR * kTileMaxC];
    sum_partials(g.partials, gridDim.x, K, (int)gridDim.y, tot);
    for (int idx = threadIdx.x; idx < (int)gridDim.y * K; idx += blockDim.x) {
      const int e = g.out[idx / K][idx % K];
      if (e >= 0) sums[e] = tot[idx];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) g.ctrl->ticket[TK_GRAM] = 0u;
  for (int e = threadIdx.x; e < g.ne; e += blockDim.x) g.ctrl->sums[e] = sums[e];
  gram_tail(g.mode, g.ctrl, sums, sums + g.ne);
}

// ---------------------------------------------------------------- update fused with W, b1

// The direction-block update of outer iteration k (Eq. blockdirupdate) fused with the step
// system of iteration k+1, in one pass: Q <- Z + Q beta, AQ <- AZ + AQ beta (FIRST: the first
// block, Q <- Z, AQ <- AZ), then
// W = Q^T AQ and b1 = Q^T r accumulated in registers from the new columns while they are in
// registers.  W is symmetric by definition (A is), so only its upper triangle is accumulated
// (entry (i, j), i <= j, at tri(i, j) = j (j + 1) / 2 + i; b1_i at S (S + 1) / 2 + i).  The last
// CTA sums the per-CTA partials in a fixed order, mirrors the triangle into the s x s layout
// the reduced-solve tail reads (W_ij at i + j s, b1_i at s^2 + i) and solves alpha = FGS(W, b1).
__host__ __device__ constexpr int tri(int i, int j) { return j * (j + 1) / 2 + i; }

// Mirrors the packed upper triangle of W and the S entries of b1 that follow it into the full
// layout; executed by the whole CTA, ends with __syncthreads().
template <int S>
__device__ __forceinline__ void expand_sym_w(const double* packed, double* full) {
  constexpr int NW = S * (S + 1) / 2;
  for (int e = threadIdx.x; e < S * S + S; e += blockDim.x) {
    if (e < S * S) {
      const int i = e % S, j = e / S;
      full[e] = packed[i <= j ? tri(i, j) : tri(j, i)];
    } else {
      full[e] = packed[NW + e - S * S];
    }
  }
  __syncthreads();
}

template <int S, bool FIRST>
__global__ void __launch_bounds__(kThreads, 1) k_upd_gram(UpdGramArgs a) {
  if (a.ctrl->done) return;
  constexpr int NW = S * (S + 1) / 2;
  constexpr int K = NW + S;
  __shared__ double sb[S * S];
  __shared__ double buf[kTiledSmem];
  __shared__ double pa[S];  // alpha of the previous step, when its x update is pending
  __shared__ int pend;
  if (!FIRST) {
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) sb[e] = a.ctrl->beta[e];
    if (threadIdx.x < S) pa[threadIdx.x] = a.ctrl->alpha[threadIdx.x];
    if (threadIdx.x == 0) pend = a.x ? a.ctrl->x_pending : 0;
  }
  __syncthreads();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  const int64_t ld = a.ld;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += stride) {
    double qn[S], an[S];
    if constexpr (FIRST) {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        qn[j] = __ldg(a.Z + j * ld + p);
        an[j] = __ldg(a.AZ + j * ld + p);
      }
    } else {
      double qo[S], ao[S];
#pragma unroll
      for (int l = 0; l < S; ++l) {
        qo[l] = a.Q[l * ld + p];
        ao[l] = a.AQ[l * ld + p];
      }
      if (pend) {  // x += Q_old alpha_prev: the previous step's x update, deferred to here
        double dx = 0.0;
#pragma unroll
        for (int l = 0; l < S; ++l) dx = fma(qo[l], pa[l], dx);
        a.x[p] += dx;
      }
#pragma unroll
      for (int j = 0; j < S; ++j) {
        double vq = __ldg(a.Z + j * ld + p), va = __ldg(a.AZ + j * ld + p);
#pragma unroll
        for (int l = 0; l < S; ++l) {
          vq = fma(qo[l], sb[l + j * S], vq);
          va = fma(ao[l], sb[l + j * S], va);
        }
        qn[j] = vq;
        an[j] = va;
      }
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      a.Q[j * ld + p] = qn[j];
      a.AQ[j * ld + p] = an[j];
    }
    const double rp = __ldg(a.r + p);
#pragma unroll
    for (int j = 0; j < S; ++j)
#pragma unroll
      for (int i = 0; i <= j; ++i) acc[tri(i, j)] = fma(qn[i], an[j], acc[tri(i, j)]);
#pragma unroll
    for (int i = 0; i < S; ++i) acc[NW + i] = fma(qn[i], rp, acc[NW + i]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) buf[wid * K + k] = v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v += buf[w * K + k];
    a.partials[(size_t)blockIdx.x * K + k] = v;
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int tk = atomicAdd(&a.ctrl->ticket[TK_GRAM], 1u);
    last = (tk == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  sum_partials(a.partials, gridDim.x, K, 1, buf);
  if (threadIdx.x == 0) a.ctrl->ticket[TK_GRAM] = 0u;
  double* sums = buf + K;  // s^2 + s entries in the full layout
  expand_sym_w<S>(buf, sums);
  for (int e = threadIdx.x; e < S * S + S; e += blockDim.x) a.ctrl->sums[e] = sums[e];
  gram_tail(GM_LITERAL_W, a.ctrl, sums, sums + S * S + S);
}

// ---------------------------------------------------------------- mixed path (FP32 basis)

// Conjugation system of Section 2: b2 = -Q^T AZ from FP32 blocks, then beta = FGS(W, b2).
// Four consecutive points per thread and trip (16-byte loads); the next trip's eight vectors are
// loaded before this trip's products, so every thread keeps 256 bytes in flight while it
// computes (two CTAs of 256 threads per SM, 128 registers).
template <int S>
__global__ void __launch_bounds__(kThreads, 2) k_gram_b2f(MixedArgs a) {
  if (a.ctrl->done) return;
  constexpr int K = S * S;
  __shared__ double buf[kTiledSmem];
  __shared__ double pre[S * S];  // the kept FGS operator, for the last CTA's tail
  preload_operator(a.ctrl, pre);  // (visible to the tail after the reduction's barriers)
  float hi[K], lo[K];
#pragma unroll
  for (int k = 0; k < K; ++k) hi[k] = lo[k] = 0.0f;
  const int64_t ld = a.ld;  // a multiple of 64: every column is 16-byte aligned
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = a.n >> 2;
  // column pointers formed once: the loop body indexes them with v alone
  const float4* qc[S];
  const float4* zc[S];
#pragma unroll
  for (int i = 0; i < S; ++i) {
    qc[i] = reinterpret_cast<const float4*>(a.Q + i * ld);
    zc[i] = reinterpret_cast<const float4*>(a.AZ + i * ld);
  }
  float4 q[S], z[S];
  int64_t v = gid;
  if (v < n4) {
#pragma unroll
    for (int i = 0; i < S; ++i) {
      q[i] = __ldg(qc[i] + v);
      z[i] = __ldg(zc[i] + v);
    }
  }
  for (; v < n4; v += stride) {
    float4 qn[S], zn[S];
    const int64_t vn = v + stride;
    if (vn < n4) {
#pragma unroll
      for (int i = 0; i < S; ++i) {
        qn[i] = __ldg(qc[i] + vn);
        zn[i] = __ldg(zc[i] + vn);
      }
    }
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int j = 0; j < S; ++j) df_acc_dot4(hi[i + j * S], lo[i + j * S], q[i], z[j]);
#pragma unroll
    for (int i = 0; i < S; ++i) {
      q[i] = qn[i];
      z[i] = zn[i];
    }
  }
  for (int64_t p = 4 * n4 + gid; p < a.n; p += stride) {  // the last n mod 4 points
    float q[S], z[S];
#pragma unroll
    for (int i = 0; i < S; ++i) q[i] = __ldg(a.Q + i * ld + p);
#pragma unroll
    for (int j = 0; j < S; ++j) z[j] = __ldg(a.AZ + j * ld + p);
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int j = 0; j < S; ++j) df_acc_prod(hi[i + j * S], lo[i + j * S], q[i], z[j]);
  }
  if (!df_grid_sums<K>(hi, lo, buf, a.partials, &a.ctrl->ticket[TK_GRAM])) return;
  for (int e = threadIdx.x; e < K; e += blockDim.x) a.ctrl->sums[e] = buf[e];
  gram_tail(GM_LITERAL_B2, a.ctrl, buf, buf + K, pre);
}

// (xh, xl) += sum_j v_j (alh_j + all_j) in double-float, the operations of the x/r update's
// former x part: the product with the FP32 high part of each step length exactly, its low
// part by one FMA, then one renormalised addition.
template <int NC>
__device__ __forceinline__ void df_axpy_step(const float (&v)[NC], const float* alh,
                                             const float* all, int nc, float& xh, float& xl) {
  float dxh = 0.0f, dxl = 0.0f;
#pragma unroll
  for (int j = 0; j < NC; ++j) {
    if (j < nc) {
      df_acc_prod(dxh, dxl, v[j], alh[j]);
      dxl = fmaf(v[j], all[j], dxl);
    }
  }
  df_add(xh, xl, dxh, dxl);
}

// The pending x step of the FP32 s-step form (ctrl->x_pending, alpha split into FP32 high and
// low parts) in shared memory for a direction-update kernel; executed by the whole CTA, the
// caller synchronises.
template <int S>
struct PendingX {
  float alh[S], all[S];
  int on;
  __device__ void load(const Ctrl* c) {
    if (threadIdx.x == 0) on = c->x_pending;
    if (threadIdx.x < S) {
      const double v = c->alpha[threadIdx.x];
      const float h = __double2float_rn(v);
      alh[threadIdx.x] = h;
      all[threadIdx.x] = __double2float_rn(v - (double)h);
    }
  }
};

// Direction-block update in FP32 (FIRST: Q = Z, AQ = AZ) fused with W = Q^T AQ, b1 = Q^T r
// accumulated in double-float (r = rhi + rlo), then alpha = FGS(W, b1) in the last CTA.
template <int S, bool FIRST>
__global__ void __launch_bounds__(kThreads, 2) k_upd_gramf(MixedArgs a) {
  if (a.ctrl->done) return;
  constexpr int NW = S * (S + 1) / 2;  // upper triangle of W (symmetric), then b1
  constexpr int K = NW + S;
  __shared__ float sb[S * S];
  __shared__ double buf[kTiledSmem];
  __shared__ PendingX<S> px;  // x += Q alpha of the previous step, while Q is read
  if (!FIRST) {
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) sb[e] = (float)a.ctrl->beta[e];
    px.load(a.ctrl);
  }
  __syncthreads();
  float hi[K], lo[K];
#pragma unroll
  for (int k = 0; k < K; ++k) hi[k] = lo[k] = 0.0f;
  const int64_t ld = a.ld;  // a multiple of 64: every column is 16-byte aligned
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  auto accum = [&](const float (&qn)[S], const float (&an)[S], float rh, float rl) {
#pragma unroll
    for (int j = 0; j < S; ++j)
#pragma unroll
      for (int i = 0; i <= j; ++i) df_acc_prod(hi[tri(i, j)], lo[tri(i, j)], qn[i], an[j]);
#pragma unroll
    for (int i = 0; i < S; ++i) {
      df_acc_prod(hi[NW + i], lo[NW + i], qn[i], rh);
      lo[NW + i] = fmaf(qn[i], rl, lo[NW + i]);
    }
  };
  // four consecutive points per thread and trip: 16-byte loads and stores
  const int64_t n4 = a.n >> 2;
  for (int64_t v = gid; v < n4; v += stride) {
    float4 qn4[S], an4[S];
    if constexpr (FIRST) {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        qn4[j] = __ldg(reinterpret_cast<const float4*>(a.Z + j * ld) + v);
        an4[j] = __ldg(reinterpret_cast<const float4*>(a.AZ + j * ld) + v);
      }
    } else {
      float4 qo4[S], ao4[S];
#pragma unroll
      for (int l = 0; l < S; ++l) {
        qo4[l] = reinterpret_cast<const float4*>(a.Q + l * ld)[v];
        ao4[l] = reinterpret_cast<const float4*>(a.AQ + l * ld)[v];
      }
      if (px.on) {  // x += Q_old alpha_prev (the previous step's deferred x update)
        float4 xh = reinterpret_cast<float4*>(a.xhi)[v], xl = reinterpret_cast<float4*>(a.xlo)[v];
        float q[S];
#define SSTEP_PX_LANE(c)                                   \
        for (int l = 0; l < S; ++l) q[l] = qo4[l].c;       \
        df_axpy_step<S>(q, px.alh, px.all, S, xh.c, xl.c);
        SSTEP_PX_LANE(x)
        SSTEP_PX_LANE(y)
        SSTEP_PX_LANE(z)
        SSTEP_PX_LANE(w)
#undef SSTEP_PX_LANE
        reinterpret_cast<float4*>(a.xhi)[v] = xh;
        reinterpret_cast<float4*>(a.xlo)[v] = xl;
      }
#pragma unroll
      for (int j = 0; j < S; ++j) {
        float4 vq = __ldg(reinterpret_cast<const float4*>(a.Z + j * ld) + v);
        float4 va = __ldg(reinterpret_cast<const float4*>(a.AZ + j * ld) + v);
#pragma unroll
        for (int l = 0; l < S; ++l) {
          const float bl = sb[l + j * S];
          vq.x = fmaf(qo4[l].x, bl, vq.x);
          vq.y = fmaf(qo4[l].y, bl, vq.y);
          vq.z = fmaf(qo4[l].z, bl, vq.z);
          vq.w = fmaf(qo4[l].w, bl, vq.w);
          va.x = fmaf(ao4[l].x, bl, va.x);
          va.y = fmaf(ao4[l].y, bl, va.y);
          va.z = fmaf(ao4[l].z, bl, va.z);
          va.w = fmaf(ao4[l].w, bl, va.w);
        }
        qn4[j] = vq;
        an4[j] = va;
      }
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      reinterpret_cast<float4*>(a.Q + j * ld)[v] = qn4[j];
      reinterpret_cast<float4*>(a.AQ + j * ld)[v] = an4[j];
    }
    const float4 rh4 = __ldg(reinterpret_cast<const float4*>(a.rhi) + v);
    const float4 rl4 = __ldg(reinterpret_cast<const float4*>(a.rlo) + v);
    float qn[S], an[S];
#define SSTEP_UPD_LANE(c)                   \
    for (int j = 0; j < S; ++j) {           \
      qn[j] = qn4[j].c;                     \
      an[j] = an4[j].c;                     \
    }                                       \
    accum(qn, an, rh4.c, rl4.c);
    SSTEP_UPD_LANE(x)
    SSTEP_UPD_LANE(y)
    SSTEP_UPD_LANE(z)
    SSTEP_UPD_LANE(w)
#undef SSTEP_UPD_LANE
  }
  for (int64_t p = 4 * n4 + gid; p < a.n; p += stride) {  // the last n mod 4 points
    float qn[S], an[S];
    if constexpr (FIRST) {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        qn[j] = __ldg(a.Z + j * ld + p);
        an[j] = __ldg(a.AZ + j * ld + p);
      }
    } else {
      float qo[S], ao[S];
#pragma unroll
      for (int l = 0; l < S; ++l) {
        qo[l] = a.Q[l * ld + p];
        ao[l] = a.AQ[l * ld + p];
      }
      if (px.on) {  // x += Q_old alpha_prev (deferred)
        float h = a.xhi[p], l = a.xlo[p];
        df_axpy_step<S>(qo, px.alh, px.all, S, h, l);
        a.xhi[p] = h;
        a.xlo[p] = l;
      }
#pragma unroll
      for (int j = 0; j < S; ++j) {
        float vq = __ldg(a.Z + j * ld + p), va = __ldg(a.AZ + j * ld + p);
#pragma unroll
        for (int l = 0; l < S; ++l) {
          vq = fmaf(qo[l], sb[l + j * S], vq);
          va = fmaf(ao[l], sb[l + j * S], va);
        }
        qn[j] = vq;
        an[j] = va;
      }
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      a.Q[j * ld + p] = qn[j];
      a.AQ[j * ld + p] = an[j];
    }
    accum(qn, an, __ldg(a.rhi + p), __ldg(a.rlo + p));
  }
  if (!df_grid_sums<K>(hi, lo, buf, a.partials, &a.ctrl->ticket[TK_GRAM])) return;
  double* sums = buf + K;  // s^2 + s entries in the full layout
  expand_sym_w<S>(buf, sums);
  for (int e = threadIdx.x; e < S * S + S; e += blockDim.x) a.ctrl->sums[e] = sums[e];
  gram_tail(GM_LITERAL_W, a.ctrl, sums, sums + S * S + S);
}

// r -= AQ alpha and the stop test, with r kept as an FP32 (hi, lo) pair between residual
// replacements, ||r||^2 in double-float, stop test in the last CTA.  The step's x += Q alpha is
// left pending (ctrl->x_pending): the next direction update, which reads Q anyway, adds it to
// the FP32 (hi, lo) increments of x, or the fold before a residual replacement does.
template <int S>
__global__ void __launch_bounds__(kThreads) k_update_xrf(MixedArgs a) {
  if (a.ctrl->done) return;
  __shared__ float ah[S], al[S];
  __shared__ double buf[kTiledSmem];
  if (threadIdx.x < S) {
    const double v = a.ctrl->alpha[threadIdx.x];
    const float h = __double2float_rn(v);
    ah[threadIdx.x] = h;
    al[threadIdx.x] = __double2float_rn(v - (double)h);
  }
  __syncthreads();
  float rrh[1] = {0.0f}, rrl[1] = {0.0f};
  const int64_t ld = a.ld;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // one point: r -= AQ alpha in double-float, ||r||^2 accumulated (x += Q alpha is deferred to
  // the next pass that reads Q: the direction update, or the fold before a replacement)
  auto point = [&](const float (&aq)[S], float& rh, float& rl) {
    float drh = 0.0f, drl = 0.0f;
#pragma unroll
    for (int j = 0; j < S; ++j) {
      df_acc_prod(drh, drl, aq[j], ah[j]);
      drl = fmaf(aq[j], al[j], drl);
    }
    df_add(rh, rl, -drh, -drl);
    df_acc_prod(rrh[0], rrl[0], rh, rh);
    rrl[0] = fmaf(2.0f * rh, rl, rrl[0]);
  };
  // four consecutive points per thread and trip with 16-byte loads and stores (ld and the
  // vector lengths are multiples of 64, so every column is 16-byte aligned)
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n4 = a.n >> 2;
  for (int64_t v = gid; v < n4; v += stride) {
    float4 aq4[S];
#pragma unroll
    for (int j = 0; j < S; ++j) aq4[j] = __ldg(reinterpret_cast<const float4*>(a.AQ + j * ld) + v);
    float4 rh = reinterpret_cast<float4*>(a.rhi)[v], rl = reinterpret_cast<float4*>(a.rlo)[v];
    float aq[S];
#define SSTEP_XR_LANE(c)                    \
    for (int j = 0; j < S; ++j) aq[j] = aq4[j].c; \
    point(aq, rh.c, rl.c);
    SSTEP_XR_LANE(x)
    SSTEP_XR_LANE(y)
    SSTEP_XR_LANE(z)
    SSTEP_XR_LANE(w)
#undef SSTEP_XR_LANE
    reinterpret_cast<float4*>(a.rhi)[v] = rh;
    reinterpret_cast<float4*>(a.rlo)[v] = rl;
  }
  for (int64_t p = 4 * n4 + gid; p < a.n; p += stride) {  // the last n mod 4 points
    float aq[S];
#pragma unroll
    for (int j = 0; j < S; ++j) aq[j] = __ldg(a.AQ + j * ld + p);
    float rh = a.rhi[p], rl = a.rlo[p];
    point(aq, rh, rl);
    a.rhi[p] = rh;
    a.rlo[p] = rl;
  }
  if (!df_grid_sums<1>(rrh, rrl, buf, a.partials, &a.ctrl->ticket[TK_UPDATE])) return;
  if (threadIdx.x == 0) {
    a.ctrl->x_pending = 1;  // x lacks Q_k alpha_k
    stop_test(a.ctrl, buf[0]);
    if (a.hist) a.hist[a.ctrl->iters] = sqrt(buf[0] / a.ctrl->nb2);
  }
}

// Direction-block update alone in FP32 (FIRST: Q = Z, AQ = AZ) for step sizes whose fused form would not fit
// in registers; W and b1 then come from k_gram_df.
template <int S, bool FIRST>
__global__ void __launch_bounds__(kThreads) k_upd_qaq_f(MixedArgs a) {
  if (a.ctrl->done) return;
  __shared__ float sb[S * S];
  __shared__ PendingX<S> px;  // x += Q alpha of the previous step, while Q is read
  if (!FIRST) {
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) sb[e] = (float)a.ctrl->beta[e];
    px.load(a.ctrl);
  }
  __syncthreads();
  const int64_t ld = a.ld;  // a multiple of 64: every column is 16-byte aligned
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // four consecutive points per thread and trip: 16-byte loads and stores
  const int64_t n4 = a.n >> 2;
  for (int64_t v = gid; v < n4; v += stride) {
    if constexpr (FIRST) {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        reinterpret_cast<float4*>(a.Q + j * ld)[v] =
            __ldg(reinterpret_cast<const float4*>(a.Z + j * ld) + v);
        reinterpret_cast<float4*>(a.AQ + j * ld)[v] =
            __ldg(reinterpret_cast<const float4*>(a.AZ + j * ld) + v);
      }
    } else {
      float4 qo[S], ao[S];
#pragma unroll
      for (int l = 0; l < S; ++l) {
        qo[l] = reinterpret_cast<const float4*>(a.Q + l * ld)[v];
        ao[l] = reinterpret_cast<const float4*>(a.AQ + l * ld)[v];
      }
      if (px.on) {  // x += Q_old alpha_prev (deferred)
        float4 xh = reinterpret_cast<float4*>(a.xhi)[v], xl = reinterpret_cast<float4*>(a.xlo)[v];
        float q[S];
#define SSTEP_PX_LANE(c)                                   \
        for (int l = 0; l < S; ++l) q[l] = qo[l].c;        \
        df_axpy_step<S>(q, px.alh, px.all, S, xh.c, xl.c);
        SSTEP_PX_LANE(x)
        SSTEP_PX_LANE(y)
        SSTEP_PX_LANE(z)
        SSTEP_PX_LANE(w)
#undef SSTEP_PX_LANE
        reinterpret_cast<float4*>(a.xhi)[v] = xh;
        reinterpret_cast<float4*>(a.xlo)[v] = xl;
      }
#pragma unroll
      for (int j = 0; j < S; ++j) {
        float4 vq = __ldg(reinterpret_cast<const float4*>(a.Z + j * ld) + v);
        float4 va = __ldg(reinterpret_cast<const float4*>(a.AZ + j * ld) + v);
#pragma unroll
        for (int l = 0; l < S; ++l) {
          const float bl = sb[l + j * S];
          vq.x = fmaf(qo[l].x, bl, vq.x);
          vq.y = fmaf(qo[l].y, bl, vq.y);
          vq.z = fmaf(qo[l].z, bl, vq.z);
          vq.w = fmaf(qo[l].w, bl, vq.w);
          va.x = fmaf(ao[l].x, bl, va.x);
          va.y = fmaf(ao[l].y, bl, va.y);
          va.z = fmaf(ao[l].z, bl, va.z);
          va.w = fmaf(ao[l].w, bl, va.w);
        }
        reinterpret_cast<float4*>(a.Q + j * ld)[v] = vq;
        reinterpret_cast<float4*>(a.AQ + j * ld)[v] = va;
      }
    }
  }
  for (int64_t p = 4 * n4 + gid; p < a.n; p += stride) {  // the last n mod 4 points
    if constexpr (FIRST) {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        a.Q[j * ld + p] = __ldg(a.Z + j * ld + p);
        a.AQ[j * ld + p] = __ldg(a.AZ + j * ld + p);
      }
    } else {
      float qo[S], ao[S];
#pragma unroll
      for (int l = 0; l < S; ++l) {
        qo[l] = a.Q[l * ld + p];
        ao[l] = a.AQ[l * ld + p];
      }
      if (px.on) {  // x += Q_old alpha_prev (deferred)
        float h = a.xhi[p], l = a.xlo[p];
        df_axpy_step<S>(qo, px.alh, px.all, S, h, l);
        a.xhi[p] = h;
        a.xlo[p] = l;
      }
#pragma unroll
      for (int j = 0; j < S; ++j) {
        float vq = __ldg(a.Z + j * ld + p), va = __ldg(a.AZ + j * ld + p);
#pragma unroll
        for (int l = 0; l < S; ++l) {
          vq = fmaf(qo[l], sb[l + j * S], vq);
          va = fmaf(ao[l], sb[l + j * S], va);
        }
        a.Q[j * ld + p] = vq;
        a.AQ[j * ld + p] = va;
      }
    }
  }
}

// Direction-block update fused with W = Q^T AQ (its upper triangle: W is symmetric) and
// b1 = Q^T r for 5 <= s <= 8: the work of k_upd_gramf with two points per thread and trip
// (8-byte loads and stores) and one CTA per SM, since the s (s + 1) / 2 + s double-float sums
// take up to 88 registers; the two points of a trip share one update of each low part.  The
// last CTA forms alpha (gram_tail).
template <int S, bool FIRST>
__global__ void __launch_bounds__(kThreads, 1) k_upd_gramwf(MixedArgs a) {
  if (a.ctrl->done) return;
  constexpr int NW = S * (S + 1) / 2;
  constexpr int K = NW + S;
  __shared__ float sb[S * S];
  __shared__ double buf[kTiledSmem];
  __shared__ PendingX<S> px;  // x += Q alpha of the previous step, while Q is read
  if (!FIRST) {
    for (int e = threadIdx.x; e < S * S; e += blockDim.x) sb[e] = (float)a.ctrl->beta[e];
    px.load(a.ctrl);
  }
  __syncthreads();
  float hi[K], lo[K];
#pragma unroll
  for (int k = 0; k < K; ++k) hi[k] = lo[k] = 0.0f;
  const int64_t ld = a.ld;  // a multiple of 64: every column is 16-byte aligned
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n2 = a.n >> 1;
  for (int64_t v = gid; v < n2; v += stride) {
    float2 qn[S], an[S];
    if constexpr (FIRST) {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        qn[j] = __ldg(reinterpret_cast<const float2*>(a.Z + j * ld) + v);
        an[j] = __ldg(reinterpret_cast<const float2*>(a.AZ + j * ld) + v);
      }
    } else {
      float2 qo[S], ao[S];
#pragma unroll
      for (int l = 0; l < S; ++l) {
        qo[l] = reinterpret_cast<const float2*>(a.Q + l * ld)[v];
        ao[l] = reinterpret_cast<const float2*>(a.AQ + l * ld)[v];
      }
      if (px.on) {  // x += Q_old alpha_prev (deferred)
        float2 xh = reinterpret_cast<float2*>(a.xhi)[v], xl = reinterpret_cast<float2*>(a.xlo)[v];
        float q[S];
#pragma unroll
        for (int l = 0; l < S; ++l) q[l] = qo[l].x;
        df_axpy_step<S>(q, px.alh, px.all, S, xh.x, xl.x);
#pragma unroll
        for (int l = 0; l < S; ++l) q[l] = qo[l].y;
        df_axpy_step<S>(q, px.alh, px.all, S, xh.y, xl.y);
        reinterpret_cast<float2*>(a.xhi)[v] = xh;
        reinterpret_cast<float2*>(a.xlo)[v] = xl;
      }
#pragma unroll
      for (int j = 0; j < S; ++j) {
        float2 vq = __ldg(reinterpret_cast<const float2*>(a.Z + j * ld) + v);
        float2 va = __ldg(reinterpret_cast<const float2*>(a.AZ + j * ld) + v);
#pragma unroll
        for (int l = 0; l < S; ++l) {
          const float bl = sb[l + j * S];
          vq.x = fmaf(qo[l].x, bl, vq.x);
          vq.y = fmaf(qo[l].y, bl, vq.y);
          va.x = fmaf(ao[l].x, bl, va.x);
          va.y = fmaf(ao[l].y, bl, va.y);
        }
        qn[j] = vq;
        an[j] = va;
      }
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      reinterpret_cast<float2*>(a.Q + j * ld)[v] = qn[j];
      reinterpret_cast<float2*>(a.AQ + j * ld)[v] = an[j];
    }
    const float2 rh = __ldg(reinterpret_cast<const float2*>(a.rhi) + v);
    const float2 rl = __ldg(reinterpret_cast<const float2*>(a.rlo) + v);
#pragma unroll
    for (int j = 0; j < S; ++j)
#pragma unroll
      for (int i = 0; i <= j; ++i) {
        float& h = hi[tri(i, j)];
        const float l0 = df_step(h, qn[i].x, an[j].x), l1 = df_step(h, qn[i].y, an[j].y);
        lo[tri(i, j)] = __fadd_rn(lo[tri(i, j)], __fadd_rn(l0, l1));
      }
#pragma unroll
    for (int i = 0; i < S; ++i) {
      float& h = hi[NW + i];
      const float l0 = df_step(h, qn[i].x, rh.x), l1 = df_step(h, qn[i].y, rh.y);
      lo[NW + i] = fmaf(qn[i].x, rl.x, fmaf(qn[i].y, rl.y, __fadd_rn(lo[NW + i], __fadd_rn(l0, l1))));
    }
  }
  for (int64_t p = 2 * n2 + gid; p < a.n; p += stride) {  // the last point when n is odd
    float qn[S], an[S];
    if constexpr (FIRST) {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        qn[j] = __ldg(a.Z + j * ld + p);
        an[j] = __ldg(a.AZ + j * ld + p);
      }
    } else {
      float qo[S], ao[S];
#pragma unroll
      for (int l = 0; l < S; ++l) {
        qo[l] = a.Q[l * ld + p];
        ao[l] = a.AQ[l * ld + p];
      }
      if (px.on) {  // x += Q_old alpha_prev (deferred)
        float h = a.xhi[p], l = a.xlo[p];
        df_axpy_step<S>(qo, px.alh, px.all, S, h, l);
        a.xhi[p] = h;
        a.xlo[p] = l;
      }
#pragma unroll
      for (int j = 0; j < S; ++j) {
        float vq = __ldg(a.Z + j * ld + p), va = __ldg(a.AZ + j * ld + p);
#pragma unroll
        for (int l = 0; l < S; ++l) {
          vq = fmaf(qo[l], sb[l + j * S], vq);
          va = fmaf(ao[l], sb[l + j * S], va);
        }
        qn[j] = vq;
        an[j] = va;
      }
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
      a.Q[j * ld + p] = qn[j];
      a.AQ[j * ld + p] = an[j];
    }
    const float rh = __ldg(a.rhi + p), rl = __ldg(a.rlo + p);
#pragma unroll
    for (int j = 0; j < S; ++j)
#pragma unroll
      for (int i = 0; i <= j; ++i) df_acc_prod(hi[tri(i, j)], lo[tri(i, j)], qn[i], an[j]);
#pragma unroll
    for (int i = 0; i < S; ++i) {
      df_acc_prod(hi[NW + i], lo[NW + i], qn[i], rh);
      lo[NW + i] = fmaf(qn[i], rl, lo[NW + i]);
    }
  }
  if (!df_grid_sums<K>(hi, lo, buf, a.partials, &a.ctrl->ticket[TK_GRAM])) return;
  double* sums = buf + K;  // s^2 + s entries in the full layout
  expand_sym_w<S>(buf, sums);
  for (int e = threadIdx.x; e < S * S + S; e += blockDim.x) a.ctrl->sums[e] = sums[e];
  gram_tail(GM_LITERAL_W, a.ctrl, sums, sums + S * S + S);
}

// Register-tiled Gram products of FP32 vectors with double-float accumulation (the FP32
// counterpart of k_gram_tiled).  A column may carry a second FP32 vector (ylo) holding the
// low part of an FP64 vector split as hi + lo.
template <int NR, int NC>
__global__ void __launch_bounds__(kThreads, 2) k_gram_df(GramTilesF g) {
  if (g.ctrl->done) return;
  constexpr int K = NR * NC;
  __shared__ double buf[kTiledSmem];
  const int t = blockIdx.y;
  const float* xp[NR];
  const float* yp[NC];
#pragma unroll
  for (int i = 0; i < NR; ++i) xp[i] = g.x[t][i];
#pragma unroll
  for (int j = 0; j < NC; ++j) yp[j] = g.y[t][j];
  const float* ylo = g.ylo[t][NC - 1];  // only the last column may carry a low part
  float hi[K], lo[K];
#pragma unroll
  for (int k = 0; k < K; ++k) hi[k] = lo[k] = 0.0f;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // four consecutive points per thread and trip (columns are 16-byte aligned): more bytes in
  // flight per thread, one set of index computations per four points
  const int64_t n4 = g.n >> 2;
  for (int64_t v = gid; v < n4; v += stride) {
    float4 xv[NR], yv[NC];
    float4 yl = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
    for (int i = 0; i < NR; ++i) xv[i] = __ldg(reinterpret_cast<const float4*>(xp[i]) + v);
#pragma unroll
    for (int j = 0; j < NC; ++j) yv[j] = __ldg(reinterpret_cast<const float4*>(yp[j]) + v);
    if (ylo) yl = __ldg(reinterpret_cast<const float4*>(ylo) + v);
    // the four points of a trip share one update of each low part (df_acc_dot4)
#pragma unroll
    for (int i = 0; i < NR; ++i) {
#pragma unroll
      for (int j = 0; j < NC; ++j) df_acc_dot4(hi[i * NC + j], lo[i * NC + j], xv[i], yv[j]);
      float& l = lo[i * NC + NC - 1];
      l = fmaf(xv[i].x, yl.x, fmaf(xv[i].y, yl.y, fmaf(xv[i].z, yl.z, fmaf(xv[i].w, yl.w, l))));
    }
  }
  for (int64_t p = 4 * n4 + gid; p < g.n; p += stride) {  // the last n mod 4 points
    float xv[NR], yv[NC];
#pragma unroll
    for (int i = 0; i < NR; ++i) xv[i] = __ldg(xp[i] + p);
#pragma unroll
    for (int j = 0; j < NC; ++j) yv[j] = __ldg(yp[j] + p);
    const float yl = ylo ? __ldg(ylo + p) : 0.0f;
#pragma unroll
    for (int i = 0; i < NR; ++i) {
#pragma unroll
      for (int j = 0; j < NC; ++j) df_acc_prod(hi[i * NC + j], lo[i * NC + j], xv[i], yv[j]);
      lo[i * NC + NC - 1] = fmaf(xv[i], yl, lo[i * NC + NC - 1]);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if constexpr (K <= 64) {
    // the warp stage on the FP32 pipe (reduce-scatter, as in df_grid_sums)
    float vh[DfScatter<K>::C], vl[DfScatter<K>::C];
    df_warp_scatter<K>(hi, lo, vh, vl);
    df_scatter_store<K>(vh, vl, buf + wid * K);
  } else {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const double v = warp_sum((double)hi[k] + (double)lo[k]);
      if (lane == 0) buf[wid * K + k] = v;
    }
  }
  __syncthreads();
  const unsigned int cta = blockIdx.x + gridDim.x * blockIdx.y;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v += buf[w * K + k];
    g.partials[(size_t)cta * K + k] = v;
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(&g.ctrl->ticket[TK_GRAM], 1u) == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double* sums = buf;
  {
    __shared__ double tot[kMaxTiles * kTileMaxR * kTileMaxC];
    sum_partials(g.partials, gridDim.x, K, (int)gridDim.y, tot);
    for (int idx = threadIdx.x; idx < (int)gridDim.y * K; idx += blockDim.x) {
      const int e = g.out[idx / K][idx % K];
      if (e >= 0) sums[e] = tot[idx];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) g.ctrl->ticket[TK_GRAM] = 0u;
  for (int e = threadIdx.x; e < g.ne; e += blockDim.x) g.ctrl->sums[e] = sums[e];
  gram_tail(g.mode, g.ctrl, sums, sums + g.ne);
}

// x64 += xh + xl (increments zeroed), the pending step first (launch_fold_x); the last CTA
// clears the pending flag, which every CTA read at entry.
__global__ void __launch_bounds__(kThreads) k_fold_x(double* x, float* xh, float* xl, int64_t n,
                                                    Ctrl* ctrl, const float* Q, int64_t ld,
                                                    int s) {
  __shared__ float alh[kOpMaxS], all[kOpMaxS];
  __shared__ int pend;
  if (threadIdx.x == 0) pend = ctrl && Q ? ctrl->x_pending : 0;
  if (threadIdx.x < s && ctrl && Q) {
    const double v = ctrl->alpha[threadIdx.x];
    const float h = __double2float_rn(v);
    alh[threadIdx.x] = h;
    all[threadIdx.x] = __double2float_rn(v - (double)h);
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float h = xh[i], l = xl[i];
    if (pend) {
      float v[kOpMaxS];
#pragma unroll
      for (int j = 0; j < kOpMaxS; ++j) v[j] = j < s ? __ldg(Q + j * ld + i) : 0.0f;
      df_axpy_step<kOpMaxS>(v, alh, all, s, h, l);
    }
    x[i] += (double)h + (double)l;
    xh[i] = 0.0f;
    xl[i] = 0.0f;
  }
  if (!ctrl) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctrl->ticket[TK_UPDATE], 1u) == gridDim.x - 1) {
      ctrl->x_pending = 0;
      ctrl->ticket[TK_UPDATE] = 0u;
    }
  }
}

// ---------------------------------------------------------------- fused block update

template <int S, int MODE>
__global__ void __launch_bounds__(kThreads) k_update(UpdArgs u) {
  if (u.ctrl && u.ctrl->done) return;
  __shared__ double sb[S * S], sa[S];
  __shared__ int pend;  // UM_QAQ: the previous step's x update is pending
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) sb[e] = u.beta ? u.beta[e] : 0.0;
  for (int e = threadIdx.x; e < S; e += blockDim.x) sa[e] = u.alpha ? u.alpha[e] : 0.0;
  if (threadIdx.x == 0) pend = (MODE == UM_QAQ && u.ctrl && u.x) ? u.ctrl->x_pending : 0;
  __syncthreads();
  double rr = 0.0;
  const int64_t ld = u.ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < u.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double q[S], aq[S];
    if constexpr (MODE == UM_FIRST) {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        q[j] = __ldg(u.Z + j * ld + i);
        aq[j] = __ldg(u.AZ + j * ld + i);
        u.Q[j * ld + i] = q[j];
        u.AQ[j * ld + i] = aq[j];
      }
    } else if constexpr (MODE == UM_FUSED || MODE == UM_QAQ) {
      double qo[S], ao[S];
#pragma unroll
      for (int l = 0; l < S; ++l) {
        qo[l] = u.Q[l * ld + i];
        ao[l] = u.AQ[l * ld + i];
      }
      if (MODE == UM_QAQ && pend) {  // x += Q_old alpha_prev (deferred; sa holds alpha_prev)
        double dx = 0.0;
#pragma unroll
        for (int l = 0; l < S; ++l) dx = fma(qo[l], sa[l], dx);
        u.x[i] += dx;
      }
#pragma unroll
      for (int j = 0; j < S; ++j) {
        double vq = __ldg(u.Z + j * ld + i), va = __ldg(u.AZ + j * ld + i);
#pragma unroll
        for (int l = 0; l < S; ++l) {
          vq = fma(qo[l], sb[l + j * S], vq);
          va = fma(ao[l], sb[l + j * S], va);
        }
        q[j] = vq;
        aq[j] = va;
        u.Q[j * ld + i] = vq;
        u.AQ[j * ld + i] = va;
      }
    } else if constexpr (MODE == UM_XR) {
#pragma unroll
      for (int j = 0; j < S; ++j) {
        q[j] = u.Q[j * ld + i];
        aq[j] = u.AQ[j * ld + i];
      }
    } else {  // UM_R: Q is not read; x's step stays pending
#pragma unroll
      for (int j = 0; j < S; ++j) aq[j] = u.AQ[j * ld + i];
    }
    if constexpr (MODE != UM_QAQ) {
      double dx = 0.0, dr = 0.0;
#pragma unroll
      for (int j = 0; j < S; ++j) {
        if constexpr (MODE != UM_R) dx = fma(q[j], sa[j], dx);
        dr = fma(aq[j], sa[j], dr);
      }
      if constexpr (MODE != UM_R) u.x[i] += dx;
      const double ri = u.r[i] - dr;
      u.r[i] = ri;
      rr = fma(ri, ri, rr);
    }
  }
  if constexpr (MODE != UM_QAQ) {
    double v[1] = {rr}, tot[1];
    if (grid_sum_last<1>(v, u.partials, u.ticket, tot)) {
      if (threadIdx.x == 0) {
        if (u.ctrl) {
          if (MODE == UM_R) u.ctrl->x_pending = 1;  // x lacks Q_k alpha_k
          stop_test(u.ctrl, tot[0]);
          if (u.hist) u.hist[u.ctrl->iters] = sqrt(tot[0] / u.ctrl->nb2);
        }
        if (u.rr_out) *u.rr_out = tot[0];
      }
    }
  }
}

template <int S>
cudaError_t launch_update_s(const UpdArgs& u, int grid, cudaStream_t st) {
  switch (u.mode) {
    case UM_FIRST: k_update<S, UM_FIRST><<<grid, kThreads, 0, st>>>(u); break;
    case UM_FUSED: k_update<S, UM_FUSED><<<grid, kThreads, 0, st>>>(u); break;
    case UM_XR: k_update<S, UM_XR><<<grid, kThreads, 0, st>>>(u); break;
    case UM_QAQ: k_update<S, UM_QAQ><<<grid, kThreads, 0, st>>>(u); break;
    case UM_R: k_update<S, UM_R><<<grid, kThreads, 0, st>>>(u); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- standalone reduced solve

__global__ void k_fgs_standalone(int s, const double* W, int nrhs, const double* B, int nu,
                                 int solver, double* X, int* status) {
  __shared__ double sh[5 * kMaxS * kMaxS + 2 * kMaxS];
  double* Ws = sh;
  double* Bs = Ws + s * s;
  double* Xs = Bs + s * nrhs;
  double* scr = Xs + s * nrhs;
  for (int e = threadIdx.x; e < s * s; e += blockDim.x) Ws[e] = W[e];
  for (int e = threadIdx.x; e < s * nrhs; e += blockDim.x) Bs[e] = B[e];
  __syncthreads();
  const bool ok = reduced_solve(s, Ws, Bs, nrhs, nu, solver, Xs, scr);
  for (int e = threadIdx.x; e < s * nrhs; e += blockDim.x) X[e] = ok ? Xs[e] : 0.0;
  if (threadIdx.x == 0 && status) *status = ok ? SSTEP_OK : SSTEP_ERR_BREAKDOWN;
}

// ---------------------------------------------------------------- PCG vector kernels

// x += alpha p; r -= alpha Ap; z = M^{-1} r; reductions r^T z and ||r||^2; then the stop
// test and beta = (r^T z)_new / (r^T z)_old in the last CTA.
__global__ void __launch_bounds__(kThreads) k_pcg_update(PcgArgs a) {
  if (a.ctrl->done) return;
  const double al = a.ctrl->pcg_alpha;
  double rz = 0.0, rr = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = a.p[i];
    a.x[i] = fma(al, pi, a.x[i]);
    const double ri = fma(-al, __ldg(a.Ap + i), a.r[i]);
    a.r[i] = ri;
    const double zi = prec_d(a.M, i) * ri;
    rz = fma(ri, zi, rz);
    rr = fma(ri, ri, rr);
  }
  double v[2] = {rz, rr}, tot[2];
  if (grid_sum_last<2>(v, a.partials, &a.ctrl->ticket[TK_PCG2], tot)) {
    if (threadIdx.x == 0) {
      Ctrl* c = a.ctrl;
      stop_test(c, tot[1]);
      if (a.hist) a.hist[c->iters] = sqrt(tot[1] / c->nb2);
      c->pcg_beta = tot[0] / c->rz;
      c->rz = tot[0];
    }
  }
}

// p = M^{-1} r + beta p
__global__ void __launch_bounds__(kThreads) k_pcg_pdir(PcgArgs a) {
  if (a.ctrl->done) return;
  const double be = a.ctrl->pcg_beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x)
    a.p[i] = fma(be, a.p[i], prec_d(a.M, i) * a.r[i]);
}

// z = M^{-1} r; p = z; rz = r^T z  (after the initial residual)
__global__ void __launch_bounds__(kThreads) k_pcg_init(PcgArgs a) {
  if (a.ctrl->done) return;
  double rz = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = a.r[i];
    const double zi = prec_d(a.M, i) * ri;
    a.p[i] = zi;
    rz = fma(ri, zi, rz);
  }
  double v[1] = {rz}, tot[1];
  if (grid_sum_last<1>(v, a.partials, &a.ctrl->ticket[TK_PCG2], tot)) {
    if (threadIdx.x == 0) a.ctrl->rz = tot[0];
  }
}

// ---------------------------------------------------------------- utilities

// U[-1,1) from SplitMix64 (Steele, Lea, Flood 2014): output k mixes seed + (k+1) * golden gamma.
__global__ void k_fill_splitmix(double* v, int64_t n, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    v[i] = splitmix_pm1(seed, i);
  }
}

// CSR sanity: rowptr[0] = 0, rowptr[n] = nnz, rowptr non-decreasing, 0 <= colind < n.
// Every read is clamped to the arrays' extents, so bad input only sets *bad.
__global__ void k_csr_check(CsrOp A, int64_t nnz, int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k0 = A.rowptr[i], k1 = A.rowptr[i + 1];
    if ((i == 0 && k0 != 0) || (i == A.n - 1 && k1 != nnz) || k0 < 0 || k1 < k0 || k1 > nnz) {
      atomicExch(bad, 1);
      continue;
    }
    for (int64_t k = k0; k < k1; ++k) {
      const int32_t c = A.colind[k];
      if (c < 0 || (int64_t)c >= A.n) {
        atomicExch(bad, 1);
        break;
      }
    }
  }
}

__global__ void k_jacobi_csr(CsrOp A, double* dinv, int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    int found = 0;
    for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k)
      if (A.colind[k] == i) { d += A.vals[k]; found = 1; }
    if (!found || !(d > 0.0)) {
      atomicExch(bad, 1);
      dinv[i] = 0.0;
    } else {
      dinv[i] = 1.0 / d;
    }
  }
}

// Per-CTA minimum of the Gershgorin lower bounds of M^{-1}A (host takes the final minimum).
__global__ void k_gershgorin_csr(CsrOp A, int jacobi, double* out) {
  __shared__ double sh[kThreads];
  double lo = 1.0e308;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0, off = 0.0;
    for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
      if (A.colind[k] == i) d += A.vals[k];
      else off += fabs(A.vals[k]);
    }
    const double b = jacobi ? 1.0 - off / d : d - off;
    lo = fmin(lo, b);
  }
  sh[threadIdx.x] = lo;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// ||v||^2 -> ctrl: which = 0 sets the power method's first scale 1/||v0||.
__global__ void __launch_bounds__(kThreads) k_norm2(const double* v, int64_t n, Ctrl* c,
                                                    double* partials, int which) {
  double a = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a = fma(v[i], v[i], a);
  double w[1] = {a}, tot[1];
  if (grid_sum_last<1>(w, partials, &c->ticket[TK_NORM], tot)) {
    if (threadIdx.x == 0) {
      if (which == 0) c->inv_scale = tot[0] > 0.0 ? 1.0 / sqrt(tot[0]) : 0.0;
      else c->sums[0] = tot[0];
    }
  }
}

int stream_ctas(int64_t n, int per_sm) {
  const int64_t want = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sm_count() * per_sm));
}

}  // namespace

// Host-side pair lists of the Gram modes (same layout as the tail reads back).
int gram_pairs(int mode, int s, int full, unsigned short* pairs, int* nl, int* nr) {
  const Layout L{s, full};
  int ne = 0;
  auto sym = [&](int lo, int ro) {  // symmetric block: L[lo+i] . R[ro+j]
    if (full) {
      for (int j = 0; j < s; ++j)
        for (int i = 0; i < s; ++i) pairs[ne++] = (unsigned short)(((lo + i) << 8) | (ro + j));
    } else {
      for (int j = 0; j < s; ++j)
        for (int i = 0; i <= j; ++i) pairs[ne++] = (unsigned short)(((lo + i) << 8) | (ro + j));
    }
  };
  auto gen = [&](int lo, int ro) {
    for (int j = 0; j < s; ++j)
      for (int i = 0; i < s; ++i) pairs[ne++] = (unsigned short)(((lo + i) << 8) | (ro + j));
  };
  auto vec = [&](int lo, int rcol) {
    for (int i = 0; i < s; ++i) pairs[ne++] = (unsigned short)(((lo + i) << 8) | rcol);
  };
  (void)L;
  switch (mode) {
    case GM_ONESYNC_FIRST:  // L = Z, R = [AZ, r]
    case GM_LITERAL_W:      // L = Q, R = [AQ, r]
      *nl = s;
      *nr = s + 1;
      sym(0, 0);
      vec(0, s);
      break;
    case GM_LITERAL_B2:  // L = Q, R = AZ
      *nl = s;
      *nr = s;
      gen(0, 0);
      break;
    case GM_ONESYNC:  // L = [Q, Z], R = [AQ, AZ, r]
      *nl = 2 * s;
      *nr = 2 * s + 1;
      sym(0, 0);        // G1 = Q^T AQ
      gen(0, s);        // G2 = Q^T AZ
      if (full) gen(s, 0);  // G3 = Z^T AQ
      sym(s, s);        // G4 = Z^T AZ
      vec(0, 2 * s);    // g5 = Q^T r
      vec(s, 2 * s);    // g6 = Z^T r
      break;
    default:
      return -1;
  }
  return ne;
}

int gram_ctas() { return sm_count() * 2; }

cudaError_t launch_gram(const GramArgs& g, cudaStream_t st) {
  if (g.ne < 1 || g.ne > kMaxEntries || g.nl < 1 || g.nr < 1 || g.nl + g.nr > 2 * kMaxGramVecs)
    return cudaErrorInvalidValue;
  // Choose entries-per-thread so that (chunks x row phases x EPT) covers ne with few idle slots.
  int best_ept = 1, best_nch = g.ne, best_rp = std::max(1, kThreads / g.ne);
  double best = -1.0;
  for (int ept = 1; ept <= 8; ++ept) {
    const int nch = (g.ne + ept - 1) / ept;
    if (nch > kThreads) continue;
    const int rp = kThreads / nch;
    const double eff = (double)g.ne * rp / ((double)kThreads * ept);
    if (eff > best + 1e-9) {
      best = eff;
      best_ept = ept;
      best_nch = nch;
      best_rp = rp;
    }
  }
  if (best < 0.0) return cudaErrorInvalidValue;
  const int ncols = g.nl + g.nr;
  size_t smem = sizeof(double) * (size_t)ncols * (kGramRows + 1);
  const size_t red = sizeof(double) * ((size_t)best_rp * g.ne + (size_t)kThreads + (size_t)g.ne +
                                       12 * kMaxS * kMaxS);
  smem = std::max(smem, red);
  const int grid = gram_ctas();
  switch (best_ept) {
#define CASE(E) \
  case E: k_gram<E><<<grid, kThreads, smem, st>>>(g, best_nch, best_rp); break;
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

namespace {

template <int NR, int NC>
cudaError_t launch_tiled_shape(const GramTiles& g, cudaStream_t st) {
  static int occ = 0;
  if (!occ) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_tiled<NR, NC>, kThreads, 0);
    if (occ < 1) occ = 1;
  }
  const int64_t want = ((int64_t)sm_count() * occ + g.ntiles - 1) / g.ntiles;
  const int64_t rows = (g.n + kThreads - 1) / kThreads;
  const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(want, rows));
  k_gram_tiled<NR, NC><<<dim3(gx, g.ntiles), kThreads, 0, st>>>(g);
  return cudaGetLastError();
}

template <int NR>
cudaError_t launch_tiled_nr(const GramTiles& g, int nc, cudaStream_t st) {
  if (nc == NR) return launch_tiled_shape<NR, NR>(g, st);
  if (nc == NR + 1) return launch_tiled_shape<NR, NR + 1>(g, st);
  if constexpr (NR <= 4) {  // the two-tile one-reduction layout is used up to s = 4
    if (nc == 2 * NR + 1) return launch_tiled_shape<NR, 2 * NR + 1>(g, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace

cudaError_t launch_gram_tiled(int mode, int s, int64_t n, int64_t ld, const double* Q,
                              const double* AQ, const double* Z, const double* AZ, const double* r,
                              Ctrl* ctrl, double* partials, cudaStream_t st) {
  if (s < 1 || s > kTileMaxR) return cudaErrorNotSupported;
  GramTiles g{};
  g.n = n;
  g.mode = mode;
  g.ctrl = ctrl;
  g.partials = partials;
  for (auto& tt : g.out)
    for (auto& o : tt) o = -1;
  const int s2 = s * s;
  auto col = [&](const double* base, int j) { return base + (int64_t)j * ld; };
  int nc = 0;
  if (mode == GM_ONESYNC_FIRST || mode == GM_LITERAL_W) {
    // W = V^T AV (entry i + j s), b1 = V^T r (entry s^2 + i); V = Z or Q
    const double* V = mode == GM_ONESYNC_FIRST ? Z : Q;
    const double* AV = mode == GM_ONESYNC_FIRST ? AZ : AQ;
    g.ntiles = 1;
    nc = s + 1;
    for (int i = 0; i < s; ++i) g.x[0][i] = col(V, i);
    for (int j = 0; j < s; ++j) g.y[0][j] = col(AV, j);
    g.y[0][s] = r;
    for (int i = 0; i < s; ++i) {
      for (int j = 0; j < s; ++j) g.out[0][i * nc + j] = (short)(i + j * s);
      g.out[0][i * nc + s] = (short)(s2 + i);
    }
    g.ne = s2 + s;
  } else if (mode == GM_LITERAL_B2) {
    g.ntiles = 1;  // Q^T AZ, entry i + j s
    nc = s;
    for (int i = 0; i < s; ++i) g.x[0][i] = col(Q, i);
    for (int j = 0; j < s; ++j) g.y[0][j] = col(AZ, j);
    for (int i = 0; i < s; ++i)
      for (int j = 0; j < s; ++j) g.out[0][i * nc + j] = (short)(i + j * s);
    g.ne = s2;
  } else if (mode == GM_ONESYNC) {
    // Entries (every block formed): G1 = Q^T AQ, G2 = Q^T AZ, G3 = Z^T AQ, G4 = Z^T AZ
    // (each i + j s after its base), g5 = Q^T r, g6 = Z^T r.
    const int b1 = 0, b2 = s2, b3 = 2 * s2, b4 = 3 * s2, b5 = 4 * s2, b6 = 4 * s2 + s;
    g.ne = 4 * s2 + 2 * s;
    if (2 * s + 1 <= kTileMaxC && s <= 4) {
      // two tiles: Q^T [AQ AZ r] and Z^T [AQ AZ r]
      g.ntiles = 2;
      nc = 2 * s + 1;
      for (int t = 0; t < 2; ++t) {
        const double* X = t == 0 ? Q : Z;
        for (int i = 0; i < s; ++i) g.x[t][i] = col(X, i);
        for (int j = 0; j < s; ++j) {
          g.y[t][j] = col(AQ, j);
          g.y[t][s + j] = col(AZ, j);
        }
        g.y[t][2 * s] = r;
        for (int i = 0; i < s; ++i) {
          for (int j = 0; j < s; ++j) {
            g.out[t][i * nc + j] = (short)((t == 0 ? b1 : b3) + i + j * s);
            g.out[t][i * nc + s + j] = (short)((t == 0 ? b2 : b4) + i + j * s);
          }
          g.out[t][i * nc + 2 * s] = (short)((t == 0 ? b5 : b6) + i);
        }
      }
    } else {
      // four tiles: {Q, Z}^T [AQ r] and {Q, Z}^T [AZ r]; r kept once per X
      g.ntiles = 4;
      nc = s + 1;
      for (int t = 0; t < 4; ++t) {
        const double* X = t < 2 ? Q : Z;
        const double* Y = (t & 1) ? AZ : AQ;
        const int base = t == 0 ? b1 : t == 1 ? b2 : t == 2 ? b3 : b4;
        for (int i = 0; i < s; ++i) g.x[t][i] = col(X, i);
        for (int j = 0; j < s; ++j) g.y[t][j] = col(Y, j);
        g.y[t][s] = r;
        for (int i = 0; i < s; ++i) {
          for (int j = 0; j < s; ++j) g.out[t][i * nc + j] = (short)(base + i + j * s);
          if (t == 0) g.out[t][i * nc + s] = (short)(b5 + i);
          if (t == 2) g.out[t][i * nc + s] = (short)(b6 + i);
        }
      }
    }
  } else {
    return cudaErrorNotSupported;
  }
  switch (s) {
    case 1: return launch_tiled_nr<1>(g, nc, st);
    case 2: return launch_tiled_nr<2>(g, nc, st);
    case 3: return launch_tiled_nr<3>(g, nc, st);
    case 4: return launch_tiled_nr<4>(g, nc, st);
    case 5: return launch_tiled_nr<5>(g, nc, st);
    case 6: return launch_tiled_nr<6>(g, nc, st);
    case 7: return launch_tiled_nr<7>(g, nc, st);
    case 8: return launch_tiled_nr<8>(g, nc, st);
    default: return cudaErrorNotSupported;
  }
}

namespace {
template <int S, bool FIRST>
cudaError_t launch_upd_gram_s(const UpdGramArgs& a, cudaStream_t st) {
  static int occ = 0;
  if (!occ) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_upd_gram<S, FIRST>, kThreads, 0);
    if (occ < 1) occ = 1;
  }
  const int64_t rows = (a.n + kThreads - 1) / kThreads;
  const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * occ, rows));
  k_upd_gram<S, FIRST><<<gx, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_upd_gram(const UpdGramArgs& a, int s, bool first, cudaStream_t st) {
  switch (s) {
#define CASE(S) \
  case S: return first ? launch_upd_gram_s<S, true>(a, st) : launch_upd_gram_s<S, false>(a, st);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: return cudaErrorNotSupported;
  }
}

namespace {
template <typename KernelT>
int occ_grid(KernelT k, int64_t n, int& cache) {
  if (!cache) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cache, k, kThreads, 0);
    if (cache < 1) cache = 1;
  }
  const int64_t rows = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * cache, rows));
}
}  // namespace

namespace {

template <int NR, int NC>
cudaError_t launch_gram_df_shape(const GramTilesF& g, cudaStream_t st) {
  static int occ = 0;
  if (!occ) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gram_df<NR, NC>, kThreads, 0);
    if (occ < 1) occ = 1;
  }
  const int64_t want = ((int64_t)sm_count() * occ + g.ntiles - 1) / g.ntiles;
  const int64_t rows = (g.n + kThreads - 1) / kThreads;
  const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(want, rows));
  k_gram_df<NR, NC><<<dim3(gx, g.ntiles), kThreads, 0, st>>>(g);
  return cudaGetLastError();
}

// 2 x 2 tiles of X^T [Y | r]: X = s FP32 columns, Y = s FP32 columns (entries i + j s),
// r = rhi + rlo (entries s^2 + i, kept from the tiles of the first column half), as the
// literal-form layouts expect.  Padding rows/columns point at column 0 and are not kept.
cudaError_t launch_gram_df_split(int mode, const MixedArgs& a, int s, const float* X,
                                 const float* Y, bool with_r, cudaStream_t st) {
  GramTilesF g{};
  g.n = a.n;
  g.mode = mode;
  g.ctrl = a.ctrl;
  g.partials = a.partials;
  g.ntiles = 4;
  const int h = (s + 1) / 2;
  const int nr = h, nc = h + (with_r ? 1 : 0);
  g.ne = s * s + (with_r ? s : 0);
  for (auto& tt : g.out)
    for (auto& o : tt) o = -1;
  for (int t = 0; t < 4; ++t) {
    const int i0 = (t >> 1) * h, j0 = (t & 1) * h;
    for (int ri = 0; ri < nr; ++ri) {
      const int i = i0 + ri;
      g.x[t][ri] = X + (int64_t)(i < s ? i : 0) * a.ld;
    }
    for (int c = 0; c < h; ++c) {
      const int j = j0 + c;
      g.y[t][c] = Y + (int64_t)(j < s ? j : 0) * a.ld;
      for (int ri = 0; ri < nr; ++ri) {
        const int i = i0 + ri;
        if (i < s && j < s) g.out[t][ri * nc + c] = (short)(i + j * s);
      }
    }
    if (with_r) {
      g.y[t][h] = a.rhi;
      g.ylo[t][h] = a.rlo;
      if (j0 == 0)
        for (int ri = 0; ri < nr; ++ri) {
          const int i = i0 + ri;
          if (i < s) g.out[t][ri * nc + h] = (short)(s * s + i);
        }
    }
  }
  switch (nr * 16 + nc) {
    case 3 * 16 + 3: return launch_gram_df_shape<3, 3>(g, st);
    case 3 * 16 + 4: return launch_gram_df_shape<3, 4>(g, st);
    case 4 * 16 + 4: return launch_gram_df_shape<4, 4>(g, st);
    case 4 * 16 + 5: return launch_gram_df_shape<4, 5>(g, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

cudaError_t launch_gram_b2_f32(const MixedArgs& a, int s, cudaStream_t st) {
  if (s > 4) return launch_gram_df_split(GM_LITERAL_B2, a, s, a.Q, a.AZ, false, st);
  switch (s) {
#define CASE(S)                                                            \
  case S: {                                                                \
    static int occ = 0;                                                    \
    k_gram_b2f<S><<<occ_grid(k_gram_b2f<S>, a.n, occ), kThreads, 0, st>>>(a); \
    return cudaGetLastError();                                             \
  }
    CASE(1) CASE(2) CASE(3) CASE(4)
#undef CASE
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_upd_gram_f32(const MixedArgs& a, int s, bool first, cudaStream_t st) {
  const char* tp = std::getenv("SSTEP_FP32_UPD_TWO_PASS");  // read per launch (a test switch)
  const bool two_pass = tp && tp[0] == '1';
  if (s > 4 && !two_pass) {  // one pass, two points per thread (k_upd_gramwf)
    switch (s) {
#define CASE(S)                                                                               \
  case S:                                                                                     \
    if (first) {                                                                              \
      static int occ = 0;                                                                     \
      k_upd_gramwf<S, true><<<occ_grid(k_upd_gramwf<S, true>, a.n, occ), kThreads, 0, st>>>(a); \
    } else {                                                                                  \
      static int occ = 0;                                                                     \
      k_upd_gramwf<S, false><<<occ_grid(k_upd_gramwf<S, false>, a.n, occ), kThreads, 0, st>>>(a); \
    }                                                                                         \
    return cudaGetLastError();
      CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
      default: return cudaErrorNotSupported;
    }
  }
  if (s > 4) {  // Q, AQ update and W, b1 as two passes (SSTEP_FP32_UPD_TWO_PASS=1)
    const int grid = update_ctas(a.n);
    switch (s) {
#define CASE(S)                                                                   \
  case S:                                                                         \
    if (first) k_upd_qaq_f<S, true><<<grid, kThreads, 0, st>>>(a);                \
    else k_upd_qaq_f<S, false><<<grid, kThreads, 0, st>>>(a);                     \
    break;
      CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
      default: return cudaErrorNotSupported;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_gram_df_split(GM_LITERAL_W, a, s, a.Q, a.AQ, true, st);
  }
  switch (s) {
#define CASE(S)                                                                            \
  case S: {                                                                                \
    if (first) {                                                                           \
      static int occ = 0;                                                                  \
      k_upd_gramf<S, true><<<occ_grid(k_upd_gramf<S, true>, a.n, occ), kThreads, 0, st>>>(a); \
    } else {                                                                               \
      static int occ = 0;                                                                  \
      k_upd_gramf<S, false><<<occ_grid(k_upd_gramf<S, false>, a.n, occ), kThreads, 0, st>>>(a); \
    }                                                                                      \
    return cudaGetLastError();                                                             \
  }
    CASE(1) CASE(2) CASE(3) CASE(4)
#undef CASE
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_update_xr_f32(const MixedArgs& a, int s, cudaStream_t st) {
  // one full wave of resident CTAs (as many as the registers allow, up to 2048 threads per SM:
  // latency-bound otherwise); the grid-stride loop spreads the points evenly over them
  switch (s) {
#define CASE(S)                                                                      \
  case S: {                                                                          \
    static int occ = 0;                                                              \
    k_update_xrf<S><<<occ_grid(k_update_xrf<S>, a.n / 4, occ), kThreads, 0, st>>>(a); \
    return cudaGetLastError();                                                       \
  }
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    default: return cudaErrorNotSupported;
  }
}

namespace {
// dL/dA_ij = -lambda_i x_j on the stored pattern (row-per-thread over the CSR rows).
__global__ void k_pattern_grad(CsrOp A, const double* lam, const double* x, double* g,
                               double scale, int accumulate) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double li = -scale * __ldg(lam + i);
    for (int64_t k = __ldg(A.rowptr + i); k < __ldg(A.rowptr + i + 1); ++k) {
      const double v = li * __ldg(x + __ldg(A.colind + k));
      g[k] = accumulate ? g[k] + v : v;
    }
  }
}
}  // namespace

cudaError_t launch_pattern_grad(const CsrOp& A, const double* lam, const double* x, double* g,
                                double scale, int accumulate, cudaStream_t st) {
  k_pattern_grad<<<stream_ctas(A.n, 8), kThreads, 0, st>>>(A, lam, x, g, scale, accumulate);
  return cudaGetLastError();
}

namespace {
__global__ void k_d2f(const double* a, float* b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __double2float_rn(a[i]);
}
}  // namespace

cudaError_t launch_d2f(const double* a, float* b, int64_t n, cudaStream_t st) {
  k_d2f<<<stream_ctas(n, 4), kThreads, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

namespace {
// x += Q alpha when the step is pending (the products in increasing j from 0, the order of the
// x update it replaces); the last CTA clears the flag every CTA read at entry.
__global__ void __launch_bounds__(kThreads) k_flush_x(double* x, const double* Q, int64_t n,
                                                     int64_t ld, int s, Ctrl* ctrl) {
  __shared__ double sa[kMaxS];
  __shared__ int pend;
  if (threadIdx.x == 0) pend = ctrl->x_pending;
  if (threadIdx.x < s) sa[threadIdx.x] = ctrl->alpha[threadIdx.x];
  __syncthreads();
  if (pend) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
      double dx = 0.0;
      for (int j = 0; j < s; ++j) dx = fma(Q[j * ld + i], sa[j], dx);
      x[i] += dx;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctrl->ticket[TK_UPDATE], 1u) == gridDim.x - 1) {
      ctrl->x_pending = 0;
      ctrl->ticket[TK_UPDATE] = 0u;
    }
  }
}
}  // namespace

cudaError_t launch_flush_x(double* x, const double* Q, int64_t n, int64_t ld, int s, Ctrl* ctrl,
                           cudaStream_t st) {
  if (s < 1 || s > kMaxS || !ctrl) return cudaErrorInvalidValue;
  k_flush_x<<<stream_ctas(n, 4), kThreads, 0, st>>>(x, Q, n, ld, s, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_fold_x(double* x64, float* xhi, float* xlo, int64_t n, Ctrl* ctrl,
                          const float* Q, int64_t ld, int s, cudaStream_t st) {
  if (Q && (s < 1 || s > kOpMaxS)) return cudaErrorInvalidValue;
  k_fold_x<<<stream_ctas(n, 4), kThreads, 0, st>>>(x64, xhi, xlo, n, ctrl, Q, ld, s);
  return cudaGetLastError();
}

// Raises k_gram's dynamic shared-memory limit on the current device (a per-device function
// attribute), once per device ordinal.
cudaError_t gram_init() {
  constexpr int kDevs = 64;
  static int done_dev[kDevs] = {};
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  int* done = (dev >= 0 && dev < kDevs) ? &done_dev[dev] : nullptr;
  if (done && *done) return cudaSuccess;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (optin <= 0) optin = 48 * 1024;
  cudaError_t e = cudaSuccess;
  // The dynamic limit plus the kernel's static shared memory may not exceed the opt-in size.
#define SET(E)                                                                              \
  if (e == cudaSuccess) {                                                                   \
    cudaFuncAttributes fa{};                                                                \
    e = cudaFuncGetAttributes(&fa, k_gram<E>);                                              \
    if (e == cudaSuccess)                                                                   \
      e = cudaFuncSetAttribute(k_gram<E>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                               optin - (int)fa.sharedSizeBytes);                            \
  }
  SET(1) SET(2) SET(3) SET(4) SET(5) SET(6) SET(7) SET(8)
#undef SET
  if (e == cudaSuccess && done) *done = 1;
  return e;
}

int update_ctas(int64_t n) { return stream_ctas(n, 4); }

cudaError_t launch_update(const UpdArgs& u, cudaStream_t st) {
  const int grid = update_ctas(u.n);
  switch (u.s) {
#define CASE(S) \
  case S: return launch_update_s<S>(u, grid, st);
    CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
    CASE(9) CASE(10) CASE(11) CASE(12) CASE(13) CASE(14) CASE(15) CASE(16)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fgs_standalone(int s, const double* W, int nrhs, const double* B, int nu,
                                  int solver, double* X, int* status_dev, cudaStream_t st) {
  k_fgs_standalone<<<1, 128, 0, st>>>(s, W, nrhs, B, nu, solver, X, status_dev);
  return cudaGetLastError();
}

int pcg_ctas(int64_t n) { return stream_ctas(n, 8); }

cudaError_t launch_pcg_update(const PcgArgs& a, cudaStream_t st) {
  static int occ = 0;  // one full wave of resident CTAs
  k_pcg_update<<<occ_grid(k_pcg_update, a.n, occ), kThreads, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_pcg_pdir(const PcgArgs& a, cudaStream_t st) {
  k_pcg_pdir<<<pcg_ctas(a.n), kThreads, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_pcg_init(const PcgArgs& a, cudaStream_t st) {
  k_pcg_init<<<pcg_ctas(a.n), kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fill_splitmix(double* v, int64_t n, uint64_t seed, cudaStream_t st) {
  k_fill_splitmix<<<stream_ctas(n, 4), kThreads, 0, st>>>(v, n, seed);
  return cudaGetLastError();
}
cudaError_t launch_csr_check(const CsrOp& A, int64_t nnz, int* bad, cudaStream_t st) {
  k_csr_check<<<stream_ctas(A.n, 4), kThreads, 0, st>>>(A, nnz, bad);
  return cudaGetLastError();
}
cudaError_t launch_jacobi_csr(const CsrOp& A, double* dinv, int* bad, cudaStream_t st) {
  k_jacobi_csr<<<stream_ctas(A.n, 4), kThreads, 0, st>>>(A, dinv, bad);
  return cudaGetLastError();
}
cudaError_t launch_norm2(const double* v, int64_t n, Ctrl* c, double* partials, int which,
                         cudaStream_t st) {
  k_norm2<<<stream_ctas(n, 4), kThreads, 0, st>>>(v, n, c, partials, which);
  return cudaGetLastError();
}
int gershgorin_ctas(int64_t n) { return stream_ctas(n, 4); }
cudaError_t launch_gershgorin_csr(const CsrOp& A, int jacobi, double* out_min, cudaStream_t st) {
  k_gershgorin_csr<<<gershgorin_ctas(A.n), kThreads, 0, st>>>(A, jacobi, out_min);
  return cudaGetLastError();
}

}  // namespace sstep
