/*
 * sstep.h -- C ABI of libsstep.so: Chebyshev-basis s-step preconditioned conjugate gradient
 * (PCG-S) with Forward Gauss-Seidel (FGS) Gram solves, and classical PCG, on one NVIDIA GB300
 * (sm_103a).  Method: D'Ambra, Bernaschi, Carrozzo, Thomas, "Scalable s-step Preconditioned
 * Conjugate Gradient with Chebyshev Basis and Gauss-Seidel Gram Solve" (arXiv 2603.09790).
 *
 * General conventions
 *  - All floating point is IEEE binary64 unless a name says otherwise.
 *  - Vectors are dense arrays of n doubles.  Blocks of k vectors are column-major with leading
 *    dimension ld >= n (column j starts at base + j*ld).
 *  - "device pointer" means memory the GPU can address (cudaMalloc / torch CUDA tensors).
 *    Entry points marked "device or host" accept either; host memory is staged through the
 *    library's own device buffers, with the copies ordered on the handle's stream.
 *  - Every entry point returns an sstep_status and never aborts, throws or traps.  A
 *    description of the last failure on the calling thread is returned by sstep_last_error().
 *  - Work is ordered on the CUDA stream given at set-up (passed as void*).  NULL: a private
 *    blocking stream of the handle, which is ordered with the caller's work on the legacy
 *    default stream (a capturable stand-in for it).  sstep_solve* return after the solve has
 *    finished on that stream.
 *  - Not thread-safe per handle: one handle must not be used from two threads at once.
 */
#ifndef SSTEP_H
#define SSTEP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SSTEP_API __attribute__((visibility("default")))
#else
#define SSTEP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sstep_ctx* sstep_handle; /* opaque, owned by the library */

typedef enum {
  SSTEP_OK = 0,
  SSTEP_NOT_CONVERGED = 1,  /* max_outer reached; x and info are still filled */
  SSTEP_ERR_INVALID = 2,    /* bad argument or descriptor */
  SSTEP_ERR_BREAKDOWN = 3,  /* Gram diagonal <= 0 or non-finite (W_ii, pAp) */
  SSTEP_ERR_NONFINITE = 4,  /* non-finite residual norm */
  SSTEP_ERR_CUDA = 5,       /* a CUDA runtime call failed */
  SSTEP_ERR_OOM = 6,        /* device allocation failed */
  SSTEP_ERR_UNSUPPORTED = 7, /* valid request that the library does not implement */
  SSTEP_ERR_TIMEOUT = 8      /* a bounded device-side wait (a copy that never arrived) ran out;
                                the solve stopped, the CUDA context stays usable */
} sstep_status;

/* ------------------------------------------------------------------ operator A */
enum { SSTEP_MATRIX_CSR = 0, SSTEP_MATRIX_STENCIL = 1, SSTEP_MATRIX_Q1 = 2 };

/* The SPD matrix A of Ax = b (Section 1).
 * CSR: n rows, rowptr[n+1] (int64), colind[nnz] (int32, 0-based), vals[nnz]; device or host
 *      pointers; copied into library-owned device memory at set-up (the caller may free them
 *      afterwards).  Each row must hold its diagonal entry when the Jacobi preconditioner is used.
 * STENCIL: matrix-free finite-difference operator on the interior points of an nx*ny*nz grid
 *      (row index i + nx*(j + ny*k); Dirichlet neighbours dropped).  points = 5 (2D, nz = 1),
 *      7 or 27 (3D).  weights: NULL for the Poisson weights (diagonal 4 / 6 / 26, neighbours -1),
 *      or `points` host doubles in the order of increasing linear offset (for 7 points:
 *      -z, -y, -x, centre, +x, +y, +z; for 27: dz-major, then dy, then dx).  In the
 *      FP32-basis form a 7-point grid with nx a multiple of 4 (nx >= 72, ny >= 18) has its MPK
 *      steps and its PCG product fed by tensor-memory-accelerator copies;
 *      SSTEP_STENCIL_TMA=0 in the environment at set-up selects plain loads (the same MPK
 *      results bit for bit; p^T A p summed over another grid).
 * Q1: matrix-free trilinear (Q1) finite-element diffusion operator (a variable-coefficient
 *      SPD matrix; the method takes any SPD A, Section 1): the nx*ny*nz interior vertices
 *      (row index i + nx*(j + ny*k)) of a grid of (nx+1)*(ny+1)*(nz+1) unit cells, Dirichlet boundary vertices eliminated.  weights: the
 *      per-cell conductivities kappa, (nx+1)*(ny+1)*(nz+1) doubles, cell cx + (nx+1)*(cy +
 *      (ny+1)*cz) (device or host pointer; copied at set-up).  Every kappa must be finite and
 *      positive (else SSTEP_ERR_INVALID).  Entries: a_ii = (1/3) sum of the 8 kappa around
 *      vertex i; -(1/12) times the sum of the kappa of the cells shared with a neighbour two or
 *      three offsets of +-1 away; 0 for the six axis neighbours (21 entries per interior row).
 *      The same matrix as assembling the Q1 element stiffness kappa_e (K1 x M1 x M1 + M1 x K1 x
 *      M1 + M1 x M1 x K1), K1 = [[1,-1],[-1,1]], M1 = [[1/3,1/6],[1/6,1/3]], over the cells.
 *      The library keeps a copy of kappa plus 13*n doubles of vertex coefficients (FP64
 *      kernels) and, in the FP32-basis form, an FP32 copy of kappa.
 *      points is ignored; n may be 0 or nx*ny*nz.  Preconditioners NONE and JACOBI; the
 *      FP64 and FP32-basis s-step forms and PCG.  In the FP32-basis form with nx a multiple
 *      of 4 (nx >= 72, ny >= 10) the middle MPK steps are fed by tensor-memory-accelerator
 *      copies; SSTEP_Q1_TMA=0 in the environment at set-up selects plain loads (same results
 *      bit for bit). */
typedef struct {
  int kind;
  int64_t n;
  const int64_t* rowptr;
  const int32_t* colind;
  const double* vals;
  int64_t nnz;
  int nx, ny, nz, points;
  const double* weights;
} sstep_matrix;

/* ------------------------------------------------------------------ preconditioner M */
/* The paper treats M^{-1} as a black box (Section 4): NONE is M = I (the CG-S runs of
 * Section 6.1), JACOBI is M = diag(A).  AMG (CSR operators, FP64 s-step forms) is one V-cycle
 * of this library's aggregation AMG; the paper's own AMG is external (Section 5), so the
 * library defines it: coupling w_ij = -a_ij / sqrt(a_ii a_jj); greedy pairwise matching of the
 * rows in increasing order (largest w_ij > 0, ties to the lower index), applied twice per
 * level; unsmoothed piecewise-constant prolongation P; Galerkin A_c = P^T A P summed in a fixed
 * order (reproducible bit for bit); one l1-Jacobi sweep (D = diag(sum_j |a_ij|)) before and
 * after the coarse correction; a dense solve (from the Cholesky factor, set up on the host)
 * once n <= amg_coarse_max.  The V-cycle is symmetric positive definite.  Set-up runs on the
 * host; every application runs on the device. */
enum { SSTEP_PREC_NONE = 0, SSTEP_PREC_JACOBI = 1, SSTEP_PREC_AMG = 2 };
typedef struct {
  int kind;
  int amg_coarse_max;  /* AMG: largest directly solved level, 1..4096 (0: 512) */
  int amg_max_levels;  /* AMG: at most this many levels, 1..32 (0: 25) */
} sstep_precond;

/* ------------------------------------------------------------------ options */
enum {
  SSTEP_ALGO_ONESYNC = 0, /* Algorithm 1 with the Gram blocks of [Q_k, Z_{k+1}] formed in one
                             reduction per outer iteration (W_{k+1} assembled from them and beta) */
  SSTEP_ALGO_LITERAL = 1, /* Algorithm 1 as printed: W = Q^T AQ, b1 = Q^T r formed from the updated
                             blocks (direction update and step system fused in one pass), b2 after the MPK.
                             Fewer FP64 products than the one-reduction form (2s^2 + s against
                             4s^2 + 2s per outer iteration); the default */
  SSTEP_ALGO_PCG = 2      /* classical preconditioned CG (Hestenes-Stiefel), the comparator */
};
/* Reduced solves.  FGS: nu forward Gauss-Seidel sweeps from 0 (Section 3.1, Eq. fgs-iteration).
 * FGS_OPERATOR: the same nu sweeps applied as one s x s matrix, x = P_nu b with
 * P_nu = (I + M + ... + M^{nu-1}) (D + L)^{-1}, M = I - (D + L)^{-1} W, formed by repeated
 * doubling in O(log nu) small products (s <= 8); equal to FGS in exact arithmetic, different
 * in rounding; formed once per W_k and applied to both systems that share it (alpha_k,
 * beta_k).  The FP32-basis path uses it whenever FGS is asked for.
 * CHOLESKY: exact solves (Section 3.3). */
enum { SSTEP_GRAM_FGS = 0, SSTEP_GRAM_CHOLESKY = 1, SSTEP_GRAM_FGS_OPERATOR = 2 };

typedef struct {
  int s;              /* step size, 1 <= s <= 16 (Algorithm 1 "step size s") */
  int sweeps;         /* nu, FGS sweeps per reduced solve (Algorithm 1 "number of FGS sweeps") */
  double rtol;        /* tau: stop when ||r|| <= tau ||b|| (Algorithm 1's stop test) */
  int max_outer;      /* k_max (outer iterations; PCG: iterations) */
  int algo;           /* SSTEP_ALGO_* */
  int gram_solver;    /* SSTEP_GRAM_FGS (default), SSTEP_GRAM_FGS_OPERATOR or SSTEP_GRAM_CHOLESKY */
  int power_iters;    /* power-method cap (Section 2: 50) */
  double power_tol;   /* power-method relative-change stop (Section 2: 1e-3); <= 0 runs power_iters */
  double lambda_min;  /* lower end of the Chebyshev interval (Section 2 uses 0); < 0 = Gershgorin bound */
  double lambda_max;  /* > 0: used as given; otherwise estimated by the power method at set-up */
  const double* power_v0; /* start vector of the power method (n doubles, device or host); NULL =
                             U[-1,1) from SplitMix64 with seed 1 in index order */
  int check_every;    /* outer iterations between host reads of the stop flag (0 = automatic) */
  int gram_blocks;    /* SSTEP_GRAM_BLOCKS_FULL: every Gram block as computed (Algorithm 1);
                         SSTEP_GRAM_BLOCKS_SYM: upper triangles of Q^T AQ, Z^T AZ and
                         Z^T AQ = (Q^T AZ)^T (fewer products).  Cholesky always uses FULL. */
  int precision;      /* SSTEP_PRECISION_FP64 (default), or SSTEP_PRECISION_FP32_RR: the basis
                         Z, AZ, Q, AQ and the MPK SpMV in FP32; Gram sums, x and r increments in
                         double-float on the FP32 pipe (TwoProd/TwoSum, ~48-bit); FGS in FP64;
                         every rr_period outer iterations x is folded and r = b - A x is
                         recomputed in FP64 (residual replacement).  Literal form, s <= 8. */
  int rr_period;      /* outer iterations between residual replacements (<= 0: s) */
  /* Batched persistent solver (implied when nsys > 1; see sstep_setup).  s = 0 lets the
   * autotuner pick s from {2, 4, 8}; cluster = 0 / block_threads = 0 let it pick the CTAs per
   * thread-block cluster (one cluster works on one system and right-hand side at a time) from
   * {2, 4, 8, 16} and the threads per CTA from {256, 512}. */
  int persistent;     /* 1: use the batched persistent solver even for nsys = 1 */
  int cluster;        /* CTAs per cluster: 0 (autotune), 1, 2, 4, 8 or 16 */
  int block_threads;  /* threads per CTA: 0 (autotune), 256 or 512 (512 only for s <= 4) */
} sstep_opts;
enum { SSTEP_PRECISION_FP64 = 0, SSTEP_PRECISION_FP32_RR = 1 };
enum { SSTEP_GRAM_BLOCKS_FULL = 0, SSTEP_GRAM_BLOCKS_SYM = 1 };

typedef struct {
  int status;             /* sstep_status of the solve */
  int outer_iters;        /* executed x/r updates (outer iterations; PCG: iterations) */
  int inner_equiv;        /* outer_iters * s (PCG: iterations) */
  double relres;          /* ||r|| / ||b|| of the recursively updated residual at exit */
  double relres_true;     /* ||b - A x|| / ||b|| at exit */
  double lambda_max;      /* lambda_max used for the Chebyshev basis */
  double lambda_min;      /* lambda_min used */
  double ms_setup;        /* wall time of sstep_setup (operator copy, Jacobi, power method) */
  double ms_solve;        /* wall time of the solve, host-to-host */
  long long launches;     /* kernels launched by the solve (graph replays count every node,
                             including launches after convergence that return at entry) */
} sstep_info;

/* Fill *o with the defaults: s = 4, sweeps = 2, rtol = 1e-8, max_outer = 10000, literal form,
 * FGS, power_iters = 50, power_tol = 1e-3, lambda_min = 0, lambda_max = 0 (estimate). */
SSTEP_API void sstep_default_opts(sstep_opts* o);

/* Build a solver for A (Section 2: "estimate lambda_max once, before starting"): copies A to the
 * device, forms M^{-1}, runs the power method on M^{-1}A when o->lambda_max <= 0, derives the
 * Chebyshev scalars c_alpha = 2/(lmax-lmin), c_sigma = (lmax+lmin)/(lmax-lmin), c_gamma = 1, and
 * allocates the basis blocks Z, AZ, Q, AQ (4 s vectors) and x, r, b buffers.
 * nsys = 1 (and persistent = 0): one operator A[0], any kind.
 * nsys > 1 (or persistent = 1): the batched persistent solver for the nsys systems A[0..nsys-1],
 * each a 7-point STENCIL with constant weights whose six neighbour weights are equal (NULL:
 * Poisson), with M = NONE or JACOBI, the literal form, FGS, precision FP64 or FP32_RR and
 * s in {2, 4, 8} (0: autotuned).  Each system gets its own power-method lambda_max (unless
 * o->lambda_max > 0 is given for all) and its Gershgorin lambda_min when o->lambda_min < 0.
 * The paper solves one system at a time; batching is this library's extension.
 * stream: cudaStream_t passed as void*.  On error *out is NULL. */
SSTEP_API sstep_status sstep_setup(const sstep_matrix* A, int nsys, const sstep_precond* M,
                         const sstep_opts* o, void* stream, sstep_handle* out);

/* Solve A x = b (Algorithm 1, or classical PCG when algo = SSTEP_ALGO_PCG).
 * b: n doubles (device or host).  x: n doubles (device or host), x^(0) on entry, solution on
 * exit.  b = 0 gives x = 0 with 0 iterations; ||r^(0)|| <= tau ||b|| gives 0 iterations.
 * info may be NULL.  Returns the solve status (also in info->status). */
SSTEP_API sstep_status sstep_solve(sstep_handle h, const double* b, double* x, sstep_info* info);

/* Single-system handle: solve nrhs right-hand sides with the same A one after another;
 * b[i], x[i] as in sstep_solve; infos may be NULL or hold nrhs entries.
 * Batched handle (nsys systems): b and x hold nsys * nrhs DEVICE pointers, system-major
 * (b[sys * nrhs + j] is right-hand side j of system sys, n_sys doubles; x likewise, x^(0) on
 * entry); infos may be NULL or hold nsys * nrhs entries in the same order.  All problems are
 * solved by one persistent kernel launch (replayed from a CUDA graph): each thread-block
 * cluster takes the next (system, right-hand side) problem from a device work queue, largest
 * systems first, and runs Algorithm 1 on it to convergence with cluster barriers and
 * distributed-shared-memory reductions.  Results equal those of independent solves up to
 * rounding order.  Returns the first non-OK status, else SSTEP_OK. */
SSTEP_API sstep_status sstep_solve_batched(sstep_handle h, int nrhs, const double* const* b,
                                 double* const* x, sstep_info* infos);

/* Batched handle: the configuration in use (chosen by the autotuner where the options left
 * it open): step size s, CTAs per cluster, threads per CTA, number of clusters resident at
 * once (= workspace slots), and the wall time the autotuner spent at set-up (0 when the
 * choice came from its in-process cache or from the options).  Any output may be NULL.
 * SSTEP_ERR_INVALID for a single-system handle. */
SSTEP_API sstep_status sstep_get_batch_config(sstep_handle h, int* s, int* cluster, int* threads,
                                              int* slots, double* tune_ms);

/* AMG handle (precond kind SSTEP_PREC_AMG): the hierarchy, for inspection.  *nlevels receives
 * the number of levels.  sstep_amg_level copies level l's matrix (CSR: rowptr n+1, colind nnz,
 * vals nnz) and its aggregation map agg (n entries; the coarsest level has none and agg is left
 * untouched) into HOST arrays; any pointer may be NULL (n and nnz first, to size the arrays). */
SSTEP_API sstep_status sstep_amg_levels(sstep_handle h, int* nlevels);
SSTEP_API sstep_status sstep_amg_level(sstep_handle h, int l, int64_t* n, int64_t* nnz,
                                       int64_t* rowptr, int32_t* colind, double* vals,
                                       int32_t* agg);
/* x = M^{-1} b: one V-cycle of the handle's AMG on device vectors b and x (n doubles each,
 * distinct), ordered on the handle's stream and finished on return. */
SSTEP_API sstep_status sstep_amg_apply(sstep_handle h, const double* b, double* x);

/* Reduced-solve diagnostics of the last solve (Section 3.3 experiments): for every outer
 * iteration k < *count, eta_a[k] = ||Q_k^T r^(k) - W_k alpha_k||_2 / ||Q_k^T r^(k)||_2 and, for
 * k < *count - 1, eta_b[k] = ||-Q_k^T AZ_{k+1} - W_k beta_k||_F / ||Q_k^T AZ_{k+1}||_F; W receives
 * W_k (s x s column-major, one after another) for k < *countw <= min(maxw, 64).  HOST arrays
 * of maxlen (eta_a, eta_b) and maxw * s * s (W) doubles; any output may be NULL.  The device
 * keeps each outer iteration's reduced systems (W_k, Q_k^T r, alpha_k, -Q_k^T AZ_{k+1}, beta_k:
 * plain stores in the reduced-solve step, no arithmetic on the solve's path); this call forms
 * the eta values from them in FP64 on the host.  *count = 0 for classical PCG. */
SSTEP_API sstep_status sstep_get_diagnostics(sstep_handle h, double* eta_a, double* eta_b,
                                             int maxlen, int* count, double* W, int maxw,
                                             int* countw);

/* Release everything the handle owns (NULL is accepted). */
SSTEP_API sstep_status sstep_free(sstep_handle h);

/* Static description of a status code. */
SSTEP_API const char* sstep_status_string(sstep_status s);
/* Description of the last failure on the calling thread ("" if none). */
SSTEP_API const char* sstep_last_error(void);

/* ------------------------------------------------------------------ hot-path steps
 * The steps of one outer iteration, exposed one by one on an existing handle (its operator,
 * preconditioner, Chebyshev scalars and stream).  All pointers are device pointers with
 * leading dimension n; the calls are asynchronous on the handle's stream. */

/* Algorithm 2 (MPK for the Chebyshev basis): from residual r, write
 * Z = [z_1 .. z_s] with z_j = T_{j-1}(A_hat) M^{-1} r and AZ = [A z_1 .. A z_s]
 * (the columns 2..s+1 of the paper's P; column 1 of P is r itself).
 * s_override in 1..16 replaces the handle's s (0 keeps it).  The recurrence runs on z
 * directly: z_{q+1} = 2 c_alpha M^{-1}(A z_q) - 2 c_sigma z_q - c_gamma z_{q-1}. */
SSTEP_API sstep_status sstep_mpk(sstep_handle h, const double* r, double* Z, double* AZ, int s_override);

/* Block Gram products (the step system W = Q^T AQ and the conjugation right-hand sides
 * -Q^T AZ of Section 2): for e = 0..ne-1,
 * out[e] = sum_i L[pairs[2e]][i] * R[pairs[2e+1]][i], i < n.  L: nl device pointers to n-vectors,
 * R: nr device pointers; pairs: 2*ne host ints; out: ne doubles (device).  nl, nr <= 40,
 * ne <= 512.  Deterministic: the same inputs and launch give bit-identical sums.
 * stream: cudaStream_t as void*. */
SSTEP_API sstep_status sstep_block_gram(int64_t n, int nl, const double* const* L, int nr,
                              const double* const* R, int ne, const int* pairs, double* out,
                              void* stream);

/* sstep_block_gram without any device allocation.  The paper has no counterpart: this is a
 * library convenience for callers that cannot allocate device memory when they call it, for
 * example programs whose framework already holds the device's memory in its own pool (an extra
 * cudaMalloc fails or fragments it) or latency-sensitive callers that must not pay for the
 * allocator or for a free that waits on the device.  Same arguments and result as
 * sstep_block_gram; the caller still passes L, R and out.  Scratch comes from one fixed area of
 * about 1.06 MB compiled into the library, kept on every GPU that loads it until exit.  Limits:
 * ne <= 256 (else SSTEP_ERR_INVALID with a message), devices with at most 256 SMs (else
 * SSTEP_ERR_UNSUPPORTED).  The first call on a device looks up the area's address and keeps
 * it for that device ordinal: make it before any stream capture, and do not call this entry
 * point on a device again after cudaDeviceReset on it (the kept address belongs to the
 * destroyed context).  All calls share the area: calls that overlap on the GPU (different
 * streams, or threads without ordering) race and return wrong sums, so order them. */
SSTEP_API sstep_status sstep_block_gram_noalloc(int64_t n, int nl, const double* const* L, int nr,
                                                const double* const* R, int ne, const int* pairs,
                                                double* out, void* stream);

/* nu FGS sweeps from 0 on W X = B for nrhs right-hand sides (Section 3.1, Eq. fgs-iteration on
 * W itself: W = D + L_W + L_W^T).  W: s x s column-major, B and X: s x nrhs column-major, all
 * device pointers; 1 <= s <= 16, 1 <= nrhs <= 16.  Breakdown (W_ii <= 0 or non-finite) is
 * written to *status_dev (device int, may be NULL) as SSTEP_ERR_BREAKDOWN, else SSTEP_OK.
 * solver = SSTEP_GRAM_CHOLESKY solves exactly instead; SSTEP_GRAM_FGS_OPERATOR (s <= 8,
 * else SSTEP_ERR_UNSUPPORTED) forms P_nu and returns X = P_nu B, the products in increasing
 * order of the summed index.  stream: cudaStream_t as void*. */
SSTEP_API sstep_status sstep_fgs(int s, const double* W, int nrhs, const double* B, int nu, int solver,
                       double* X, int* status_dev, void* stream);

/* The block updates of Section 2 fused: with beta (s x s) and alpha (s) in device memory,
 * Q <- Z + Q beta, AQ <- AZ + AQ beta, x <- x + Q alpha, r <- r - AQ alpha (new Q, AQ),
 * and *rr_out = ||r||^2 (device double).  beta may be NULL (first outer iteration: Q <- Z,
 * AQ <- AZ).  Blocks have leading dimension n. */
SSTEP_API sstep_status sstep_block_update(sstep_handle h, const double* Z, const double* AZ, double* Q,
                                double* AQ, const double* alpha, const double* beta, double* x,
                                double* r, double* rr_out, int s_override);

/* y = A x with the handle's operator (device pointers). */
SSTEP_API sstep_status sstep_spmv(sstep_handle h, const double* x, double* y);

/* lambda_max and lambda_min used by the handle, and the Chebyshev scalars of Section 2. */
SSTEP_API sstep_status sstep_get_basis_info(sstep_handle h, double* lambda_min, double* lambda_max,
                                  double* c_alpha, double* c_sigma, double* c_gamma,
                                  int* power_iters_run);

/* Gradient of a loss L(x(A)) with respect to the stored entries of a CSR matrix A, given the
 * adjoint lambda = A^{-T} dL/dx (for SPD A, a second solve with the same handle):
 * dL/dA_ij = -lambda_i x_j, written for each stored (i, j) in CSR order:
 * grad_vals[k] = (accumulate ? grad_vals[k] : 0) - scale * lambda[row(k)] * x[colind[k]].
 * Device pointers (rowptr n+1, colind nnz, lambda and x n, grad_vals nnz).  The paper has no
 * counterpart; it makes the solver differentiable with respect to A's values. */
SSTEP_API sstep_status sstep_pattern_grad(int64_t n, const int64_t* rowptr, const int32_t* colind,
                                          const double* lam, const double* x, double* grad_vals,
                                          double scale, int accumulate, void* stream);

/* The differentiated Q1 diffusion solve (the paper has no counterpart; this is the adjoint of a
 * linear solve).  Q1 finite elements on the unit cells of an (nx+1) x (ny+1) x (nz+1) cell grid,
 * one conductivity per cell (cell cx + (nx+1)(cy + (ny+1) cz)), unknowns at the nx*ny*nz
 * interior vertices (vertex i + nx (j + ny k) at grid point (i+1, j+1, k+1)), Dirichlet
 * boundary eliminated: A = sum_c kappa_c P_c^T K_ref P_c with the trilinear element stiffness
 * K_ref (local vertex lx + 2 ly + 4 lz).  All pointers are device pointers; stream is a
 * cudaStream_t as void*; the calls are stream-ordered and allocate nothing but the 4-byte flag
 * of sstep_q1_assemble. */

/* kappa[c] = exp(theta[c]) for c < ncell (conductivity from log-conductivity). */
SSTEP_API sstep_status sstep_q1_exp(int64_t ncell, const double* theta, double* kappa, void* stream);

/* Assembled CSR values of the Q1 operator for conductivities kappa on the pattern (rowptr
 * int64 n+1, colind int32) of an n = nx*ny*nz vertex grid: vals[k] for entry (i, j) = sum
 * over the cells c shared by vertices i and j of kappa_c K_ref[l_i(c), l_j(c)].  A column that
 * is not one of the 27 neighbours of its row: SSTEP_ERR_INVALID (the stream is synchronised to
 * read the flag). */
SSTEP_API sstep_status sstep_q1_assemble(int nx, int ny, int nz, const double* kappa,
                                         const int64_t* rowptr, const int32_t* colind,
                                         double* vals, void* stream);

/* Gradient of a loss L(x), x = A(kappa)^{-1} b, with respect to the cell conductivities, from
 * x and the adjoint lambda (A lambda = dL/dx): grad[c] (+)= -lambda_c^T K_ref x_c, where
 * lambda_c, x_c hold the cell's 8 vertex values (0 at boundary vertices).  wrt_log = 1 gives
 * dL/dtheta_c = kappa_c dL/dkappa_c for kappa = exp(theta).  grad: (nx+1)(ny+1)(nz+1)
 * doubles. */
SSTEP_API sstep_status sstep_q1_grad(int nx, int ny, int nz, const double* kappa, const double* lam,
                                     const double* x, double* grad, int wrt_log, int accumulate,
                                     void* stream);

/* Gradient of a loss with respect to the weights of a batch of 7-point stencil systems
 * A_i = wc_i I + wo_i N (N: the sum of the six axis neighbours inside the grid; the form the
 * batched solver takes), each with `nrhs` right-hand sides, from the solutions x and the adjoint
 * solutions lambda (A_i lambda = dL/dx): grad[2 i] = dL/dwc_i = -sum_r lambda_ir^T x_ir and
 * grad[2 i + 1] = dL/dwo_i = -sum_r lambda_ir^T N x_ir, the right-hand sides r summed in
 * increasing order.  dims: host int[3 nsys] (nx, ny, nz per system); lam, x: host arrays of
 * nsys * nrhs device pointers, system-major; grad: device double[2 nsys].  Allocates a
 * stream-ordered table of the problems.  The paper has no counterpart. */
SSTEP_API sstep_status sstep_stencil7_weight_grad(int nsys, int nrhs, const int* dims,
                                                  const double* const* lam,
                                                  const double* const* x, double* grad,
                                                  void* stream);

/* Replace the values of the handle's operator, device or host: CSR vals[nnz] (same pattern), or
 * the Q1 cell conductivities ((nx+1)(ny+1)(nz+1) doubles, checked like at set-up).  M^{-1}
 * (Jacobi), the AMG hierarchy and the FP32 copies are refreshed; the Chebyshev interval is
 * kept.  Constant stencils: SSTEP_ERR_INVALID. */
SSTEP_API sstep_status sstep_update_values(sstep_handle h, const double* vals);

/* Residual history of the last solve: relres[k] = ||r^(k)|| / ||b|| for k = 0..iters
 * (recursively updated residual after each outer iteration).  relres: host array of maxlen
 * doubles; *count receives the number written. */
SSTEP_API sstep_status sstep_get_history(sstep_handle h, double* relres, int maxlen, int* count);

/* Device time per phase of one outer iteration, measured with CUDA events on the handle's
 * stream: starting from x = 0 for right-hand side b (device or host, n doubles), runs the first
 * outer iteration and then `iters` more without a stop test, launched one by one.  ms (host,
 * 5 doubles) receives the averages per outer iteration of 4 phases and their sum:
 * literal form: [MPK (all s steps), b2 = -Q^T AZ with beta, the Q/AQ update fused with W, b1,
 * alpha and the previous step's x += Q alpha, r update with the stop test]; one-reduction form:
 * [MPK, Gram reduction with the reduced solves, block update, 0]; PCG: [A p with p^T A p,
 * x/r/z update, direction update, 0].
 * The handle's own x, r and basis blocks are overwritten. */
SSTEP_API sstep_status sstep_profile(sstep_handle h, const double* b, int iters, double* ms);

#ifdef __cplusplus
}
#endif
#endif /* SSTEP_H */
