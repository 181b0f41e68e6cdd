// common.cuh -- internal definitions shared by the translation units of libsstep.so.
// Device-side control block, deterministic grid reductions, operator descriptors.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sstep.h"

namespace sstep {

constexpr int kMaxS = 16;          // largest step size
constexpr int kMaxEntries = 1088;  // largest number of Gram entries per reduction (s = 16, full)
constexpr int kMaxGramVecs = 40;   // largest number of vectors on one side of a Gram product
constexpr int kThreads = 256;      // threads per CTA of the streaming kernels
constexpr int kMaxCtas = 2048;     // upper bound on CTAs of a reduction kernel (partials buffer)
constexpr int kNumTickets = 8;
// Register tiles of the Gram kernels: at most kMaxTiles tiles of kTileMaxR x kTileMaxC products.
constexpr int kTileMaxR = 8, kTileMaxC = 17, kMaxTiles = 4;
constexpr int kTiledSmem = 8 * 72 > 1100 ? 8 * 72 : 1100;  // warp partials / sums + tail scratch

enum Ticket { TK_GRAM = 0, TK_UPDATE = 1, TK_OP = 2, TK_NORM = 3, TK_PCG1 = 4, TK_PCG2 = 5 };

// Reduced-system mode of the Gram kernel's tail (run by the last CTA after the reduction).
enum GramMode {
  GM_SUMS = 0,           // only write the reduced sums
  GM_ONESYNC_FIRST = 1,  // k = 0: W = Z^T AZ, b1 = Z^T r, alpha = FGS(W, b1)
  GM_ONESYNC = 2,        // beta = FGS(W_k, -Q^T AZ); W_{k+1} = ...; alpha = FGS(W_{k+1}, b1)
  GM_LITERAL_W = 3,      // W = Q^T AQ, b1 = Q^T r, alpha = FGS(W, b1)          (step system)
  GM_LITERAL_B2 = 4      // beta = FGS(W, -Q^T AZ)                              (conjugation)
};

// Update kernel modes (the block updates of Section 2).
enum UpdMode {
  UM_FIRST = 0,  // Q = Z, AQ = AZ, then x += Q alpha, r -= AQ alpha
  UM_FUSED = 1,  // Q = Z + Q beta, AQ = AZ + AQ beta, then x += Q alpha, r -= AQ alpha
  UM_XR = 2,     // x += Q alpha, r -= AQ alpha only                  (literal form)
  UM_QAQ = 3,    // Q = Z + Q beta, AQ = AZ + AQ beta only (literal form), after the pending
                 // x += Q alpha of the previous step (Ctrl::x_pending)
  UM_R = 4       // r -= AQ alpha, x's step left pending              (literal form solve)
};

// Device-resident control block of one solve.  Written only by the last CTA of a reduction
// kernel (or by single-CTA kernels); read at kernel entry by every CTA of later kernels.
struct Ctrl {
  double nb2;        // ||b||^2
  double rtol2;      // rtol^2
  double tol2;       // (rtol ||b||)^2, set by the initial-residual kernel
  double rr;         // ||r||^2 of the current residual
  double rr0;        // ||r^(0)||^2
  double rz;         // PCG: r^T z
  double rz_prev;    // FP32 PCG: r^T z before the last update (a residual replacement
                     // recomputes r^T z and takes beta against this value)
  double pcg_alpha, pcg_beta;
  double lam, inv_scale, power_tol;  // power method: estimate, 1/previous estimate, stop tolerance
  int power_done, power_iters, power_max;
  int done;          // 1: stop (converged, failed or capped)
  int status;        // sstep_status
  int iters;         // executed updates
  int max_iters;
  int s, nu, solver, full_gram;
  int first_pending; // 1 while the next outer iteration is the first one
  double alpha[kMaxS];
  double beta[kMaxS * kMaxS];    // column-major s x s
  double W[kMaxS * kMaxS];       // W_k used for alpha_k (and for beta_k)
  double P[64];                  // FGS operator P_nu(W_k) (solver SSTEP_GRAM_FGS_OPERATOR, s <= 8)
  int p_valid;                   // 1 once P holds the operator of the current W
  // FP32-basis s-step form: 1 while x still lacks the last step's Q_k alpha_k; the direction
  // update that next reads Q_k adds it, or the fold before a residual replacement does
  int x_pending;
  double sums[kMaxEntries];      // reduced Gram sums of the last reduction
  unsigned int ticket[kNumTickets];
  // the reduced systems of every outer iteration k <= red_max (Section 3.3 experiments), kept
  // by the Gram tails for the host to form eta_alpha and eta_beta: record k (red_stride
  // doubles at red + k red_stride) holds W_k (s x s), b1_k (s), alpha_k (s), B2_k = -Q_k^T
  // AZ_{k+1} (s x s) and beta_k (s x s), each column-major; plain stores, no arithmetic.
  double* red;
  int red_max, red_stride;
};
constexpr int kDiagW = 64;  // outer iterations whose W_k the diagnostics return
__host__ __device__ constexpr int red_stride_for(int s) { return 3 * s * s + 2 * s; }

// ---------------------------------------------------------------- operator descriptors

struct St7TmaMaps;  // TMA descriptors of the FP32 7-point steps (k_operator.cu)
struct StencilOp {
  int nx, ny, nz, points;
  int poisson;       // 1: off-diagonal weights all -1 (fast path)
  double w[27];      // weights in order of increasing linear offset
  double wc;         // centre weight
  const St7TmaMaps* tma;  // FP32 path: tensor maps of the vectors its steps read, or null
};

struct CsrOp {
  int64_t n;
  const int64_t* rowptr;
  const int32_t* colind;
  const double* vals;
};

// Matrix-free Q1 (trilinear finite-element) diffusion operator on the nx*ny*nz interior
// vertices of a grid of (nx+1)(ny+1)(nz+1) unit cells, per-cell conductivity kappa (cell
// cx + (nx+1)(cy + (ny+1) cz)), Dirichlet boundary vertices eliminated.
struct Q1TmaMaps;  // TMA descriptors of the FP32 MPK step (k_q1.cu)
struct Q1Op {
  int nx, ny, nz;
  const double* kappa;    // FP64 conductivities, rows of nx+1
  const float* kappaf;    // FP32 copy for the FP32-basis path (null when unused), rows of kpitch
  int kpitch;             // row pitch of kappaf: nx+1 rounded up to a multiple of 4
  const Q1TmaMaps* tma;   // tensor maps of the basis columns and kappaf, or null
};

// Preconditioner: dinv == nullptr means the uniform scalar dinv_u (M = I gives dinv_u = 1).
struct Prec {
  const double* dinv;
  double dinv_u;
};

__device__ __forceinline__ double prec_d(const Prec& M, int64_t i) {
  return M.dinv ? __ldg(M.dinv + i) : M.dinv_u;
}

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Element i (0-based) of the SplitMix64 stream with the given seed (Steele, Lea, Flood 2014),
// mapped to U[-1, 1): the (i+1)-th state is seed + (i+1) * golden gamma, so every element is
// computed independently.  Used for seeded input vectors (power-method start, test inputs).
__host__ __device__ __forceinline__ double splitmix_pm1(uint64_t seed, int64_t i) {
  uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
}

// Error-free transformations on the FP32 pipe (Knuth's TwoSum; Dekker/Ogita-Rump-Oishi
// products by FMA).  A (hi, lo) pair accumulates products of FP32 numbers with about 48 bits,
// so Gram sums of FP32 vectors carry FP64-class accuracy while the narrow FP64 pipe of this
// part stays idle.  Intrinsics keep the compiler from contracting the sequences.
//
// (hi, lo) += a b in 8 operations: p = fl(a b); TwoSum(hi, p) = s + (t1 + (p - bb)) exactly,
// with bb = s - hi, t1 = hi - (s - bb) exact; the product's own error e = a b - p joins the
// low-order part p - bb in one FMA, fma(a, b, -bb) = fl(a b - bb) = fl((p - bb) + e).  That
// one rounding of a quantity of size <= u (|s| + |p|) costs u^2 (|s| + |p|): the same order as
// the separate TwoProd + TwoSum + two low-order adds (10 operations), which round (err + e).
__device__ __forceinline__ void df_acc_prod(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float t1 = __fsub_rn(hi, __fsub_rn(s, bb));
  const float t2 = __fmaf_rn(a, b, -bb);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(t1, t2));
}

// (hi, lo) += a.x b.x + a.y b.y + a.z b.z + a.w b.w: the four TwoSum steps of df_acc_prod on
// hi, their low-order parts (each t1 + fl(a b - bb)) summed pairwise and added to lo once:
// 7 instead of 8 operations per product, the same u^2 error class per product.
__device__ __forceinline__ float df_step(float& s, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float s1 = __fadd_rn(s, p);
  const float bb = __fsub_rn(s1, s);
  const float t1 = __fsub_rn(s, __fsub_rn(s1, bb));
  const float t2 = __fmaf_rn(a, b, -bb);
  s = s1;
  return __fadd_rn(t1, t2);
}
__device__ __forceinline__ void df_acc_dot4(float& hi, float& lo, float4 a, float4 b) {
  const float l0 = df_step(hi, a.x, b.x), l1 = df_step(hi, a.y, b.y);
  const float l2 = df_step(hi, a.z, b.z), l3 = df_step(hi, a.w, b.w);
  lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(l0, l1), __fadd_rn(l2, l3)));
}

// (ah, al) += (bh, bl), renormalised.
__device__ __forceinline__ void df_add(float& ah, float& al, float bh, float bl) {
  const float s = __fadd_rn(ah, bh);
  const float bb = __fsub_rn(s, ah);
  const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  const float lo = __fadd_rn(err, __fadd_rn(al, bl));
  const float h = __fadd_rn(s, lo);
  ah = h;
  al = __fsub_rn(lo, __fsub_rn(h, s));
}

// Block-wide sum of NV values per thread; result valid in thread 0.  Fixed order.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* NV * 32 */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k * 32 + wid] = v[k];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < nw ? sh[k * 32 + lane] : 0.0;
      v[k] = warp_sum(t);
    }
  }
  __syncthreads();
}

// Final step of a "last CTA to arrive" reduction with per-entry partials: for E = T * K entries
// (T tiles of K values; entry e = tt * K + k), out[e] = sum over b < nblk of
// partials[(tt * nblk + b) * K + k].  Every thread of the CTA works: thread idx takes entry
// idx % E and the partials b = idx / E, idx / E + G, ... (G = blockDim / E groups), eight L2
// loads in flight at a time; then the G group sums of each entry are added: in order by one
// thread when G <= 32, else by one warp (lane l taking groups l, l + 32, ... in order, then a
// fixed butterfly over the lanes).  On this part an FP64 warp instruction occupies its
// sub-partition for tens of cycles however few lanes are active, so a chain of G dependent
// additions (G = 256 for a single entry) becomes G / 32 + 5.  A fixed order for a given launch
// shape, so deterministic.  E <= 1024.  Ends with __syncthreads().
__device__ __forceinline__ void sum_partials(const double* partials, unsigned int nblk, int K,
                                             int T, double* out) {
  constexpr int kScratch = 1024;
  __shared__ double scratch[kScratch];
  const int E = K * T;
  const int G = max(1, min((int)blockDim.x, kScratch) / E);
  for (int idx = threadIdx.x; idx < G * E; idx += blockDim.x) {
    const int e = idx % E, g = idx / E;
    const double* p = partials + (size_t)(e / K) * nblk * K + (e % K);
    double v = 0.0;
    unsigned int b = g;
    for (; b + 7u * G < nblk; b += 8u * G) {
      double t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = __ldcg(p + (size_t)(b + u * G) * K);
#pragma unroll
      for (int u = 0; u < 8; ++u) v += t[u];
    }
    for (; b < nblk; b += G) v += __ldcg(p + (size_t)b * K);
    scratch[idx] = v;
  }
  __syncthreads();
  if (G <= 32) {  // a short chain: one thread per entry adds the group sums in order
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
      double v = 0.0;
      for (int g = 0; g < G; ++g) v += scratch[g * E + e];
      out[e] = v;
    }
  } else {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = w; e < E; e += nw) {
      double v = 0.0;
      for (int g = lane; g < G; g += 32) v += scratch[g * E + e];
      v = warp_sum(v);
      if (lane == 0) out[e] = v;
    }
  }
  __syncthreads();
}

// Deterministic grid reduction: every CTA contributes NV values; the last CTA to arrive sums
// the per-CTA partials in a fixed order and returns true (result in `tot`, valid in all of
// its threads).  No CTA waits for another: the last arriving CTA does the final step.
template <int NV>
__device__ bool grid_sum_last(double (&v)[NV], double* partials, unsigned int* ticket,
                              double (&tot)[NV]) {
  __shared__ double sh[NV * 32];
  __shared__ bool last;
  // Grids may be 1D, 2D or 3D: partials are indexed by the linear block index.
  const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  const unsigned int nblk = gridDim.x * gridDim.y * gridDim.z;
  block_sum<NV>(v, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) partials[(size_t)bid * NV + k] = v[k];
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    last = (t == nblk - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int b = threadIdx.x; b < (int)nblk; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += __ldcg(partials + (size_t)b * NV + k);
  }
  block_sum<NV>(acc, sh);
  __shared__ double res[NV];
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) res[k] = acc[k];
    *ticket = 0u;  // re-arm for the next launch (stream order separates launches)
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) tot[k] = res[k];
  return true;
}

// Warp stage of df_grid_sums for K <= 64 values per lane, a reduce-scatter: with KP the next
// power of two >= K (missing values 0) and L = min(5, log2 KP), level t < L pairs lanes at
// distance 16 >> t; the lane whose bit (4 - t) is set keeps the upper half of its current values
// and sends the lower half, its partner the reverse, and each adds what it receives.  After the
// L levels a lane holds C = KP >> L values, value c being index ((lane >> (5 - L)) << log2 C) + c
// summed over the 2^L lanes that share the lane's other bits; plain butterfly levels over the
// remaining 5 - L lane bits finish the warp sums.  KP - C + 5 - L double-float additions per lane
// instead of 5 K.
template <int K>
struct DfScatter {
  static constexpr int KP = K <= 1 ? 1 : K <= 2 ? 2 : K <= 4 ? 4 : K <= 8 ? 8 : K <= 16 ? 16
                          : K <= 32 ? 32 : 64;
  static constexpr int LOGKP = KP == 1 ? 0 : KP == 2 ? 1 : KP == 4 ? 2 : KP == 8 ? 3 : KP == 16 ? 4
                             : KP == 32 ? 5 : 6;
  static constexpr int L = LOGKP < 5 ? LOGKP : 5;
  static constexpr int C = KP >> L;         // values per lane at the end
  static constexpr int LOGC = LOGKP - L;
  static constexpr int R = 1 << (5 - L);    // lanes per group that end with the same values
  // index of value c held by `lane`
  __device__ static int index(int lane, int c) { return ((lane >> (5 - L)) << LOGC) + c; }
};

template <int K>
__device__ __forceinline__ void df_warp_scatter(const float (&hi)[K], const float (&lo)[K],
                                                float (&vh)[DfScatter<K>::C],
                                                float (&vl)[DfScatter<K>::C]) {
  using D = DfScatter<K>;
  static_assert(K >= 1 && K <= 64, "K <= 64 values per thread");
  const int lane = threadIdx.x & 31;
  float h[D::KP], l[D::KP];
#pragma unroll
  for (int k = 0; k < D::KP; ++k) {
    h[k] = k < K ? hi[k] : 0.0f;
    l[k] = k < K ? lo[k] : 0.0f;
  }
#pragma unroll
  for (int t = 0; t < D::L; ++t) {
    const int half = D::KP >> (t + 1), o = 16 >> t;
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const float sh = upper ? h[k] : h[k + half], sl = upper ? l[k] : l[k + half];
      const float kh = upper ? h[k + half] : h[k], kl = upper ? l[k + half] : l[k];
      const float rh = __shfl_xor_sync(0xffffffffu, sh, o);
      const float rl = __shfl_xor_sync(0xffffffffu, sl, o);
      h[k] = kh;
      l[k] = kl;
      df_add(h[k], l[k], rh, rl);
    }
  }
#pragma unroll
  for (int c = 0; c < D::C; ++c) {
    float a = h[c], b = l[c];
#pragma unroll
    for (int o = 16 >> D::L; o > 0; o >>= 1) {
      const float rh = __shfl_xor_sync(0xffffffffu, a, o), rl = __shfl_xor_sync(0xffffffffu, b, o);
      df_add(a, b, rh, rl);
    }
    vh[c] = a;
    vl[c] = b;
  }
}

// Writes a warp's K sums (after df_warp_scatter) to out[0 .. K) as FP64, one conversion per lane
// that ends with a value.
template <int K>
__device__ __forceinline__ void df_scatter_store(const float (&vh)[DfScatter<K>::C],
                                                 const float (&vl)[DfScatter<K>::C], double* out) {
  using D = DfScatter<K>;
  const int lane = threadIdx.x & 31;
  if (lane % D::R != 0) return;
#pragma unroll
  for (int c = 0; c < D::C; ++c) {
    const int v = D::index(lane, c);
    if (v < K) out[v] = (double)vh[c] + (double)vl[c];
  }
}

// Last step of df_grid_sums: out[e] = sum over b < nblk of partials[b * K + e] (K <= 64).
// G = the largest power of two with G K <= blockDim groups; thread g K + e loads the partials
// b = g, g + G, ..., up to 24 at a time (one round trip to L2 for up to 24 G CTAs) and adds them
// by a pairwise tree; the G group sums of an entry are then added by a tree over g in shared
// memory.  A fixed order for a given launch shape.  Ends with __syncthreads().
__device__ __forceinline__ void sum_partials_df(const double* partials, unsigned int nblk, int K,
                                                double* out) {
  __shared__ double scr[kThreads];
  int G = 1;
  while (2 * G * K <= (int)blockDim.x && 2 * G * K <= kThreads) G *= 2;
  const int idx = threadIdx.x;
  if (idx < G * K) {
    const int e = idx % K, g = idx / K;
    double v = 0.0;
    for (unsigned int b0 = g; b0 < nblk; b0 += 24u * G) {
      double t[24];
#pragma unroll
      for (int u = 0; u < 24; ++u) {
        const unsigned int b = b0 + u * G;
        t[u] = b < nblk ? __ldcg(partials + (size_t)b * K + e) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 12; ++u) t[u] += t[u + 12];
#pragma unroll
      for (int u = 0; u < 6; ++u) t[u] += t[u + 6];
#pragma unroll
      for (int u = 0; u < 3; ++u) t[u] += t[u + 3];
      v += (t[0] + t[1]) + t[2];
    }
    scr[idx] = v;
  }
  __syncthreads();
  for (int h = G / 2; h >= 1; h /= 2) {
    if (idx < h * K) scr[idx] += scr[idx + h * K];
    __syncthreads();
  }
  if (idx < K) out[idx] = scr[idx];
  __syncthreads();
}

// Per-thread double-float (hi, lo) pairs -> FP64 per-CTA partials -> fixed-order sum in the
// last CTA (no CTA waits for another).  Grids may be 1D, 2D or 3D; K <= 64, blockDim a multiple
// of 32 up to kThreads.  buf: shared memory of at least (blockDim.x / 32) * K doubles.  Returns
// true in the last CTA, with the K sums in buf[0..K) (valid in all of its threads).
template <int K>
__device__ bool df_grid_sums(const float (&hi)[K], const float (&lo)[K], double* buf,
                             double* partials, unsigned int* ticket) {
  static_assert(K >= 1 && K <= 64, "K <= 64 values per thread");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  const unsigned int nblk = gridDim.x * gridDim.y * gridDim.z;
  // the warp stage on the FP32 pipe; each lane then holds the warp sum of one value, so that a
  // warp converts its K values to FP64 in one instruction sequence (an FP64 instruction costs a
  // sub-partition tens of cycles however few of its lanes are active)
  float vh[DfScatter<K>::C], vl[DfScatter<K>::C];
  df_warp_scatter<K>(hi, lo, vh, vl);
  df_scatter_store<K>(vh, vl, buf + wid * K);
  __syncthreads();
  // the warps' sums of a value in four interleaved chains
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int w = 0;
    for (; w + 3 < nw; w += 4) {
      a0 += buf[w * K + k];
      a1 += buf[(w + 1) * K + k];
      a2 += buf[(w + 2) * K + k];
      a3 += buf[(w + 3) * K + k];
    }
    for (; w < nw; ++w) a0 += buf[w * K + k];
    partials[(size_t)bid * K + k] = (a0 + a1) + (a2 + a3);
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(ticket, 1u) == nblk - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  sum_partials_df(partials, nblk, K, buf);
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// Stop test of Algorithm 1 on ||r||^2 (also used by PCG), executed by one thread.
__device__ __forceinline__ void stop_test(Ctrl* c, double rr) {
  c->rr = rr;
  c->iters += 1;
  if (!(rr == rr) || rr > 1.79e308) {
    c->status = SSTEP_ERR_NONFINITE;
    c->done = 1;
  } else if (rr <= c->tol2) {
    c->status = SSTEP_OK;
    c->done = 1;
  } else if (c->iters >= c->max_iters) {
    c->status = SSTEP_NOT_CONVERGED;
    c->done = 1;
  }
}

}  // namespace sstep

// ---------------------------------------------------------------- host-side launchers
// (defined in the kernel translation units, called by the API translation unit)
namespace sstep {

struct OpDesc {
  int kind;  // SSTEP_MATRIX_*
  StencilOp st;
  CsrOp csr;
  Q1Op q1;
  int64_t n;
};

// Epilogue selector of the operator kernels.
enum OpEpi {
  EP_SPMV = 0,      // y = A u
  EP_MPK = 1,       // Az = A u;  znext = c1 M^{-1}(A u) - c2 u - c3 zprev
  EP_MPK_FIRST = 2, // u = r: z1 = M^{-1} r;  Az = A z1;  z2 = c1 M^{-1} Az - c2 z1
  EP_RESID = 3,     // r = b - A u; reductions ||r||^2, ||b||^2   (initial residual)
  EP_POWER = 4,     // y = scale * M^{-1} A u; reduction ||y||^2
  EP_PCG_AP = 5,    // Ap = A p; reduction p^T Ap
  EP_TRUERES = 6,   // reduction ||b - A u||^2 (no store)
  EP_RR = 7         // residual replacement r = b - A u (FP64), split into FP32 hi + lo,
                    // ||r||^2 and the stop test on it
};

struct EpiArgs {
  int epi;
  const double* u;      // operator input
  double* y;            // A u (stored when non-null)
  double* znext;        // MPK: next basis vector
  double* z1;           // MPK first step: z1 output
  const double* zprev;  // MPK: z_{q-1} (null on the second basis vector)
  const double* b;      // residual epilogues
  float* rhi;           // residual epilogues of the mixed path: r split into FP32 hi + lo
  float* rlo;
  double c1, c2, c3;    // recurrence coefficients
  double a1u;           // c1 * M^{-1} when M^{-1} is a uniform scalar
  Prec M;
  Ctrl* ctrl;
  double* partials;
};

cudaError_t launch_operator(const OpDesc& A, const EpiArgs& e, cudaStream_t st);

// ---------------------------------------------------------------- FP32-basis (mixed) path
// One MPK step with FP32 storage and arithmetic (Algorithm 2; recurrence on z).
struct MpkF32Args {
  const float* u;      // z_q (first step: r_hi, the FP32 value nearest r)
  float* y;            // A z_q
  float* znext;        // z_{q+1} (null on the last step)
  float* z1;           // first step: z_1 = M^{-1} r
  const float* zprev;  // z_{q-1} (null on the first two steps)
  const float* dinv;   // non-uniform M^{-1} in FP32, or null
  float dinv_u;        // uniform M^{-1}
  float c1, c2;        // z_{q+1} = c1 M^{-1} (A z_q) - c2 z_q - z_{q-1}
  float w[27];         // stencil weights in FP32
  float wc;
  const float* valsf;  // CSR values in FP32
  int first;
  Ctrl* ctrl;
  // FP32 PCG product step (first = 0, znext = null): with pap set, the kernel also forms
  // p^T (A p) (u = p, y = A p) in double-float, and its last CTA sets alpha = r^T z / p^T A p
  int pap;
  double* partials;
};
cudaError_t launch_mpk_f32(const OpDesc& A, const MpkF32Args& e, cudaStream_t st);
// Tensor maps for the TMA-fed FP32 7-point steps: one per vector (cols[c], n floats each) that
// an MPK or PCG product step reads.  Null when the grid does not allow them (not 7 points, nx
// not a multiple of 4, nx < 72 or ny < 18) or the driver cannot encode them; the steps then run
// on plain loads.
St7TmaMaps* st7_tma_build(const StencilOp& op, const float* const* cols, int ncols);
void st7_tma_free(St7TmaMaps* m);

// FP32 PCG product step: the last CTA turns the grid's double-float sum p^T (A p) into
// alpha = r^T z / p^T A p (breakdown when p^T A p is not positive and finite).  Reached by every
// thread of every CTA; nothing is changed when an earlier failure already stopped the solve.
__device__ __forceinline__ void pap_finish(const MpkF32Args& e, const float (&hi)[1],
                                           const float (&lo)[1]) {
  __shared__ double buf[32];
  if (!df_grid_sums<1>(hi, lo, buf, e.partials, &e.ctrl->ticket[TK_PCG1])) return;
  if (threadIdx.x == 0) {
    Ctrl* c = e.ctrl;
    const double pap = buf[0];
    if (c->done) return;
    if (!(pap > 0.0) || pap > 1.79e308) {
      c->status = SSTEP_ERR_BREAKDOWN;
      c->done = 1;
    } else {
      c->pcg_alpha = c->rz / pap;
    }
  }
}

// Q1 operator kernels (k_q1.cu), reached through launch_operator / launch_mpk_f32.
cudaError_t launch_q1_operator(const Q1Op& A, const EpiArgs& e, cudaStream_t st);
cudaError_t launch_q1_mpk_f32(const Q1Op& A, const MpkF32Args& e, cudaStream_t st);
int q1_grid_ctas(const Q1Op& A);
// Set-up pass over the vertices: *bad = 1 when a conductivity is not finite and positive;
// dinv (if non-null) = 1 / a_ii; out_min[CTA] = the CTA's minimum of the Gershgorin lower
// bound (jacobi: 1 - sum_j |a_ij| / a_ii, else a_ii - sum_j |a_ij|, j != i).
int q1_setup_ctas(int64_t n);
cudaError_t launch_q1_setup(const Q1Op& A, int jacobi, double* dinv, double* out_min, int* bad,
                            cudaStream_t st);
// FP32 conductivities with rows padded to kpitch (the layout the tensor map needs).
cudaError_t launch_q1_kappaf(const Q1Op& A, float* kappaf, cudaStream_t st);
// Tensor maps for the TMA-fed FP32 MPK step: one per basis column (cols[c], n floats each) and
// one for kappaf.  Null when the grid does not allow them (nx not a multiple of 4) or the
// driver cannot encode them; the step then runs on plain loads.
Q1TmaMaps* q1_tma_build(const Q1Op& A, const float* const* cols, int ncols);
void q1_tma_free(Q1TmaMaps* m);

// Blocks of the mixed path: Q, AQ, Z, AZ in FP32; x and r as FP64 plus FP32 (hi, lo)
// increments; Gram sums accumulated in double-float (TwoProd + TwoSum on the FP32 pipe).
struct MixedArgs {
  int64_t n, ld;
  const float* Z;
  const float* AZ;
  float* Q;
  float* AQ;
  float* rhi;   // r = rhi + rlo between residual replacements
  float* rlo;
  float* xhi;   // x = x64 + xhi + xlo between residual replacements
  float* xlo;
  Ctrl* ctrl;
  double* partials;
  double* hist;
};
// Tiles of FP32 Gram products (double-float accumulation); ylo: optional low part of a column.
struct GramTilesF {
  int64_t n;
  int ntiles, mode, ne;
  const float* x[kMaxTiles][kTileMaxR];
  const float* y[kMaxTiles][kTileMaxC];
  const float* ylo[kMaxTiles][kTileMaxC];
  short out[kMaxTiles][kTileMaxR * kTileMaxC];
  Ctrl* ctrl;
  double* partials;
};
cudaError_t launch_gram_b2_f32(const MixedArgs& a, int s, cudaStream_t st);
cudaError_t launch_upd_gram_f32(const MixedArgs& a, int s, bool first, cudaStream_t st);
cudaError_t launch_update_xr_f32(const MixedArgs& a, int s, cudaStream_t st);
cudaError_t launch_d2f(const double* a, float* b, int64_t n, cudaStream_t st);
// g[k] (+)= -scale * lam[row(k)] * x[col(k)] over the CSR pattern
// Differentiated Q1 solve (k_adjoint.cu): kappa = exp(theta); assembled CSR values of the Q1
// operator; dL/dkappa (or dL/dtheta) = -lambda_c^T K_ref x_c per cell.
cudaError_t launch_q1_exp(int64_t ncell, const double* theta, double* kappa, cudaStream_t st);
cudaError_t launch_q1_assemble(int nx, int ny, int nz, const double* kappa, int64_t n,
                               const int64_t* rowptr, const int32_t* colind, double* vals,
                               int* bad, cudaStream_t st);
cudaError_t launch_q1_grad(int nx, int ny, int nz, const double* kappa, const double* lam,
                           const double* x, double* grad, int wrt_log, int accumulate,
                           cudaStream_t st);
// Bilinear forms of a batch of 7-point problems (k_adjoint.cu): per problem lam^T x and
// lam^T (N x), N the six-neighbour sum; then per-group sums with a scale.
struct Bil7Prob {
  int nx, ny, nz;
  const double* lam;
  const double* x;
};
cudaError_t launch_stencil7_bilinear(const Bil7Prob* probs_dev, int nprob, double* out,
                                     cudaStream_t st);
cudaError_t launch_sum_groups(const double* in, int groups, int per, int w, double scale,
                              double* out, cudaStream_t st);
cudaError_t launch_pattern_grad(const CsrOp& A, const double* lam, const double* x, double* g,
                                double scale, int accumulate, cudaStream_t st);
// x64 += xhi + xlo; xhi = xlo = 0 (before a residual replacement and at the end)
// x64 += xhi + xlo (increments zeroed), after adding the pending step Q alpha (Q: the s FP32
// columns at Q with leading dimension ld, alpha = ctrl->alpha) to the increments when
// ctrl->x_pending; clears ctrl->x_pending.  Q == nullptr: no pending step (FP32 PCG).
cudaError_t launch_fold_x(double* x64, float* xhi, float* xlo, int64_t n, Ctrl* ctrl,
                          const float* Q, int64_t ld, int s, cudaStream_t st);

struct GramArgs {
  int64_t n;
  int nl, nr, ne;
  const double* L[kMaxGramVecs];
  const double* R[kMaxGramVecs];
  unsigned short pairs[kMaxEntries];  // (l << 8) | r
  int mode;           // GramMode
  Ctrl* ctrl;
  double* partials;
  double* out;        // optional copy of the sums (GM_SUMS)
};
cudaError_t launch_gram(const GramArgs& g, cudaStream_t st);

// Register-tiled Gram products for the structured modes (every block formed, s <= 8).
struct GramTiles {
  int64_t n;
  int ntiles, mode, ne;
  const double* x[kMaxTiles][kTileMaxR];
  const double* y[kMaxTiles][kTileMaxC];
  short out[kMaxTiles][kTileMaxR * kTileMaxC];  // entry of product (i, j), -1 = not needed
  Ctrl* ctrl;
  double* partials;
};
// Direction-block update fused with W, b1 of the next outer iteration (see k_upd_gram), s <= 8.
struct UpdGramArgs {
  int64_t n, ld;
  const double* Z;
  const double* AZ;
  double* Q;
  double* AQ;
  const double* r;
  Ctrl* ctrl;
  double* partials;
  double* x;  // the pending x += Q alpha of the previous step is added here (ctrl->x_pending)
};
cudaError_t launch_upd_gram(const UpdGramArgs& a, int s, bool first, cudaStream_t st);

// Builds the tiles of a Gram mode from the solver's blocks (leading dimension ld) and launches;
// returns cudaErrorNotSupported when the mode/s has no tiled form (caller falls back).
cudaError_t launch_gram_tiled(int mode, int s, int64_t n, int64_t ld, const double* Q,
                              const double* AQ, const double* Z, const double* AZ, const double* r,
                              Ctrl* ctrl, double* partials, cudaStream_t st);
cudaError_t gram_init();  // sets the Gram kernels' dynamic shared-memory limit (call outside capture)
// Pair list of a Gram mode (returns ne; fills nl, nr), and the CTA count of launch_gram.
int gram_pairs(int mode, int s, int full, unsigned short* pairs, int* nl, int* nr);
int gram_ctas();
int update_ctas(int64_t n);
int pcg_ctas(int64_t n);
int gershgorin_ctas(int64_t n);

struct UpdArgs {
  int64_t n, ld;
  int s, mode;
  const double* Z;
  const double* AZ;
  double* Q;
  double* AQ;
  double* x;
  double* r;
  const double* alpha;  // device (s)
  const double* beta;   // device (s x s, column-major)
  Ctrl* ctrl;           // stop test + rr (may be null: then rr_out)
  double* rr_out;
  double* partials;
  unsigned int* ticket;
  double* hist;         // optional ||r||/||b|| history
};
cudaError_t launch_update(const UpdArgs& u, cudaStream_t st);
// x += Q alpha (Q: s FP64 columns with leading dimension ld, alpha = ctrl->alpha) when
// ctrl->x_pending, which it clears: the step the literal-form solve left pending at its end.
cudaError_t launch_flush_x(double* x, const double* Q, int64_t n, int64_t ld, int s, Ctrl* ctrl,
                           cudaStream_t st);

cudaError_t launch_fgs_standalone(int s, const double* W, int nrhs, const double* B, int nu,
                                  int solver, double* X, int* status_dev, cudaStream_t st);

struct PcgArgs {
  int64_t n;
  double* x;
  double* r;
  double* p;
  const double* Ap;
  Prec M;
  Ctrl* ctrl;
  double* partials;
  double* hist;
};
cudaError_t launch_pcg_update(const PcgArgs& a, cudaStream_t st);   // x, r, z, rz, rr, beta
cudaError_t launch_pcg_pdir(const PcgArgs& a, cudaStream_t st);     // p = z + beta p
cudaError_t launch_pcg_init(const PcgArgs& a, cudaStream_t st);     // z = M^-1 r, p = z, rz

// Classical PCG with the FP32-basis path's precision recipe: p and A p in FP32, x and r as
// FP32 (hi, lo) increments over the FP64 x and a residual replaced in FP64 every rr_period
// iterations, reductions in double-float.  z = M^{-1} r_hi is formed where it is used.
struct PcgF32Args {
  int64_t n;
  float* p;
  const float* Ap;
  float* xhi;
  float* xlo;
  float* rhi;
  float* rlo;
  const float* dinv;  // non-uniform M^{-1} in FP32, or null
  float dinv_u;       // uniform M^{-1}
  Ctrl* ctrl;
  double* partials;
  double* hist;
};
// x += alpha p, r -= alpha Ap (double-float), r^T z and ||r||^2, stop test, beta
cudaError_t launch_pcgf_update(const PcgF32Args& a, cudaStream_t st);
// r^T z of the current r (after the initial residual or a replacement): init sets beta = 0,
// else beta = (r^T z) / rz_prev
cudaError_t launch_pcgf_rz(const PcgF32Args& a, int init, cudaStream_t st);
// p = z + beta p (init: p = z)
cudaError_t launch_pcgf_pdir(const PcgF32Args& a, int init, cudaStream_t st);

cudaError_t launch_fill_splitmix(double* v, int64_t n, uint64_t seed, cudaStream_t st);
cudaError_t launch_jacobi_csr(const CsrOp& A, double* dinv, int* bad, cudaStream_t st);
cudaError_t launch_csr_check(const CsrOp& A, int64_t nnz, int* bad, cudaStream_t st);
cudaError_t launch_norm2(const double* v, int64_t n, Ctrl* c, double* partials, int which,
                         cudaStream_t st);
cudaError_t launch_gershgorin_csr(const CsrOp& A, int jacobi, double* out_min, cudaStream_t st);

int operator_grid_ctas(const OpDesc& A);  // CTAs of one operator launch (partials sizing)

// Sets the calling thread's message returned by sstep_last_error() (defined in api.cu).
void set_last_error(const char* msg);

// Aggregation AMG preconditioner (amg.cu): host set-up, device V-cycle.
struct AmgHier;
sstep_status amg_build(const int64_t* rowptr_dev, const int32_t* colind_dev, const double* vals_dev,
                       int64_t n, int64_t nnz, int64_t coarse_max, int max_levels,
                       cudaStream_t st, AmgHier** out);
cudaError_t amg_apply(const AmgHier* H, const double* b, double* x, cudaStream_t st);  // b != x
int amg_kernels_per_apply(const AmgHier* H);
int amg_nlevels(const AmgHier* H);
sstep_status amg_level_copy(const AmgHier* H, int l, int64_t* n, int64_t* nnz, int64_t* rowptr,
                            int32_t* colind, double* vals, int32_t* agg);
void amg_free(AmgHier* H);
cudaError_t launch_cheb_combine(int64_t n, const double* t, const double* zq, const double* zprev,
                                double c1, double c2, double c3, double* znext, cudaStream_t st);
cudaError_t launch_power_scale(int64_t n, double* t, Ctrl* c, double* partials, cudaStream_t st);

// Batched persistent solver (batch.cu): many 7-point stencil systems x right-hand sides.
struct BatchCtx;
sstep_status batch_setup(const sstep_matrix* A, int nsys, const sstep_precond* M,
                         const sstep_opts* o, cudaStream_t st, BatchCtx** out);
sstep_status batch_solve(BatchCtx* b, int nrhs, const double* const* bv, double* const* xv,
                         sstep_info* infos);
void batch_config(const BatchCtx* b, int* s, int* cluster, int* threads, int* slots,
                  double* tune_ms);
void batch_free(BatchCtx* b);

}  // namespace sstep
