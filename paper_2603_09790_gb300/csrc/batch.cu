// batch.cu -- batched persistent PCG-S: many independent 7-point stencil systems, each with
// several right-hand sides, solved by one kernel launch.
//
// Each (system, right-hand side) pair is a "problem".  A thread-block cluster of C CTAs takes
// the next problem from a device work queue (largest systems first) and runs Algorithm 1
// (literal form: the step system fused with the direction-block update, b2 after the MPK of
// Algorithm 2) on it to
// convergence, then takes the next one.  The problem's unknowns are split into C contiguous
// ranges, one per CTA; every reduction is a warp-shuffle and shared-memory sum inside each CTA,
// then a fixed-order sum over the C CTAs' partials read through distributed shared memory
// after a cluster barrier.  Every CTA of the cluster therefore holds bit-identical sums, runs
// the s x s FGS solves itself, and takes the same control decisions: no grid-wide
// synchronisation, no flag spinning, only hardware cluster barriers.  Stencil neighbours that
// another CTA owns are read through L2 (ld.global.cg) after the barrier that follows their
// writes.
//
// The basis is FP64 or FP32 (FP32_RR): with FP32 the Gram sums and the x, r increments are
// double-float on the FP32 pipe (x = x_fp64 + (xh + xl), r = rh + rl), and every rr_period outer
// iterations x is folded and r = b - A x recomputed in FP64 (residual replacement), as in the
// single-system FP32 path.
//
// The paper solves one system at a time (Section 5); batching and the autotuner over (s,
// cluster size, threads per CTA) are this library's additions.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace sstep {
namespace {

constexpr int kBWarps = 16;  // at most 512 threads per CTA

struct BSys {      // one 7-point constant-coefficient stencil system
  int nx, ny, nz, n;
  double wc, wo;   // centre weight and the (equal) neighbour weight
  double d;        // uniform M^{-1}: 1 / wc (Jacobi) or 1 (none)
  double ca, cs;   // Chebyshev scalars c_alpha, c_sigma (c_gamma = 1)
  double lmax, lmin;
};
struct BProb {     // one (system, right-hand side) problem
  const double* b;
  double* x;
  int sys, out;
};
struct BRes {
  int status, iters;
  double rr, nb2, rr_true;
};

struct BArgs {
  const BSys* sys;
  const BProb* prob;
  BRes* res;
  int nprob;
  int* queue;
  char* ws;           // one slot of slot_bytes per cluster
  size_t slot_bytes;
  int64_t ld;         // elements between the vectors of a slot
  int nu, max_outer, rr_period;
  double rtol;
  double* lam;        // power method: lambda_max per system
  int power_iters;
  double power_tol;
};

template <int S>
struct BSh {
  static constexpr int K = S * S + S;
  double wbuf[kBWarps * K];
  double part[2][K];
  double sums[K];
  double W[S * S], Bm[S * S], beta[S * S], alpha[S], rinv[S];
  float betaf[S * S];
  int prob, ok;
};

template <typename T>
__device__ __forceinline__ T fmat(T a, T b, T c) {
  if constexpr (std::is_same<T, double>::value) return fma(a, b, c);
  else return fmaf(a, b, c);
}

__device__ __forceinline__ void coords(int p, int nx, int ny, int& ix, int& iy, int& iz) {
  const int row = p / nx;
  ix = p - row * nx;
  iz = row / ny;
  iy = row - iz * ny;
}

// (A u)_p for the 7-point stencil, Dirichlet neighbours dropped; uc = u_p (own value).
// Neighbours go through L2: another CTA of the cluster may have written them.
template <typename T, typename U>
__device__ __forceinline__ T stencil7(const U* u, int p, int ix, int iy, int iz, const BSys& sy,
                                      T wc, T wo, T uc) {
  const int nx = sy.nx, nxy = sy.nx * sy.ny;
  const T xm = ix > 0 ? (T)__ldcg(u + p - 1) : T(0);
  const T xp = ix + 1 < sy.nx ? (T)__ldcg(u + p + 1) : T(0);
  const T ym = iy > 0 ? (T)__ldcg(u + p - nx) : T(0);
  const T yp = iy + 1 < sy.ny ? (T)__ldcg(u + p + nx) : T(0);
  const T zm = iz > 0 ? (T)__ldcg(u + p - nxy) : T(0);
  const T zp = iz + 1 < sy.nz ? (T)__ldcg(u + p + nxy) : T(0);
  T s = (xm + xp) + (ym + yp);
  s += zm;
  s += zp;
  return fmat<T>(wc, uc, wo * s);
}

// Cluster-wide fixed-order sum of NV values per thread; result in sh.sums (every CTA).
// WARP_DONE: lane 0 of every warp already holds its warp's totals.
template <int S, int NV, bool WARP_DONE = false>
__device__ __forceinline__ void csum(cg::cluster_group& cl, const double (&v)[NV], BSh<S>& sh,
                                     int& par) {
  static_assert(NV <= BSh<S>::K, "reduction too wide");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const double w = WARP_DONE ? v[k] : warp_sum(v[k]);
    if (lane == 0) sh.wbuf[wid * NV + k] = w;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sh.wbuf[w * NV + k];
    sh.part[par][k] = t;
  }
  __threadfence();  // this phase's global writes before the barrier (neighbours read them next)
  cl.sync();
  const int C = (int)cl.num_blocks();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double t = 0.0;
    for (int rk = 0; rk < C; ++rk) t += cl.map_shared_rank(&sh.part[par][0], rk)[k];
    sh.sums[k] = t;
  }
  par ^= 1;
  __syncthreads();
}

// Double-float per-thread sums -> FP64 cluster sums: the warp stage runs on the FP32 pipe
// (double-float shuffles), one FP64 conversion per warp.
template <int S, int NV>
__device__ __forceinline__ void csum_df(cg::cluster_group& cl, float (&hi)[NV], float (&lo)[NV],
                                        BSh<S>& sh, int& par) {
#pragma unroll
  for (int k = 0; k < NV; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, hi[k], o);
      const float ol = __shfl_xor_sync(0xffffffffu, lo[k], o);
      df_add(hi[k], lo[k], oh, ol);
    }
  }
  double v[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = (double)hi[k] + (double)lo[k];
  csum<S, NV, true>(cl, v, sh, par);
}

// Solve W X = B (nrhs columns) with nu FGS sweeps from 0 (Section 3.1), every CTA redundantly.
// Returns false on breakdown (W_ii <= 0 or a non-finite entry); uniform across the cluster.
template <int S>
__device__ bool bsolve(BSh<S>& sh, const double* B, int nrhs, int nu, double* X) {
  if (threadIdx.x == 0) {
    int ok = 1;
    for (int i = 0; i < S; ++i) {
      const double dd = sh.W[i + i * S];
      if (!(dd > 0.0) || dd > 1.79e308) ok = 0;
    }
    for (int i = 0; i < S * S; ++i)
      if (!(sh.W[i] == sh.W[i]) || fabs(sh.W[i]) > 1.79e308) ok = 0;
    if (ok)
      for (int i = 0; i < S; ++i) sh.rinv[i] = 1.0 / sh.W[i + i * S];
    sh.ok = ok;
  }
  __syncthreads();
  if (!sh.ok) return false;
  if ((int)threadIdx.x < nrhs) {
    const double* b = B + threadIdx.x * S;
    double* x = X + threadIdx.x * S;
    for (int i = 0; i < S; ++i) x[i] = 0.0;
    for (int sw = 0; sw < nu; ++sw) {
      for (int i = 0; i < S; ++i) {
        double a0 = b[i], a1 = 0.0;
        int j = 0;
        for (; j + 1 < S; j += 2) {
          if (j != i) a0 = fma(-sh.W[i + j * S], x[j], a0);
          if (j + 1 != i) a1 = fma(-sh.W[i + (j + 1) * S], x[j + 1], a1);
        }
        if (j < S && j != i) a0 = fma(-sh.W[i + j * S], x[j], a0);
        x[i] = (a0 + a1) * sh.rinv[i];
      }
    }
  }
  __syncthreads();
  return true;
}

struct Range {
  int lo, hi;
};
__device__ __forceinline__ Range my_range(int n, int C, int rank) {
  int chunk = (n + C - 1) / C;
  chunk = (chunk + 31) & ~31;
  const int lo = min(n, rank * chunk);
  return Range{lo, min(n, lo + chunk)};
}

// sum_p (b - A x)_p^2 over this CTA's points in FP64; stores r (FP64) when r != nullptr, or
// r split into FP32 (hi, lo) when rh != nullptr.  Also sum b_p^2 into v[1] when NV == 2.
template <int NV>
__device__ __forceinline__ void residual(const BSys& sy, const double* b, const double* x, double* r,
                                        float* rh, float* rl, Range rg, double (&v)[NV]) {
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  for (int p = rg.lo + threadIdx.x; p < rg.hi; p += blockDim.x) {
    int ix, iy, iz;
    coords(p, sy.nx, sy.ny, ix, iy, iz);
    const double y = stencil7<double>(x, p, ix, iy, iz, sy, sy.wc, sy.wo, __ldcg(x + p));
    const double bi = __ldg(b + p);
    const double ri = bi - y;
    if (r) r[p] = ri;
    if (rh) {
      const float h = __double2float_rn(ri);
      rh[p] = h;
      rl[p] = __double2float_rn(ri - (double)h);
    }
    v[0] = fma(ri, ri, v[0]);
    if constexpr (NV == 2) v[1] = fma(bi, bi, v[1]);
  }
}

// FP32 form: x += xh + xl in FP64 and the increments restart from 0 (own points).
__device__ __forceinline__ void fold_x(double* x, float* xh, float* xl, Range rg) {
  for (int p = rg.lo + threadIdx.x; p < rg.hi; p += blockDim.x) {
    x[p] += (double)xh[p] + (double)xl[p];
    xh[p] = 0.0f;
    xl[p] = 0.0f;
  }
}

// Algorithm 2: Z = [z_1 .. z_S], AZ = [A z_1 .. A z_S] from r, with z_1 = M^{-1} r and
// z_{q+1} = 2 c_alpha M^{-1} A z_q - 2 c_sigma z_q - z_{q-1} (first step c_alpha, c_sigma).
// A cluster barrier precedes every step after the first (neighbours of z_q).  R: the storage
// type of r (FP64, or the FP32 high part of r in the FP32 form).
template <int S, typename T, typename R>
__device__ void mpk(cg::cluster_group& cl, const BSys& sy, const R* r, T* Z, T* AZ,
                    int64_t ld, Range rg) {
  const T d = (T)sy.d, wc = (T)sy.wc, wo = (T)sy.wo;
#pragma unroll 1
  for (int q = 1; q <= S; ++q) {
    if (q > 1) {
      __threadfence();
      cl.sync();
    }
    const double c1 = q == 1 ? sy.ca : 2.0 * sy.ca;
    const T a1 = (T)(c1 * sy.d), c2 = (T)(q == 1 ? sy.cs : 2.0 * sy.cs);
    const T* u = Z + (q - 1) * ld;  // z_q (q >= 2; column q-1)
    // kU points per thread and trip, every load of the trip issued before the first store,
    // so that a thread keeps several L2 round trips in flight
    constexpr int kU = 4;
    const int bd = blockDim.x;
    for (int p0 = rg.lo + threadIdx.x; p0 < rg.hi; p0 += kU * bd) {
      T y[kU], uc[kU], zp[kU];
#pragma unroll
      for (int k = 0; k < kU; ++k) {
        const int p = p0 + k * bd;
        y[k] = uc[k] = zp[k] = T(0);
        if (p < rg.hi) {
          int ix, iy, iz;
          coords(p, sy.nx, sy.ny, ix, iy, iz);
          if (q == 1) {  // uniform M^{-1}: A (d r) = d (A r)
            uc[k] = (T)r[p];
            y[k] = stencil7<T>(r, p, ix, iy, iz, sy, wc, wo, uc[k]) * d;
            uc[k] *= d;
          } else {
            uc[k] = u[p];
            y[k] = stencil7<T>(u, p, ix, iy, iz, sy, wc, wo, uc[k]);
            if (q < S) zp[k] = Z[(q - 2) * ld + p];
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kU; ++k) {
        const int p = p0 + k * bd;
        if (p >= rg.hi) break;
        if (q == 1) Z[p] = uc[k];
        AZ[(q - 1) * ld + p] = y[k];
        if (q < S) Z[q * ld + p] = fmat<T>(a1, y[k], fmat<T>(-c2, uc[k], -zp[k]));
      }
    }
  }
}

// x and r of one problem: FP64 x and r, or (FP32 form) x = x_fp64 + (xh + xl) with the
// increments in FP32 (hi, lo) pairs and r = rh + rl, between residual replacements.
struct XR {
  double* x;
  double* r;
  float *rh, *rl, *xh, *xl;
};

// x += Q alpha, r -= AQ alpha, returns ||r||^2 (cluster sum).
template <int S, typename T>
__device__ double update_xr(cg::cluster_group& cl, BSh<S>& sh, int& par, const T* Q, const T* AQ,
                            const XR& v, int64_t ld, Range rg) {
  if constexpr (std::is_same<T, double>::value) {
    double acc[1] = {0.0};
    double al[S];
#pragma unroll
    for (int j = 0; j < S; ++j) al[j] = sh.alpha[j];
    for (int p = rg.lo + threadIdx.x; p < rg.hi; p += blockDim.x) {
      double dx = 0.0, dr = 0.0;
#pragma unroll
      for (int j = 0; j < S; ++j) {
        dx = fma(Q[j * ld + p], al[j], dx);
        dr = fma(AQ[j * ld + p], al[j], dr);
      }
      v.x[p] += dx;
      const double ri = v.r[p] - dr;
      v.r[p] = ri;
      acc[0] = fma(ri, ri, acc[0]);
    }
    csum<S, 1>(cl, acc, sh, par);
  } else {  // all on the FP32 pipe, double-float as in the single-system FP32 path
    float ah[S], al[S];
#pragma unroll
    for (int j = 0; j < S; ++j) {
      ah[j] = __double2float_rn(sh.alpha[j]);
      al[j] = __double2float_rn(sh.alpha[j] - (double)ah[j]);
    }
    float rrh[1] = {0.0f}, rrl[1] = {0.0f};
    auto point = [&](const float (&q)[S], const float (&aq)[S], float& xh, float& xl, float& rh,
                     float& rl) {
      float dxh = 0.0f, dxl = 0.0f, drh = 0.0f, drl = 0.0f;
#pragma unroll
      for (int j = 0; j < S; ++j) {
        df_acc_prod(dxh, dxl, q[j], ah[j]);
        dxl = fmaf(q[j], al[j], dxl);
        df_acc_prod(drh, drl, aq[j], ah[j]);
        drl = fmaf(aq[j], al[j], drl);
      }
      df_add(xh, xl, dxh, dxl);
      df_add(rh, rl, -drh, -drl);
      df_acc_prod(rrh[0], rrl[0], rh, rh);
      rrl[0] = fmaf(2.0f * rh, rl, rrl[0]);
    };
    // four consecutive points per thread (16-byte accesses; rg.lo and ld are multiples of 4)
    const int v0 = rg.lo >> 2, v1 = rg.hi >> 2;
    for (int vi = v0 + threadIdx.x; vi < v1; vi += blockDim.x) {
      float4 q4[S], aq4[S];
#pragma unroll
      for (int j = 0; j < S; ++j) {
        q4[j] = reinterpret_cast<const float4*>(Q + j * ld)[vi];
        aq4[j] = reinterpret_cast<const float4*>(AQ + j * ld)[vi];
      }
      float4 xh = reinterpret_cast<float4*>(v.xh)[vi], xl = reinterpret_cast<float4*>(v.xl)[vi];
      float4 rh = reinterpret_cast<float4*>(v.rh)[vi], rl = reinterpret_cast<float4*>(v.rl)[vi];
      float q[S], aq[S];
#define SSTEP_BXR_LANE(c)            \
      for (int j = 0; j < S; ++j) {  \
        q[j] = q4[j].c;              \
        aq[j] = aq4[j].c;            \
      }                              \
      point(q, aq, xh.c, xl.c, rh.c, rl.c);
      SSTEP_BXR_LANE(x)
      SSTEP_BXR_LANE(y)
      SSTEP_BXR_LANE(z)
      SSTEP_BXR_LANE(w)
#undef SSTEP_BXR_LANE
      reinterpret_cast<float4*>(v.xh)[vi] = xh;
      reinterpret_cast<float4*>(v.xl)[vi] = xl;
      reinterpret_cast<float4*>(v.rh)[vi] = rh;
      reinterpret_cast<float4*>(v.rl)[vi] = rl;
    }
    for (int p = 4 * v1 + threadIdx.x; p < rg.hi; p += blockDim.x) {  // the last n mod 4 points
      float q[S], aq[S];
#pragma unroll
      for (int j = 0; j < S; ++j) {
        q[j] = Q[j * ld + p];
        aq[j] = AQ[j * ld + p];
      }
      float xh = v.xh[p], xl = v.xl[p], rh = v.rh[p], rl = v.rl[p];
      point(q, aq, xh, xl, rh, rl);
      v.xh[p] = xh;
      v.xl[p] = xl;
      v.rh[p] = rh;
      v.rl[p] = rl;
    }
    csum_df<S, 1>(cl, rrh, rrl, sh, par);
  }
  return sh.sums[0];
}

// Conjugation: b2 = -Q^T AZ, beta = FGS(W, b2).  False on breakdown.
template <int S, typename T>
__device__ bool b2_beta(cg::cluster_group& cl, BSh<S>& sh, int& par, const T* Q, const T* AZ,
                        int nu, int64_t ld, Range rg) {
  constexpr int K = S * S;
  if constexpr (std::is_same<T, double>::value) {
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int p = rg.lo + threadIdx.x; p < rg.hi; p += blockDim.x) {
      double q[S], z[S];
#pragma unroll
      for (int i = 0; i < S; ++i) q[i] = Q[i * ld + p];
#pragma unroll
      for (int j = 0; j < S; ++j) z[j] = AZ[j * ld + p];
#pragma unroll
      for (int i = 0; i < S; ++i)
#pragma unroll
        for (int j = 0; j < S; ++j) acc[i + j * S] = fma(q[i], z[j], acc[i + j * S]);
    }
    csum<S, K>(cl, acc, sh, par);
  } else {
    float hi[K], lo[K];
#pragma unroll
    for (int k = 0; k < K; ++k) hi[k] = lo[k] = 0.0f;
    // the MPK wrote AZ with another point-to-thread map: make its writes visible in the CTA
    __syncthreads();
    const int v0 = rg.lo >> 2, v1 = rg.hi >> 2;
    for (int vi = v0 + threadIdx.x; vi < v1; vi += blockDim.x) {  // four points per thread
      float4 q4[S], z4[S];
#pragma unroll
      for (int i = 0; i < S; ++i) q4[i] = reinterpret_cast<const float4*>(Q + i * ld)[vi];
#pragma unroll
      for (int j = 0; j < S; ++j) z4[j] = reinterpret_cast<const float4*>(AZ + j * ld)[vi];
#pragma unroll
      for (int i = 0; i < S; ++i)
#pragma unroll
        for (int j = 0; j < S; ++j) {
          df_acc_prod(hi[i + j * S], lo[i + j * S], q4[i].x, z4[j].x);
          df_acc_prod(hi[i + j * S], lo[i + j * S], q4[i].y, z4[j].y);
          df_acc_prod(hi[i + j * S], lo[i + j * S], q4[i].z, z4[j].z);
          df_acc_prod(hi[i + j * S], lo[i + j * S], q4[i].w, z4[j].w);
        }
    }
    for (int p = 4 * v1 + threadIdx.x; p < rg.hi; p += blockDim.x) {
      float q[S], z[S];
#pragma unroll
      for (int i = 0; i < S; ++i) q[i] = Q[i * ld + p];
#pragma unroll
      for (int j = 0; j < S; ++j) z[j] = AZ[j * ld + p];
#pragma unroll
      for (int i = 0; i < S; ++i)
#pragma unroll
        for (int j = 0; j < S; ++j) df_acc_prod(hi[i + j * S], lo[i + j * S], q[i], z[j]);
    }
    csum_df<S, K>(cl, hi, lo, sh, par);
  }
  for (int e = threadIdx.x; e < K; e += blockDim.x) sh.Bm[e] = -sh.sums[e];
  __syncthreads();
  if (!bsolve<S>(sh, sh.Bm, S, nu, sh.beta)) return false;
  for (int e = threadIdx.x; e < K; e += blockDim.x) sh.betaf[e] = (float)sh.beta[e];
  __syncthreads();
  return true;
}

// Direction-block update (Q = Z + Q beta, AQ = AZ + AQ beta, written over Z, AZ; FIRST: Q = Z
// as is) fused with the step system (W = Q^T AQ, b1 = Q^T r, alpha = FGS(W, b1)).  False on
// breakdown.
template <int S, typename T, bool FIRST>
__device__ bool upd_gram(cg::cluster_group& cl, BSh<S>& sh, int& par, T* Zn, T* AZn, const T* Qo,
                         const T* AQo, const XR& v, int nu, int64_t ld, Range rg) {
  constexpr int K = S * S + S;
  if constexpr (std::is_same<T, double>::value) {
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (int p = rg.lo + threadIdx.x; p < rg.hi; p += blockDim.x) {
      double qn[S], an[S];
      if constexpr (FIRST) {
#pragma unroll
        for (int j = 0; j < S; ++j) {
          qn[j] = Zn[j * ld + p];
          an[j] = AZn[j * ld + p];
        }
      } else {
        double qo[S], ao[S];
#pragma unroll
        for (int l = 0; l < S; ++l) {
          qo[l] = Qo[l * ld + p];
          ao[l] = AQo[l * ld + p];
        }
#pragma unroll
        for (int j = 0; j < S; ++j) {
          double vq = Zn[j * ld + p], va = AZn[j * ld + p];
#pragma unroll
          for (int l = 0; l < S; ++l) {
            vq = fma(qo[l], sh.beta[l + j * S], vq);
            va = fma(ao[l], sh.beta[l + j * S], va);
          }
          qn[j] = vq;
          an[j] = va;
          Zn[j * ld + p] = vq;
          AZn[j * ld + p] = va;
        }
      }
      const double rp = v.r[p];
#pragma unroll
      for (int i = 0; i < S; ++i) {
#pragma unroll
        for (int j = 0; j < S; ++j) acc[i + j * S] = fma(qn[i], an[j], acc[i + j * S]);
        acc[S * S + i] = fma(qn[i], rp, acc[S * S + i]);
      }
    }
    csum<S, K>(cl, acc, sh, par);
  } else {
    float hi[K], lo[K];
#pragma unroll
    for (int k = 0; k < K; ++k) hi[k] = lo[k] = 0.0f;
    auto accum = [&](const float (&qn)[S], const float (&an)[S], float rh, float rl) {
#pragma unroll
      for (int i = 0; i < S; ++i) {
#pragma unroll
        for (int j = 0; j < S; ++j) df_acc_prod(hi[i + j * S], lo[i + j * S], qn[i], an[j]);
        df_acc_prod(hi[S * S + i], lo[S * S + i], qn[i], rh);
        lo[S * S + i] = fmaf(qn[i], rl, lo[S * S + i]);
      }
    };
    // the MPK wrote Z, AZ with another point-to-thread map: make its writes visible in the CTA
    __syncthreads();
    const int v0 = rg.lo >> 2, v1 = rg.hi >> 2;
    for (int vi = v0 + threadIdx.x; vi < v1; vi += blockDim.x) {  // four points per thread
      float4 qn4[S], an4[S];
      if constexpr (FIRST) {
#pragma unroll
        for (int j = 0; j < S; ++j) {
          qn4[j] = reinterpret_cast<const float4*>(Zn + j * ld)[vi];
          an4[j] = reinterpret_cast<const float4*>(AZn + j * ld)[vi];
        }
      } else {
        float4 qo4[S], ao4[S];
#pragma unroll
        for (int l = 0; l < S; ++l) {
          qo4[l] = reinterpret_cast<const float4*>(Qo + l * ld)[vi];
          ao4[l] = reinterpret_cast<const float4*>(AQo + l * ld)[vi];
        }
#pragma unroll
        for (int j = 0; j < S; ++j) {
          float4 vq = reinterpret_cast<const float4*>(Zn + j * ld)[vi];
          float4 va = reinterpret_cast<const float4*>(AZn + j * ld)[vi];
#pragma unroll
          for (int l = 0; l < S; ++l) {
            const float bl = sh.betaf[l + j * S];
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
          reinterpret_cast<float4*>(Zn + j * ld)[vi] = vq;
          reinterpret_cast<float4*>(AZn + j * ld)[vi] = va;
        }
      }
      const float4 rh4 = reinterpret_cast<const float4*>(v.rh)[vi];
      const float4 rl4 = reinterpret_cast<const float4*>(v.rl)[vi];
      float qn[S], an[S];
#define SSTEP_BUG_LANE(c)            \
      for (int j = 0; j < S; ++j) {  \
        qn[j] = qn4[j].c;            \
        an[j] = an4[j].c;            \
      }                              \
      accum(qn, an, rh4.c, rl4.c);
      SSTEP_BUG_LANE(x)
      SSTEP_BUG_LANE(y)
      SSTEP_BUG_LANE(z)
      SSTEP_BUG_LANE(w)
#undef SSTEP_BUG_LANE
    }
    for (int p = 4 * v1 + threadIdx.x; p < rg.hi; p += blockDim.x) {  // the last n mod 4 points
      float qn[S], an[S];
      if constexpr (FIRST) {
#pragma unroll
        for (int j = 0; j < S; ++j) {
          qn[j] = Zn[j * ld + p];
          an[j] = AZn[j * ld + p];
        }
      } else {
        float qo[S], ao[S];
#pragma unroll
        for (int l = 0; l < S; ++l) {
          qo[l] = Qo[l * ld + p];
          ao[l] = AQo[l * ld + p];
        }
#pragma unroll
        for (int j = 0; j < S; ++j) {
          float vq = Zn[j * ld + p], va = AZn[j * ld + p];
#pragma unroll
          for (int l = 0; l < S; ++l) {
            vq = fmaf(qo[l], sh.betaf[l + j * S], vq);
            va = fmaf(ao[l], sh.betaf[l + j * S], va);
          }
          qn[j] = vq;
          an[j] = va;
          Zn[j * ld + p] = vq;
          AZn[j * ld + p] = va;
        }
      }
      accum(qn, an, v.rh[p], v.rl[p]);
    }
    csum_df<S, K>(cl, hi, lo, sh, par);
  }
  for (int e = threadIdx.x; e < S * S; e += blockDim.x) sh.W[e] = sh.sums[e];
  for (int i = threadIdx.x; i < S; i += blockDim.x) sh.Bm[i] = sh.sums[S * S + i];
  __syncthreads();
  return bsolve<S>(sh, sh.Bm, 1, nu, sh.alpha);
}

__device__ __forceinline__ int stop_rule(double rr, double tol2, int iters, int max_outer) {
  if (!(rr == rr) || rr > 1.79e308) return SSTEP_ERR_NONFINITE;
  if (rr <= tol2) return SSTEP_OK;
  if (iters >= max_outer) return SSTEP_NOT_CONVERGED;
  return -1;
}

// One problem, start to finish, by the whole cluster.
template <int S, typename T>
__device__ void solve_one(const BArgs& a, cg::cluster_group& cl, BSh<S>& sh, int& par, int pi,
                          char* slot) {
  const BProb pr = a.prob[pi];
  const BSys sy = a.sys[pr.sys];
  const Range rg = my_range(sy.n, (int)cl.num_blocks(), (int)cl.block_rank());
  const int64_t ld = a.ld;
  constexpr bool kMixed = std::is_same<T, float>::value;
  // slot: FP64 form [r | blocks]; FP32 form [rh | rl | xh | xl | blocks]
  XR v{pr.x, nullptr, nullptr, nullptr, nullptr, nullptr};
  T* blk;
  if constexpr (kMixed) {
    v.rh = (float*)slot;
    v.rl = v.rh + ld;
    v.xh = v.rl + ld;
    v.xl = v.xh + ld;
    blk = (T*)(v.xl + ld);
  } else {
    v.r = (double*)slot;
    blk = (T*)(v.r + ld);
  }
  // pair k of blocks: Z = blk + 2kS ld, AZ = blk + (2k+1) S ld
  auto Zp = [&](int k) { return blk + (size_t)(2 * k) * S * ld; };
  auto AZp = [&](int k) { return blk + (size_t)(2 * k + 1) * S * ld; };
  auto run_mpk = [&](T* Z, T* AZ) {
    if constexpr (kMixed) mpk<S, T, float>(cl, sy, v.rh, Z, AZ, ld, rg);
    else mpk<S, T, double>(cl, sy, v.r, Z, AZ, ld, rg);
  };
  auto barrier = [&]() {
    __threadfence();
    cl.sync();
  };

  // ---- initial residual r = b - A x0; ||b||^2
  double v2[2];
  residual<2>(sy, pr.b, pr.x, v.r, v.rh, v.rl, rg, v2);
  if constexpr (kMixed)
    for (int p = rg.lo + threadIdx.x; p < rg.hi; p += blockDim.x) v.xh[p] = v.xl[p] = 0.0f;
  csum<S, 2>(cl, v2, sh, par);
  double rr = sh.sums[0];
  const double nb2 = sh.sums[1];
  const double tol2 = a.rtol * a.rtol * nb2;
  int status = -1, iters = 0;
  if (!(rr == rr) || rr > 1.79e308 || !(nb2 == nb2) || nb2 > 1.79e308) {
    status = SSTEP_ERR_NONFINITE;
  } else if (nb2 == 0.0) {  // b = 0: x = 0, no iteration
    for (int p = rg.lo + threadIdx.x; p < rg.hi; p += blockDim.x) pr.x[p] = 0.0;
    rr = 0.0;
    status = SSTEP_OK;
  } else if (rr <= tol2) {
    status = SSTEP_OK;
  }
  if (status < 0) {
    int qp = 0;  // the pair holding Q, AQ
    run_mpk(Zp(0), AZp(0));
    // k = 0: Q_0 = Z_0, W, b1, alpha
    if (!upd_gram<S, T, true>(cl, sh, par, Zp(0), AZp(0), nullptr, nullptr, v, a.nu, ld, rg))
      status = SSTEP_ERR_BREAKDOWN;
    while (status < 0) {
      rr = update_xr<S, T>(cl, sh, par, Zp(qp), AZp(qp), v, ld, rg);  // x/r update
      ++iters;
      status = stop_rule(rr, tol2, iters, a.max_outer);               // stop test
      if constexpr (kMixed) {
        if (status < 0 && iters % a.rr_period == 0) {
          // residual replacement: x folded to FP64, then r = b - A x in FP64
          fold_x(pr.x, v.xh, v.xl, rg);
          barrier();
          double v1[1];
          residual<1>(sy, pr.b, pr.x, nullptr, v.rh, v.rl, rg, v1);
          csum<S, 1>(cl, v1, sh, par);
          rr = sh.sums[0];
          if (!(rr == rr) || rr > 1.79e308) status = SSTEP_ERR_NONFINITE;
          else if (rr <= tol2) status = SSTEP_OK;
        }
      }
      if (status >= 0) break;
      const int zp = qp ^ 1;
      run_mpk(Zp(zp), AZp(zp));                                         // basis of r
      if (!b2_beta<S, T>(cl, sh, par, Zp(qp), AZp(zp), a.nu, ld, rg)) {  // conjugation
        status = SSTEP_ERR_BREAKDOWN;
        break;
      }
      // direction update, then the step system of the next iteration
      if (!upd_gram<S, T, false>(cl, sh, par, Zp(zp), AZp(zp), Zp(qp), AZp(qp), v, a.nu, ld, rg)) {
        status = SSTEP_ERR_BREAKDOWN;
        break;
      }
      qp = zp;
    }
  }
  if constexpr (kMixed) {
    fold_x(pr.x, v.xh, v.xl, rg);
    barrier();
  }
  // true residual at exit (x's neighbours were written before the last barrier)
  double rt = rr;
  if (nb2 > 0.0 && status != SSTEP_ERR_NONFINITE) {
    double v1[1];
    residual<1>(sy, pr.b, pr.x, nullptr, nullptr, nullptr, rg, v1);
    csum<S, 1>(cl, v1, sh, par);
    rt = sh.sums[0];
  }
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    BRes o;
    o.status = status;
    o.iters = iters;
    o.rr = rr;
    o.nb2 = nb2;
    o.rr_true = rt;
    a.res[pr.out] = o;
  }
}

// Persistent kernel: clusters take problems from the queue until it is empty.
template <int S, typename T, int NT>
__global__ void __launch_bounds__(NT, 1) k_batch_solve(BArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ BSh<S> sh;
  const int C = (int)cl.num_blocks();
  const int slot = (int)(blockIdx.x / C);
  char* ws = a.ws + (size_t)slot * a.slot_bytes;
  int par = 0;
  for (;;) {
    if (cl.block_rank() == 0 && threadIdx.x == 0) sh.prob = atomicAdd(a.queue, 1);
    cl.sync();
    const int pi = *cl.map_shared_rank(&sh.prob, 0);
    cl.sync();  // nobody leaves (or overwrites sh.prob) before every CTA has read it
    if (pi >= a.nprob) break;
    solve_one<S, T>(a, cl, sh, par, pi, ws);
  }
}

// Section 2 power method on M^{-1} A per system: lambda^(l) = ||M^{-1} A v_(l-1)|| with
// ||v_(l-1)|| = 1, v_0 = U[-1,1) from SplitMix64 seed 1; stop when the relative change is
// below power_tol or after power_iters estimates.  Problems of the queue are systems here.
__global__ void __launch_bounds__(256, 1) k_batch_power(BArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ BSh<2> sh;
  const int C = (int)cl.num_blocks();
  const int slot = (int)(blockIdx.x / C);
  double* bufs[2] = {(double*)(a.ws + (size_t)slot * a.slot_bytes),
                     (double*)(a.ws + (size_t)slot * a.slot_bytes) + a.ld};
  int par = 0;
  for (;;) {
    if (cl.block_rank() == 0 && threadIdx.x == 0) sh.prob = atomicAdd(a.queue, 1);
    cl.sync();
    const int si = *cl.map_shared_rank(&sh.prob, 0);
    cl.sync();
    if (si >= a.nprob) break;
    const BSys sy = a.sys[si];
    const Range rg = my_range(sy.n, C, (int)cl.block_rank());
    double* v = bufs[0];
    double* y = bufs[1];
    double w[1] = {0.0};
    for (int p = rg.lo + threadIdx.x; p < rg.hi; p += blockDim.x) {
      const double e = splitmix_pm1(1ull, p);
      v[p] = e;
      w[0] = fma(e, e, w[0]);
    }
    csum<2, 1>(cl, w, sh, par);
    double inv = sh.sums[0] > 0.0 ? 1.0 / sqrt(sh.sums[0]) : 0.0;
    double lam = 0.0;
    for (int it = 0; it < a.power_iters; ++it) {
      w[0] = 0.0;
      for (int p = rg.lo + threadIdx.x; p < rg.hi; p += blockDim.x) {
        int ix, iy, iz;
        coords(p, sy.nx, sy.ny, ix, iy, iz);
        const double av = stencil7<double>(v, p, ix, iy, iz, sy, sy.wc, sy.wo, __ldcg(v + p));
        const double yi = inv * sy.d * av;
        y[p] = yi;
        w[0] = fma(yi, yi, w[0]);
      }
      csum<2, 1>(cl, w, sh, par);
      const double ln = sqrt(sh.sums[0]);
      const bool conv = it > 0 && a.power_tol > 0.0 && fabs(ln - lam) < a.power_tol * fabs(ln);
      lam = ln;
      inv = lam > 0.0 ? 1.0 / lam : 0.0;
      double* t = v;
      v = y;
      y = t;
      if (conv || !(lam > 0.0)) break;
    }
    if (cl.block_rank() == 0 && threadIdx.x == 0) a.lam[si] = lam;
  }
}

__global__ void k_fill_rhs(double* v, int64_t n, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] = splitmix_pm1(seed, i);
}

// ---------------------------------------------------------------- host side

using KernelFn = void (*)(BArgs);

template <int S, typename T>
KernelFn pick_nt(int nt) {
  if (nt == 256) return k_batch_solve<S, T, 256>;
  if constexpr (S <= 4)
    if (nt == 512) return k_batch_solve<S, T, 512>;
  return nullptr;
}

KernelFn pick_kernel(int s, bool mixed, int nt) {
  switch (s) {
    case 2: return mixed ? pick_nt<2, float>(nt) : pick_nt<2, double>(nt);
    case 4: return mixed ? pick_nt<4, float>(nt) : pick_nt<4, double>(nt);
    case 8: return mixed ? pick_nt<8, float>(nt) : pick_nt<8, double>(nt);
    default: return nullptr;
  }
}

double wall_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Choice {
  int s = 0, cluster = 0, threads = 0;
};

std::mutex g_tune_mu;
std::map<std::string, Choice> g_tune;  // in-process autotuner cache

}  // namespace

struct BatchCtx {
  int nsys = 0;
  std::vector<BSys> hsys;
  BSys* dsys = nullptr;
  bool mixed = false;
  int s = 0, nu = 2, max_outer = 10000, rr_period = 0, rr_opt = 0, cluster = 0, threads = 0;
  int nslots = 0;
  double rtol = 1e-8;
  int64_t ld = 0;
  size_t slot_bytes = 0;
  char* ws = nullptr;
  int* queue = nullptr;
  BProb* dprob = nullptr;
  BRes* dres = nullptr;
  BProb* hprob = nullptr;  // pinned
  BRes* hres = nullptr;    // pinned
  int cap = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  cudaGraphExec_t gexec = nullptr;
  int graph_nprob = -1;
  double ms_setup = 0.0, tune_ms = 0.0;
};

namespace {

sstep_status bfail(sstep_status st, const std::string& msg) {
  set_last_error(msg.c_str());
  return st;
}

#define BCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return bfail(e_ == cudaErrorMemoryAllocation ? SSTEP_ERR_OOM : SSTEP_ERR_CUDA,           \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

size_t slot_bytes_for(int s, bool mixed, int64_t ld) {
  // FP64 form: r and 4s basis vectors; FP32 form: rh, rl, xh, xl and 4s basis vectors
  const size_t el = mixed ? sizeof(float) : sizeof(double);
  size_t b = (mixed ? 4 * sizeof(float) : sizeof(double)) * (size_t)ld +
             el * (size_t)(4 * s) * (size_t)ld;
  b = std::max(b, sizeof(double) * 2 * (size_t)ld);  // power method: two FP64 vectors
  return (b + 255) / 256 * 256;
}

cudaLaunchConfig_t launch_cfg(int nclusters, int C, int NT, cudaStream_t st,
                              cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nclusters * C), 1, 1);
  cfg.blockDim = dim3((unsigned)NT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Clusters of C CTAs of NT threads that fit on the device at once (0: none).
int max_clusters(KernelFn fn, int C, int NT) {
  if (C > 8 && cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                    1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = launch_cfg(1, C, NT, nullptr, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, (const void*)fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch(KernelFn fn, int nclusters, int C, int NT, const BArgs& a, cudaStream_t st) {
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = launch_cfg(nclusters, C, NT, st, attr);
  return cudaLaunchKernelEx(&cfg, fn, a);
}

BArgs base_args(const BatchCtx* b) {
  BArgs a{};
  a.sys = b->dsys;
  a.queue = b->queue;
  a.ld = b->ld;
  a.nu = b->nu;
  a.max_outer = b->max_outer;
  a.rr_period = b->rr_period;
  a.rtol = b->rtol;
  return a;
}

// Order of the problems: largest systems first (longest-processing-time first).
std::vector<int> sys_order(const BatchCtx* b) {
  std::vector<int> ord(b->nsys);
  for (int i = 0; i < b->nsys; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(),
                   [&](int x, int y) { return b->hsys[x].n > b->hsys[y].n; });
  return ord;
}

// Time one configuration on a trial batch of nrhs seeded right-hand sides per system, x0 = 0:
// to convergence with the handle's own rtol and cap (fixed_outer = 0), or for exactly
// fixed_outer outer iterations (rtol 0).
sstep_status trial(BatchCtx* b, int s, int C, int NT, int nrhs, int fixed_outer, double* ms_out) {
  *ms_out = -1.0;
  KernelFn fn = pick_kernel(s, b->mixed, NT);
  if (!fn) return SSTEP_OK;
  const int nc = max_clusters(fn, C, NT);
  if (nc < 1) return SSTEP_OK;
  int64_t total = 0;
  for (const BSys& y : b->hsys) total += y.n;
  const int nprob = b->nsys * nrhs;
  const int ncl = std::min(nc, nprob);
  const size_t sb = slot_bytes_for(s, b->mixed, b->ld);
  char* ws = nullptr;
  double *bv = nullptr, *xv = nullptr;
  BProb* dp = nullptr;
  BRes* dr = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  sstep_status st = SSTEP_OK;
  auto cleanup = [&]() {
    cudaStreamSynchronize(b->st);
    if (ws) cudaFree(ws);
    if (bv) cudaFree(bv);
    if (xv) cudaFree(xv);
    if (dp) cudaFree(dp);
    if (dr) cudaFree(dr);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
  do {
    cudaError_t e;
    if ((e = cudaMalloc((void**)&ws, sb * (size_t)ncl)) != cudaSuccess ||
        (e = cudaMalloc((void**)&bv, sizeof(double) * (size_t)total * nrhs)) != cudaSuccess ||
        (e = cudaMalloc((void**)&xv, sizeof(double) * (size_t)total * nrhs)) != cudaSuccess ||
        (e = cudaMalloc((void**)&dp, sizeof(BProb) * nprob)) != cudaSuccess ||
        (e = cudaMalloc((void**)&dr, sizeof(BRes) * nprob)) != cudaSuccess) {
      cudaGetLastError();
      st = SSTEP_OK;  // too large for this configuration: skip it
      break;
    }
    std::vector<BProb> hp;
    std::vector<int64_t> off(b->nsys);
    int64_t o = 0;
    for (int i = 0; i < b->nsys; ++i) {
      off[i] = o;
      o += b->hsys[i].n;
    }
    for (int i : sys_order(b))
      for (int j = 0; j < nrhs; ++j) {
        const int64_t base = (int64_t)j * total + off[i];
        hp.push_back(BProb{bv + base, xv + base, i, (int)hp.size()});
      }
    k_fill_rhs<<<1024, 256, 0, b->st>>>(bv, total * nrhs, 7ull);
    if ((e = cudaGetLastError()) != cudaSuccess) { st = bfail(SSTEP_ERR_CUDA, cudaGetErrorString(e)); break; }
    if ((e = cudaMemcpyAsync(dp, hp.data(), sizeof(BProb) * nprob, cudaMemcpyHostToDevice, b->st)) != cudaSuccess ||
        (e = cudaMemsetAsync(xv, 0, sizeof(double) * (size_t)total * nrhs, b->st)) != cudaSuccess ||
        (e = cudaMemsetAsync(b->queue, 0, sizeof(int), b->st)) != cudaSuccess ||
        (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
      st = bfail(SSTEP_ERR_CUDA, cudaGetErrorString(e));
      break;
    }
    BArgs a = base_args(b);
    a.rr_period = b->rr_opt > 0 ? b->rr_opt : s;
    if (fixed_outer > 0) {
      a.rtol = 0.0;
      a.max_outer = fixed_outer;
    }
    a.prob = dp;
    a.res = dr;
    a.nprob = nprob;
    a.ws = ws;
    a.slot_bytes = sb;
    cudaEventRecord(e0, b->st);
    if ((e = launch(fn, ncl, C, NT, a, b->st)) != cudaSuccess) {
      cudaGetLastError();
      break;  // not launchable: skip
    }
    cudaEventRecord(e1, b->st);
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
      st = bfail(SSTEP_ERR_CUDA, cudaGetErrorString(e));
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_out = ms;
  } while (0);
  cleanup();
  return st;
}

std::string tune_key(const BatchCtx* b, int s_fixed, int c_fixed, int t_fixed) {
  char head[160];
  snprintf(head, sizeof(head), "%s|nu%d|rtol%.17g|max%d|s%d|c%d|t%d|rr%d", b->mixed ? "fp32rr" : "fp64",
           b->nu, b->rtol, b->max_outer, s_fixed, c_fixed, t_fixed, b->rr_opt);
  std::string k = head;
  for (const BSys& y : b->hsys) {  // weights and interval enter the iteration counts
    char w[96];
    snprintf(w, sizeof(w), "|%.17g,%.17g,%.17g", y.wc, y.wo, y.lmax);
    k += w;
  }
  std::vector<int> ns;
  for (const BSys& y : b->hsys) ns.push_back(y.nx * 1000000 + y.ny * 1000 + y.nz);
  std::sort(ns.begin(), ns.end());
  for (int v : ns) k += "," + std::to_string(v);
  return k;
}

sstep_status autotune(BatchCtx* b, int s_fixed, int c_fixed, int t_fixed) {
  const std::string key = tune_key(b, s_fixed, c_fixed, t_fixed);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      b->s = it->second.s;
      b->cluster = it->second.cluster;
      b->threads = it->second.threads;
      return SSTEP_OK;
    }
  }
  const double t0 = wall_ms();
  // Two stages.  (1) The step size, at one launch shape, timed to convergence on one
  // right-hand side per system (s decides the iteration counts).  (2) The launch shape (CTAs
  // per cluster, threads per CTA) at that step size, timed over a fixed number of outer
  // iterations on enough problems to fill every candidate's resident clusters a few times
  // (the shape decides how the problems spread over the SMs, not the iteration counts).
  double best = -1.0;
  Choice ch;
  const int c0 = c_fixed ? c_fixed : 4, t0s = t_fixed ? t_fixed : 256;
  int s1 = s_fixed;
  if (!s_fixed) {
    double b1 = -1.0;
    for (int s : {2, 4, 8}) {
      double ms;
      sstep_status st = trial(b, s, c0, t0s, 1, 0, &ms);
      if (st != SSTEP_OK) return st;
      if (ms > 0.0 && (b1 < 0.0 || ms < b1)) {
        b1 = ms;
        s1 = s;
      }
    }
    if (b1 < 0.0) return bfail(SSTEP_ERR_UNSUPPORTED, "no launchable batched configuration");
  }
  std::vector<int> cs = c_fixed ? std::vector<int>{c_fixed} : std::vector<int>{2, 4, 8, 16};
  std::vector<int> ts = t_fixed ? std::vector<int>{t_fixed} : std::vector<int>{256, 512};
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  const int want = std::max(b->nsys, 2 * std::max(nsm, 1));  // ~4x the resident clusters of C = 2
  const int nrhs2 = std::min(8, (want + b->nsys - 1) / b->nsys);
  if (cs.size() * ts.size() == 1) {
    ch = Choice{s1, cs[0], ts[0]};
    best = 1.0;
  } else {
    for (int c : cs)
      for (int t : ts) {
        double ms;
        sstep_status st = trial(b, s1, c, t, nrhs2, 8, &ms);
        if (st != SSTEP_OK) return st;
        if (ms > 0.0 && (best < 0.0 || ms < best)) {
          best = ms;
          ch = Choice{s1, c, t};
        }
      }
  }
  if (best < 0.0) return bfail(SSTEP_ERR_UNSUPPORTED, "no launchable batched configuration");
  b->s = ch.s;
  b->cluster = ch.cluster;
  b->threads = ch.threads;
  b->tune_ms = wall_ms() - t0;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = ch;
  return SSTEP_OK;
}

sstep_status power_all(BatchCtx* b, const sstep_opts* o) {
  std::vector<double> lam(b->nsys, 0.0);
  if (o->lambda_max > 0.0) {
    for (auto& v : lam) v = o->lambda_max;
  } else {
    const int C = 4;
    const int nc = std::max(1, std::min(max_clusters(k_batch_power, C, 256), b->nsys));
    if (max_clusters(k_batch_power, C, 256) < 1)
      return bfail(SSTEP_ERR_UNSUPPORTED, "power-method kernel cannot be launched");
    const size_t sb = slot_bytes_for(1, false, b->ld);
    char* ws = nullptr;
    double* dlam = nullptr;
    BCK(cudaMalloc((void**)&ws, sb * (size_t)nc));
    cudaError_t e = cudaMalloc((void**)&dlam, sizeof(double) * b->nsys);
    if (e != cudaSuccess) {
      cudaFree(ws);
      return bfail(SSTEP_ERR_OOM, "power-method buffers");
    }
    BArgs a = base_args(b);
    a.nprob = b->nsys;
    a.ws = ws;
    a.slot_bytes = sb;
    a.lam = dlam;
    a.power_iters = o->power_iters;
    a.power_tol = o->power_tol;
    e = cudaMemsetAsync(b->queue, 0, sizeof(int), b->st);
    if (e == cudaSuccess) e = launch(k_batch_power, nc, C, 256, a, b->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(lam.data(), dlam, sizeof(double) * b->nsys, cudaMemcpyDeviceToHost, b->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    cudaFree(ws);
    cudaFree(dlam);
    if (e != cudaSuccess) return bfail(SSTEP_ERR_CUDA, std::string("power method: ") + cudaGetErrorString(e));
  }
  for (int i = 0; i < b->nsys; ++i) {
    BSys& y = b->hsys[i];
    y.lmax = lam[i];
    if (!(y.lmax > y.lmin) || y.lmax != y.lmax)
      return bfail(SSTEP_ERR_INVALID, "lambda_max must exceed lambda_min (system " + std::to_string(i) + ")");
    y.ca = 2.0 / (y.lmax - y.lmin);
    y.cs = (y.lmax + y.lmin) / (y.lmax - y.lmin);
  }
  return SSTEP_OK;
}

sstep_status ensure_capacity(BatchCtx* b, int nprob) {
  if (nprob <= b->cap) return SSTEP_OK;
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->graph_nprob = -1;
  }
  cudaStreamSynchronize(b->st);
  if (b->dprob) cudaFree(b->dprob);
  if (b->dres) cudaFree(b->dres);
  if (b->hprob) cudaFreeHost(b->hprob);
  if (b->hres) cudaFreeHost(b->hres);
  b->dprob = nullptr;
  b->dres = nullptr;
  b->hprob = nullptr;
  b->hres = nullptr;
  b->cap = 0;
  BCK(cudaMalloc((void**)&b->dprob, sizeof(BProb) * nprob));
  BCK(cudaMalloc((void**)&b->dres, sizeof(BRes) * nprob));
  BCK(cudaMallocHost((void**)&b->hprob, sizeof(BProb) * nprob));
  BCK(cudaMallocHost((void**)&b->hres, sizeof(BRes) * nprob));
  b->cap = nprob;
  return SSTEP_OK;
}

// The CUDA graph of one batched solve: problem table in, queue reset, the persistent kernel,
// results out.
sstep_status ensure_graph(BatchCtx* b, int nprob) {
  if (b->gexec && b->graph_nprob == nprob) return SSTEP_OK;
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  KernelFn fn = pick_kernel(b->s, b->mixed, b->threads);
  BArgs a = base_args(b);
  a.prob = b->dprob;
  a.res = b->dres;
  a.nprob = nprob;
  a.ws = b->ws;
  a.slot_bytes = b->slot_bytes;
  const int ncl = std::min(b->nslots, nprob);
  cudaGraph_t g = nullptr;
  BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemcpyAsync(b->dprob, b->hprob, sizeof(BProb) * nprob, cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->queue, 0, sizeof(int), b->st);
  if (e == cudaSuccess) e = launch(fn, ncl, b->cluster, b->threads, a, b->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->hres, b->dres, sizeof(BRes) * nprob, cudaMemcpyDeviceToHost, b->st);
  cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return bfail(SSTEP_ERR_CUDA, std::string("batched graph capture: ") +
                                     cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&b->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->gexec = nullptr;
    return bfail(SSTEP_ERR_CUDA, std::string("batched graph instantiate: ") + cudaGetErrorString(e));
  }
  b->graph_nprob = nprob;
  return SSTEP_OK;
}

sstep_status setup_body(BatchCtx* b, const sstep_matrix* A, int nsys, const sstep_precond* M,
                        const sstep_opts* o) {
  if (o->algo != SSTEP_ALGO_LITERAL)
    return bfail(SSTEP_ERR_UNSUPPORTED, "the batched solver implements the literal form only");
  if (o->gram_solver != SSTEP_GRAM_FGS)
    return bfail(SSTEP_ERR_UNSUPPORTED, "the batched solver uses FGS reduced solves only");
  if (!(o->s == 0 || o->s == 2 || o->s == 4 || o->s == 8))
    return bfail(SSTEP_ERR_UNSUPPORTED, "batched s must be 0 (autotune), 2, 4 or 8");
  if (o->sweeps < 1 || o->sweeps > 1000) return bfail(SSTEP_ERR_INVALID, "sweeps must be in 1..1000");
  if (!(o->rtol >= 0.0)) return bfail(SSTEP_ERR_INVALID, "rtol must be >= 0");
  if (o->max_outer < 1) return bfail(SSTEP_ERR_INVALID, "max_outer must be >= 1");
  if (o->precision != SSTEP_PRECISION_FP64 && o->precision != SSTEP_PRECISION_FP32_RR)
    return bfail(SSTEP_ERR_INVALID, "unknown precision");
  if (!(o->cluster == 0 || o->cluster == 1 || o->cluster == 2 || o->cluster == 4 ||
        o->cluster == 8 || o->cluster == 16))
    return bfail(SSTEP_ERR_INVALID, "cluster must be 0, 1, 2, 4, 8 or 16");
  if (!(o->block_threads == 0 || o->block_threads == 256 || o->block_threads == 512))
    return bfail(SSTEP_ERR_INVALID, "block_threads must be 0, 256 or 512");
  if (o->block_threads == 512 && o->s == 8)
    return bfail(SSTEP_ERR_UNSUPPORTED, "512 threads per CTA need s <= 4");
  if (o->power_iters < 1 && !(o->lambda_max > 0.0))
    return bfail(SSTEP_ERR_INVALID, "power_iters must be >= 1 when lambda_max is estimated");
  const int prec = M ? M->kind : SSTEP_PREC_JACOBI;
  if (prec != SSTEP_PREC_NONE && prec != SSTEP_PREC_JACOBI)
    return bfail(SSTEP_ERR_INVALID, "unknown preconditioner");
  b->nsys = nsys;
  b->mixed = o->precision == SSTEP_PRECISION_FP32_RR;
  b->nu = o->sweeps;
  b->rtol = o->rtol;
  b->max_outer = o->max_outer;
  int64_t nmax = 0;
  b->hsys.resize(nsys);
  for (int i = 0; i < nsys; ++i) {
    const sstep_matrix& m = A[i];
    if (m.kind != SSTEP_MATRIX_STENCIL || m.points != 7)
      return bfail(SSTEP_ERR_UNSUPPORTED, "batched systems must be 7-point stencils");
    if (m.nx < 1 || m.ny < 1 || m.nz < 1)
      return bfail(SSTEP_ERR_INVALID, "grid dimensions must be >= 1");
    const int64_t n = (int64_t)m.nx * m.ny * m.nz;
    if (n > (int64_t)1 << 30) return bfail(SSTEP_ERR_UNSUPPORTED, "a batched system has more than 2^30 unknowns");
    if (m.n != 0 && m.n != n) return bfail(SSTEP_ERR_INVALID, "n does not match nx*ny*nz");
    BSys& y = b->hsys[i];
    y.nx = m.nx;
    y.ny = m.ny;
    y.nz = m.nz;
    y.n = (int)n;
    y.wc = 6.0;
    y.wo = -1.0;
    if (m.weights) {  // order -z, -y, -x, centre, +x, +y, +z
      const double* w = m.weights;
      for (int k : {0, 1, 2, 4, 5, 6})
        if (w[k] != w[0]) return bfail(SSTEP_ERR_UNSUPPORTED, "batched stencils need six equal neighbour weights");
      y.wc = w[3];
      y.wo = w[0];
    }
    if (!(y.wc > 0.0)) return bfail(SSTEP_ERR_INVALID, "the centre weight must be positive");
    y.d = prec == SSTEP_PREC_JACOBI ? 1.0 / y.wc : 1.0;
    // lower end: 0, or the Gershgorin bound of M^{-1} A (the row with the most neighbours)
    y.lmin = 0.0;
    if (o->lambda_min > 0.0) {
      y.lmin = o->lambda_min;
    } else if (o->lambda_min < 0.0) {
      const int nd[3] = {m.nx, m.ny, m.nz};
      int kmax = 0;
      for (int dd = 0; dd < 3; ++dd) kmax += nd[dd] >= 3 ? 2 : nd[dd] - 1;
      y.lmin = std::max(0.0, y.d * (y.wc - kmax * std::fabs(y.wo)));
    }
    nmax = std::max(nmax, n);
  }
  b->ld = (nmax + 63) / 64 * 64;
  BCK(cudaMalloc((void**)&b->queue, sizeof(int)));
  BCK(cudaMalloc((void**)&b->dsys, sizeof(BSys) * nsys));
  BCK(cudaMemcpyAsync(b->dsys, b->hsys.data(), sizeof(BSys) * nsys, cudaMemcpyHostToDevice, b->st));
  sstep_status st = power_all(b, o);
  if (st != SSTEP_OK) return st;
  BCK(cudaMemcpyAsync(b->dsys, b->hsys.data(), sizeof(BSys) * nsys, cudaMemcpyHostToDevice, b->st));
  BCK(cudaStreamSynchronize(b->st));

  // configuration: given, or autotuned (in-process cache keyed by the batch's shape)
  b->s = o->s;
  b->cluster = o->cluster;
  b->threads = o->block_threads;
  b->rr_opt = o->rr_period;  // <= 0: every s outer iterations (per candidate s when tuning)
  if (b->s == 0 || b->cluster == 0 || b->threads == 0) {
    st = autotune(b, o->s, o->cluster, o->block_threads);
    if (st != SSTEP_OK) return st;
  }
  b->rr_period = b->rr_opt > 0 ? b->rr_opt : b->s;
  KernelFn fn = pick_kernel(b->s, b->mixed, b->threads);
  if (!fn) return bfail(SSTEP_ERR_UNSUPPORTED, "no batched kernel for this (s, threads)");
  b->nslots = max_clusters(fn, b->cluster, b->threads);
  if (b->nslots < 1)
    return bfail(SSTEP_ERR_UNSUPPORTED, "the batched kernel cannot be launched with this cluster size");
  b->slot_bytes = slot_bytes_for(b->s, b->mixed, b->ld);
  BCK(cudaMalloc((void**)&b->ws, b->slot_bytes * (size_t)b->nslots));
  return SSTEP_OK;
}

}  // namespace

sstep_status batch_setup(const sstep_matrix* A, int nsys, const sstep_precond* M,
                         const sstep_opts* o, cudaStream_t st, BatchCtx** out) {
  *out = nullptr;
  if (!A || !o || nsys < 1) return bfail(SSTEP_ERR_INVALID, "bad batched set-up arguments");
  const double t0 = wall_ms();
  BatchCtx* b = new (std::nothrow) BatchCtx();
  if (!b) return bfail(SSTEP_ERR_OOM, "host allocation failed");
  if (st) {
    b->st = st;
  } else {
    // blocking: ordered with the caller's work on the legacy default stream
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamDefault) != cudaSuccess) {
      delete b;
      return bfail(SSTEP_ERR_CUDA, "stream creation failed");
    }
    b->own_stream = true;
  }
  sstep_status s = setup_body(b, A, nsys, M, o);
  if (s != SSTEP_OK) {
    batch_free(b);
    cudaGetLastError();
    return s;
  }
  b->ms_setup = wall_ms() - t0;
  *out = b;
  return SSTEP_OK;
}

sstep_status batch_solve(BatchCtx* b, int nrhs, const double* const* bv, double* const* xv,
                         sstep_info* infos) {
  if (nrhs < 0 || (nrhs > 0 && (!bv || !xv))) return bfail(SSTEP_ERR_INVALID, "bad arguments");
  if (nrhs == 0) return SSTEP_OK;
  const double t0 = wall_ms();
  const int nprob = b->nsys * nrhs;
  for (int i = 0; i < nprob; ++i) {
    if (!bv[i] || !xv[i]) return bfail(SSTEP_ERR_INVALID, "null b or x pointer");
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, bv[i]) != cudaSuccess || pa.type != cudaMemoryTypeDevice ||
        cudaPointerGetAttributes(&pa, xv[i]) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      return bfail(SSTEP_ERR_INVALID, "batched solves take device pointers for b and x");
    }
  }
  sstep_status st = ensure_capacity(b, nprob);
  if (st != SSTEP_OK) return st;
  st = ensure_graph(b, nprob);
  if (st != SSTEP_OK) return st;
  int k = 0;
  for (int i : sys_order(b))
    for (int j = 0; j < nrhs; ++j) {
      const int idx = i * nrhs + j;
      b->hprob[k++] = BProb{bv[idx], xv[idx], i, idx};
    }
  BCK(cudaGraphLaunch(b->gexec, b->st));
  BCK(cudaStreamSynchronize(b->st));
  const double ms = wall_ms() - t0;
  sstep_status first = SSTEP_OK;
  for (int idx = 0; idx < nprob; ++idx) {
    const BRes& r = b->hres[idx];
    const BSys& y = b->hsys[idx / nrhs];
    const sstep_status s = (sstep_status)r.status;
    if (s != SSTEP_OK && first == SSTEP_OK) first = s;
    if (infos) {
      sstep_info& in = infos[idx];
      in.status = s;
      in.outer_iters = r.iters;
      in.inner_equiv = r.iters * b->s;
      in.relres = r.nb2 > 0.0 ? std::sqrt(r.rr / r.nb2) : 0.0;
      in.relres_true = r.nb2 > 0.0 ? std::sqrt(r.rr_true / r.nb2) : 0.0;
      in.lambda_max = y.lmax;
      in.lambda_min = y.lmin;
      in.ms_setup = b->ms_setup;
      in.ms_solve = ms;
      in.launches = 1;
    }
  }
  return first;
}

void batch_config(const BatchCtx* b, int* s, int* cluster, int* threads, int* slots,
                  double* tune_ms) {
  if (s) *s = b->s;
  if (cluster) *cluster = b->cluster;
  if (threads) *threads = b->threads;
  if (slots) *slots = b->nslots;
  if (tune_ms) *tune_ms = b->tune_ms;
}

void batch_free(BatchCtx* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  void* bufs[] = {b->dsys, b->ws, b->queue, b->dprob, b->dres};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (b->hprob) cudaFreeHost(b->hprob);
  if (b->hres) cudaFreeHost(b->hres);
  if (b->st && b->own_stream) cudaStreamDestroy(b->st);
  delete b;
}

}  // namespace sstep
