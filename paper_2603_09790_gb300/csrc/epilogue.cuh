// epilogue.cuh -- the fused epilogues of the FP64 operator kernels (stencil, CSR and Q1 finite
// elements): what one kernel does with (A u)_i besides storing it -- one Matrix-Powers-Kernel
// step (Algorithm 2), the initial residual, a power-method step (Section 2), the PCG product
// A p, the true residual norm and the residual replacement of the FP32-basis path -- and the
// deterministic grid reduction that closes the reducing ones.  Each including translation unit
// gets its own copy (anonymous namespace).
#pragma once

#include "common.cuh"

namespace sstep {
namespace {

// ---------------------------------------------------------------- epilogues

template <int EPI>
struct EpiNV { static constexpr int v = 1; };
template <>
struct EpiNV<EP_RESID> { static constexpr int v = 2; };

template <int EPI>
__device__ __forceinline__ constexpr bool epi_reduces() {
  return EPI == EP_RESID || EPI == EP_POWER || EPI == EP_PCG_AP || EPI == EP_TRUERES ||
         EPI == EP_RR;
}

// y: (A u)_i where u is the (possibly M^{-1}-scaled) operator input; uc: that input at i.
template <int EPI>
__device__ __forceinline__ void epilogue(const EpiArgs& e, int64_t i, double y, double uc,
                                         double* red) {
  if constexpr (EPI == EP_SPMV) {
    e.y[i] = y;
  } else if constexpr (EPI == EP_MPK || EPI == EP_MPK_FIRST) {
    if constexpr (EPI == EP_MPK_FIRST) e.z1[i] = uc;  // z_1 = M^{-1} r
    e.y[i] = y;                                        // A z_q  (column q+1 of P)
    if (e.znext) {
      // c1 M^{-1}: one product per point for a diagonal M, a kernel constant when uniform;
      // c3 = gamma = 1 in the Chebyshev recurrence, so z_{q-1} enters without a product.
      const double a = e.M.dinv ? e.c1 * __ldg(e.M.dinv + i) : e.a1u;
      double t = 0.0;
      if (e.zprev) t = e.c3 == 1.0 ? -__ldg(e.zprev + i) : -e.c3 * __ldg(e.zprev + i);
      e.znext[i] = fma(a, y, fma(-e.c2, uc, t));
    }
  } else if constexpr (EPI == EP_RESID || EPI == EP_RR) {
    const double bi = __ldg(e.b + i);
    const double ri = bi - y;
    if (e.y) e.y[i] = ri;
    if (e.rhi) {  // mixed path: r = rhi + rlo with rhi the FP32 value nearest r
      const float hi = __double2float_rn(ri);
      e.rhi[i] = hi;
      e.rlo[i] = __double2float_rn(ri - (double)hi);
    }
    red[0] = fma(ri, ri, red[0]);
    if constexpr (EPI == EP_RESID) red[1] = fma(bi, bi, red[1]);
  } else if constexpr (EPI == EP_POWER) {
    // v_{l-1} = y_{l-1} / lambda_{l-1} is normalised on the fly: scale by 1/lambda_{l-1}
    const double yi = e.ctrl->inv_scale * prec_d(e.M, i) * y;
    e.y[i] = yi;
    red[0] = fma(yi, yi, red[0]);
  } else if constexpr (EPI == EP_PCG_AP) {
    e.y[i] = y;
    red[0] = fma(uc, y, red[0]);
  } else if constexpr (EPI == EP_TRUERES) {
    const double ri = __ldg(e.b + i) - y;
    red[0] = fma(ri, ri, red[0]);
  }
}

// Kernel-entry early exit: later launches of a finished solve do nothing.
template <int EPI>
__device__ __forceinline__ bool skip(const EpiArgs& e) {
  if (!e.ctrl) return false;
  if constexpr (EPI == EP_POWER) return e.ctrl->power_done != 0;
  if constexpr (EPI == EP_TRUERES || EPI == EP_SPMV) return false;
  return e.ctrl->done != 0;
}

// Finishing step of the reduction, run by one thread of the last CTA.
template <int EPI>
__device__ void finish(const EpiArgs& e, const double* tot) {
  Ctrl* c = e.ctrl;
  if constexpr (EPI == EP_RESID) {
    c->rr = tot[0];
    c->rr0 = tot[0];
    c->nb2 = tot[1];
    c->tol2 = c->rtol2 * tot[1];
    if (!(tot[0] == tot[0]) || tot[0] > 1.79e308 || !(tot[1] == tot[1])) {
      c->status = SSTEP_ERR_NONFINITE;
      c->done = 1;
    } else if (tot[1] == 0.0 || tot[0] <= c->tol2) {
      c->status = SSTEP_OK;
      c->done = 1;
    }
  } else if constexpr (EPI == EP_POWER) {
    // Section 2: stop when |lambda^(l) - lambda^(l-1)| < tol |lambda^(l)| or at the cap.
    const double lam = sqrt(tot[0]);
    c->power_iters += 1;
    const bool conv = c->power_iters > 1 && c->power_tol > 0.0 &&
                      fabs(lam - c->lam) < c->power_tol * fabs(lam);
    c->lam = lam;
    c->inv_scale = lam > 0.0 ? 1.0 / lam : 0.0;
    if (conv || c->power_iters >= c->power_max || !(lam > 0.0)) c->power_done = 1;
  } else if constexpr (EPI == EP_PCG_AP) {
    const double pAp = tot[0];
    if (!(pAp > 0.0) || pAp > 1.79e308) {
      c->status = SSTEP_ERR_BREAKDOWN;
      c->done = 1;
    } else {
      c->pcg_alpha = c->rz / pAp;
    }
  } else if constexpr (EPI == EP_TRUERES) {
    c->sums[0] = tot[0];
  } else if constexpr (EPI == EP_RR) {
    // the replaced residual is the true one: Algorithm 1's stop test applies to it too
    c->rr = tot[0];
    if (!(tot[0] == tot[0]) || tot[0] > 1.79e308) {
      c->status = SSTEP_ERR_NONFINITE;
      c->done = 1;
    } else if (tot[0] <= c->tol2) {
      c->status = SSTEP_OK;
      c->done = 1;
    }
  }
}

template <int EPI>
__device__ __forceinline__ void reduce_and_finish(const EpiArgs& e, double* red) {
  if constexpr (epi_reduces<EPI>()) {
    constexpr int NV = EpiNV<EPI>::v;
    double v[NV], tot[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = red[k];
    const int ticket = (EPI == EP_PCG_AP) ? TK_PCG1 : TK_OP;
    if (grid_sum_last<NV>(v, e.partials, &e.ctrl->ticket[ticket], tot)) {
      if (threadIdx.x == 0) finish<EPI>(e, tot);
    }
  }
}

// ---------------------------------------------------------------- FP32 MPK step (mixed path)

__device__ __forceinline__ void mpk_f32_epilogue(const MpkF32Args& e, int64_t i, float y,
                                                 float uc, bool first) {
  if (first) e.z1[i] = uc;  // z_1 = M^{-1} r
  e.y[i] = y;               // A z_q
  if (e.znext) {
    const float a = e.dinv ? e.c1 * __ldg(e.dinv + i) : e.c1 * e.dinv_u;
    const float t = e.zprev ? -__ldg(e.zprev + i) : 0.0f;
    e.znext[i] = fmaf(a, y, fmaf(-e.c2, uc, t));
  }
}

}  // namespace
}  // namespace sstep
