// k_pcg32.cu -- vector kernels of classical PCG (Section 1) in the precision recipe of the
// FP32-basis s-step path, so that the two solvers are compared at the same storage precision:
// the search direction p and A p are FP32 vectors; x and r are kept as FP32 (hi, lo)
// increments (x = x64 + xhi + xlo, r = rhi + rlo) between FP64 residual replacements; the
// inner products r^T z, ||r||^2 (here) and p^T A p (in the operator kernel that forms A p)
// are accumulated in double-float and summed across CTAs in FP64, in a fixed order.
//
// One iteration: [A p with p^T A p; alpha = r^T z / p^T A p]  ->  k_pcgf_update  ->
// k_pcgf_pdir.  Every rr_period iterations the direction update is preceded by the FP64
// residual replacement (fold x, r = b - A x, stop test) and k_pcgf_rz, which recomputes r^T z
// for the replaced r and takes beta against the r^T z of the previous iteration.
#include <algorithm>

#include "common.cuh"

namespace sstep {

namespace {

__device__ __forceinline__ float zdiag(const PcgF32Args& a, int64_t i) {
  return a.dinv ? __ldg(a.dinv + i) : a.dinv_u;
}

// x += alpha p, r -= alpha Ap in double-float (alpha split into FP32 hi + lo), then the
// double-float sums r^T z (z = M^{-1} r_hi) and ||r||^2 of the updated r.
struct PcgPoint {
  float ah, al;
  __device__ __forceinline__ void operator()(float p, float ap, float d, float& xh, float& xl,
                                             float& rh, float& rl, float (&hi)[2],
                                             float (&lo)[2]) const {
    float dxh = 0.0f, dxl = 0.0f, drh = 0.0f, drl = 0.0f;
    df_acc_prod(dxh, dxl, p, ah);
    dxl = fmaf(p, al, dxl);
    df_acc_prod(drh, drl, ap, ah);
    drl = fmaf(ap, al, drl);
    df_add(xh, xl, dxh, dxl);
    df_add(rh, rl, -drh, -drl);
    const float z = d * rh;
    df_acc_prod(hi[0], lo[0], rh, z);  // r^T z
    lo[0] = fmaf(rl, z, lo[0]);
    df_acc_prod(hi[1], lo[1], rh, rh);  // ||r||^2
    lo[1] = fmaf(2.0f * rh, rl, lo[1]);
  }
};

__global__ void __launch_bounds__(kThreads) k_pcgf_update(PcgF32Args a) {
  if (a.ctrl->done) return;
  __shared__ double buf[kTiledSmem];
  __shared__ float alh, all;
  if (threadIdx.x == 0) {
    const double v = a.ctrl->pcg_alpha;
    const float h = __double2float_rn(v);
    alh = h;
    all = __double2float_rn(v - (double)h);
  }
  __syncthreads();
  const PcgPoint point{alh, all};
  float hi[2] = {0.0f, 0.0f}, lo[2] = {0.0f, 0.0f};
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // four consecutive points per thread and trip: 16-byte loads and stores (the FP32 vectors
  // start on 256-byte boundaries)
  const int64_t n4 = a.n >> 2;
  for (int64_t v = gid; v < n4; v += stride) {
    const float4 p = __ldg(reinterpret_cast<const float4*>(a.p) + v);
    const float4 ap = __ldg(reinterpret_cast<const float4*>(a.Ap) + v);
    float4 d = make_float4(a.dinv_u, a.dinv_u, a.dinv_u, a.dinv_u);
    if (a.dinv) d = __ldg(reinterpret_cast<const float4*>(a.dinv) + v);
    float4 xh = reinterpret_cast<float4*>(a.xhi)[v], xl = reinterpret_cast<float4*>(a.xlo)[v];
    float4 rh = reinterpret_cast<float4*>(a.rhi)[v], rl = reinterpret_cast<float4*>(a.rlo)[v];
    point(p.x, ap.x, d.x, xh.x, xl.x, rh.x, rl.x, hi, lo);
    point(p.y, ap.y, d.y, xh.y, xl.y, rh.y, rl.y, hi, lo);
    point(p.z, ap.z, d.z, xh.z, xl.z, rh.z, rl.z, hi, lo);
    point(p.w, ap.w, d.w, xh.w, xl.w, rh.w, rl.w, hi, lo);
    reinterpret_cast<float4*>(a.xhi)[v] = xh;
    reinterpret_cast<float4*>(a.xlo)[v] = xl;
    reinterpret_cast<float4*>(a.rhi)[v] = rh;
    reinterpret_cast<float4*>(a.rlo)[v] = rl;
  }
  for (int64_t i = 4 * n4 + gid; i < a.n; i += stride) {  // the last n mod 4 points
    float xh = a.xhi[i], xl = a.xlo[i], rh = a.rhi[i], rl = a.rlo[i];
    point(__ldg(a.p + i), __ldg(a.Ap + i), zdiag(a, i), xh, xl, rh, rl, hi, lo);
    a.xhi[i] = xh;
    a.xlo[i] = xl;
    a.rhi[i] = rh;
    a.rlo[i] = rl;
  }
  if (!df_grid_sums<2>(hi, lo, buf, a.partials, &a.ctrl->ticket[TK_PCG2])) return;
  if (threadIdx.x == 0) {
    Ctrl* c = a.ctrl;
    const double rz = buf[0], rr = buf[1];
    stop_test(c, rr);
    if (a.hist) a.hist[c->iters] = sqrt(rr / c->nb2);
    c->rz_prev = c->rz;
    c->pcg_beta = rz / c->rz;
    c->rz = rz;
  }
}

// r^T z of the current r = rhi + rlo, z = M^{-1} r_hi; init: beta = 0, else beta = rz / rz_prev.
__global__ void __launch_bounds__(kThreads) k_pcgf_rz(PcgF32Args a, int init) {
  if (a.ctrl->done) return;
  __shared__ double buf[kTiledSmem];
  float hi[1] = {0.0f}, lo[1] = {0.0f};
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = a.n >> 2;
  for (int64_t v = gid; v < n4; v += stride) {
    const float4 rh = __ldg(reinterpret_cast<const float4*>(a.rhi) + v);
    const float4 rl = __ldg(reinterpret_cast<const float4*>(a.rlo) + v);
    float4 d = make_float4(a.dinv_u, a.dinv_u, a.dinv_u, a.dinv_u);
    if (a.dinv) d = __ldg(reinterpret_cast<const float4*>(a.dinv) + v);
    const float r4[4] = {rh.x, rh.y, rh.z, rh.w}, l4[4] = {rl.x, rl.y, rl.z, rl.w};
    const float d4[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const float z = d4[l] * r4[l];
      df_acc_prod(hi[0], lo[0], r4[l], z);
      lo[0] = fmaf(l4[l], z, lo[0]);
    }
  }
  for (int64_t i = 4 * n4 + gid; i < a.n; i += stride) {
    const float rh = __ldg(a.rhi + i), rl = __ldg(a.rlo + i);
    const float z = zdiag(a, i) * rh;
    df_acc_prod(hi[0], lo[0], rh, z);
    lo[0] = fmaf(rl, z, lo[0]);
  }
  if (!df_grid_sums<1>(hi, lo, buf, a.partials, &a.ctrl->ticket[TK_PCG2])) return;
  if (threadIdx.x == 0) {
    Ctrl* c = a.ctrl;
    const double rz = buf[0];
    if (init) {
      c->pcg_beta = 0.0;
      c->rz_prev = rz;
    } else {
      c->pcg_beta = rz / c->rz_prev;
    }
    c->rz = rz;
  }
}

// p = z + beta p with z = M^{-1} r_hi (init: p = z; p's old contents are not read).
__global__ void __launch_bounds__(kThreads) k_pcgf_pdir(PcgF32Args a, int init) {
  if (a.ctrl->done) return;
  const float be = __double2float_rn(a.ctrl->pcg_beta);
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n4 = a.n >> 2;
  for (int64_t v = gid; v < n4; v += stride) {
    const float4 rh = __ldg(reinterpret_cast<const float4*>(a.rhi) + v);
    float4 d = make_float4(a.dinv_u, a.dinv_u, a.dinv_u, a.dinv_u);
    if (a.dinv) d = __ldg(reinterpret_cast<const float4*>(a.dinv) + v);
    float4 z = make_float4(d.x * rh.x, d.y * rh.y, d.z * rh.z, d.w * rh.w);
    if (!init) {
      const float4 p = reinterpret_cast<const float4*>(a.p)[v];
      z.x = fmaf(be, p.x, z.x);
      z.y = fmaf(be, p.y, z.y);
      z.z = fmaf(be, p.z, z.z);
      z.w = fmaf(be, p.w, z.w);
    }
    reinterpret_cast<float4*>(a.p)[v] = z;
  }
  for (int64_t i = 4 * n4 + gid; i < a.n; i += stride) {
    const float z = zdiag(a, i) * __ldg(a.rhi + i);
    a.p[i] = init ? z : fmaf(be, a.p[i], z);
  }
}

// One full wave of resident CTAs of `kernel` (as many as its registers allow, up to 2048 threads
// per SM: the vector kernels are latency-bound otherwise), no more CTAs than four points per
// thread; the grid-stride loops spread the points evenly over them.
template <typename KernelT>
int pcgf_ctas(KernelT kernel, int& per_sm, int64_t n) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  if (!per_sm &&
      (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess ||
       per_sm < 1))
    per_sm = 1;
  const int64_t want = (int64_t)sms * std::min(per_sm, 8);
  const int64_t need = (n / 4 + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, need));
}

}  // namespace

cudaError_t launch_pcgf_update(const PcgF32Args& a, cudaStream_t st) {
  static int occ = 0;
  k_pcgf_update<<<pcgf_ctas(k_pcgf_update, occ, a.n), kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pcgf_rz(const PcgF32Args& a, int init, cudaStream_t st) {
  static int occ = 0;
  k_pcgf_rz<<<pcgf_ctas(k_pcgf_rz, occ, a.n), kThreads, 0, st>>>(a, init);
  return cudaGetLastError();
}

cudaError_t launch_pcgf_pdir(const PcgF32Args& a, int init, cudaStream_t st) {
  static int occ = 0;
  k_pcgf_pdir<<<pcgf_ctas(k_pcgf_pdir, occ, a.n), kThreads, 0, st>>>(a, init);
  return cudaGetLastError();
}

}  // namespace sstep
