// k_operator.cu -- y = A u for the stencil and CSR operators, with fused epilogues:
// one Matrix-Powers-Kernel step (Algorithm 2: SpMV + M^{-1} + Chebyshev three-term
// recurrence), initial residual, power-method step (Section 2), the PCG product A p, and the
// true residual norm.
//
// Stencil operators (5/7/27 points) are matrix-free.  A CTA owns a 32 x 8 tile of the xy plane
// and marches through a chunk of z planes (2.5D blocking): the current plane with its one-point
// xy halo is staged in shared memory, the z neighbours of the thread's own column travel in
// registers.  Each input value is read from HBM once per sweep; halo values of neighbouring
// tiles come from L2.  The 27-point Poisson operator (HPCG, Section 6) uses sum factorisation
// of the 3x3x3 box: 27 u - box(u) costs 7.5 FP64 operations per point instead of 26.
#include <algorithm>

#include "common.cuh"
#include "epilogue.cuh"
#include "tma.cuh"

namespace sstep {

namespace {

constexpr int TX = 32, TY = 8;

// ---------------------------------------------------------------- 5/7-point stencil

// A(u) at one point of a 5/7-point stencil: in-plane neighbours from the staged plane p
// (with its one-point halo), z neighbours ub (z-1) and ua (z+1) from registers.
template <int PTS, bool POISSON>
__device__ __forceinline__ double stencil7_point(const StencilOp& op, const double (*p)[TX + 2],
                                                 int tx, int ty, double ub, double uc, double ua) {
  if constexpr (POISSON) {
    double s = (p[ty + 1][tx] + p[ty + 1][tx + 2]) + (p[ty][tx + 1] + p[ty + 2][tx + 1]);
    if constexpr (PTS == 7) s += ub + ua;
    return fma(op.wc, uc, -s);
  } else if constexpr (PTS == 7) {
    double a = op.w[0] * ub;
    a = fma(op.w[1], p[ty][tx + 1], a);
    a = fma(op.w[2], p[ty + 1][tx], a);
    a = fma(op.w[3], uc, a);
    a = fma(op.w[4], p[ty + 1][tx + 2], a);
    a = fma(op.w[5], p[ty + 2][tx + 1], a);
    return fma(op.w[6], ua, a);
  } else {
    double a = op.w[0] * p[ty][tx + 1];
    a = fma(op.w[1], p[ty + 1][tx], a);
    a = fma(op.w[2], uc, a);
    a = fma(op.w[3], p[ty + 1][tx + 2], a);
    return fma(op.w[4], p[ty + 2][tx + 1], a);
  }
}

// Two z planes per iteration, two sets of staged planes (one barrier per iteration), and the
// next iteration's centre and halo values loaded into registers before the barrier so that
// their latency overlaps the arithmetic.  SCALE: multiply every loaded input value by M^{-1}
// (MPK first step with a non-uniform M).
template <int PTS, bool POISSON, int EPI, bool SCALE>
__global__ void __launch_bounds__(TX * TY) k_stencil7(StencilOp op, EpiArgs e, int zc) {
  if (skip<EPI>(e)) return;
  __shared__ double t[2][2][TY + 2][TX + 2];
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const int x = blockIdx.x * TX + tx, y = blockIdx.y * TY + ty;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
  const int64_t pxy = (int64_t)nx * ny;
  const bool in = x < nx && y < ny;
  const int64_t col = (int64_t)y * nx + x;
  const double* __restrict__ u = e.u;
  // Halo duty: threads on the tile's x edges load the x-1 / x+1 column, those on its y edges
  // the y-1 / y+1 row; outside the grid the value is 0 (Dirichlet neighbours dropped).
  const int hx = tx == 0 ? -1 : (tx == TX - 1 ? 1 : 0);
  const int hy = ty == 0 ? -1 : (ty == TY - 1 ? 1 : 0);
  const bool hxok = hx != 0 && x + hx >= 0 && x + hx < nx && y < ny;
  const bool hyok = hy != 0 && y + hy >= 0 && y + hy < ny && x < nx;
  const int64_t hxoff = col + hx, hyoff = col + (int64_t)hy * nx;
  auto ld = [&](int64_t off, int zz, bool ok) -> double {
    if (!ok || zz < 0 || zz >= nz) return 0.0;
    const int64_t idx = off + (int64_t)zz * pxy;
    double v = __ldg(u + idx);
    if constexpr (SCALE) v *= __ldg(e.M.dinv + idx);
    return v;
  };
  double red[2] = {0.0, 0.0};
  double ub = ld(col, z0 - 1, in), uc = ld(col, z0, in);
  double ua = ld(col, z0 + 1, in), ua2 = ld(col, z0 + 2, in);
  double hx0 = ld(hxoff, z0, hxok), hx1 = ld(hxoff, z0 + 1, hxok);
  double hy0 = ld(hyoff, z0, hyok), hy1 = ld(hyoff, z0 + 1, hyok);
  int set = 0;
  for (int z = z0; z < z1; z += 2) {
    double (*P0)[TX + 2] = t[set][0];
    double (*P1)[TX + 2] = t[set][1];
    P0[ty + 1][tx + 1] = uc;
    P1[ty + 1][tx + 1] = ua;
    if (hx) {
      P0[ty + 1][tx + 1 + hx] = hx0;
      P1[ty + 1][tx + 1 + hx] = hx1;
    }
    if (hy) {
      P0[ty + 1 + hy][tx + 1] = hy0;
      P1[ty + 1 + hy][tx + 1] = hy1;
    }
    // next pair of planes: centres z+3, z+4 and halos of z+2, z+3
    const double n3 = ld(col, z + 3, in), n4 = ld(col, z + 4, in);
    const double nhx0 = ld(hxoff, z + 2, hxok), nhx1 = ld(hxoff, z + 3, hxok);
    const double nhy0 = ld(hyoff, z + 2, hyok), nhy1 = ld(hyoff, z + 3, hyok);
    __syncthreads();
    if (in) {
      double a0 = stencil7_point<PTS, POISSON>(op, P0, tx, ty, ub, uc, ua);
      double c0 = uc;
      if constexpr (EPI == EP_MPK_FIRST && !SCALE) {  // uniform M^{-1}: A (d r) = d (A r)
        a0 *= e.M.dinv_u;
        c0 *= e.M.dinv_u;
      }
      epilogue<EPI>(e, (int64_t)z * pxy + col, a0, c0, red);
      if (z + 1 < z1) {
        double a1 = stencil7_point<PTS, POISSON>(op, P1, tx, ty, uc, ua, ua2);
        double c1 = ua;
        if constexpr (EPI == EP_MPK_FIRST && !SCALE) {
          a1 *= e.M.dinv_u;
          c1 *= e.M.dinv_u;
        }
        epilogue<EPI>(e, (int64_t)(z + 1) * pxy + col, a1, c1, red);
      }
    }
    ub = ua;
    uc = ua2;
    ua = n3;
    ua2 = n4;
    hx0 = nhx0;
    hx1 = nhx1;
    hy0 = nhy0;
    hy1 = nhy1;
    set ^= 1;
  }
  reduce_and_finish<EPI>(e, red);
}

// ---------------------------------------------------------------- 27-point stencil

// POISSON: y = 27 u - box3x3x3(u) by sum factorisation (row sums in x, column sums in y,
// plane sums in z kept in registers).  General constant weights: 27 products per point.
template <bool POISSON, int EPI, bool SCALE>
__global__ void __launch_bounds__(TX * TY) k_stencil27(StencilOp op, EpiArgs e, int zc) {
  if (skip<EPI>(e)) return;
  __shared__ double pl[3][TY + 2][TX + 2];  // planes z-1, z, z+1 (general weights)
  __shared__ double rs[TY + 2][TX];         // x row sums of the newest plane (Poisson)
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const int x = blockIdx.x * TX + tx, y = blockIdx.y * TY + ty;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
  const int64_t pxy = (int64_t)nx * ny;
  const bool in = x < nx && y < ny;
  const double* __restrict__ u = e.u;
  auto ld = [&](int xx, int yy, int zz) -> double {
    if (xx < 0 || xx >= nx || yy < 0 || yy >= ny || zz < 0 || zz >= nz) return 0.0;
    const int64_t idx = (int64_t)zz * pxy + (int64_t)yy * nx + xx;
    double v = __ldg(u + idx);
    if constexpr (SCALE) v *= __ldg(e.M.dinv + idx);
    return v;
  };
  // Stage plane zz (with xy halo) into slot `s` of pl.
  auto stage = [&](int slot, int zz) {
    double (*p)[TX + 2] = pl[slot];
    p[ty + 1][tx + 1] = ld(x, y, zz);
    if (tx == 0) {
      p[ty + 1][0] = ld(x - 1, y, zz);
      if (ty == 0) p[0][0] = ld(x - 1, y - 1, zz);
      if (ty == TY - 1) p[TY + 1][0] = ld(x - 1, y + 1, zz);
    }
    if (tx == TX - 1) {
      p[ty + 1][TX + 1] = ld(x + 1, y, zz);
      if (ty == 0) p[0][TX + 1] = ld(x + 1, y - 1, zz);
      if (ty == TY - 1) p[TY + 1][TX + 1] = ld(x + 1, y + 1, zz);
    }
    if (ty == 0) p[0][tx + 1] = ld(x, y - 1, zz);
    if (ty == TY - 1) p[TY + 1][tx + 1] = ld(x, y + 1, zz);
  };
  double red[2] = {0.0, 0.0};
  if constexpr (POISSON) {
    // s2 = column (y) sums of x row sums, for planes z-1, z, z+1 of the thread's column.
    auto plane_s2 = [&](int zz) -> double {
      stage(0, zz);
      __syncthreads();
      rs[ty + 1][tx] = pl[0][ty + 1][tx] + pl[0][ty + 1][tx + 1] + pl[0][ty + 1][tx + 2];
      if (ty == 0) rs[0][tx] = pl[0][0][tx] + pl[0][0][tx + 1] + pl[0][0][tx + 2];
      if (ty == TY - 1)
        rs[TY + 1][tx] = pl[0][TY + 1][tx] + pl[0][TY + 1][tx + 1] + pl[0][TY + 1][tx + 2];
      __syncthreads();
      const double v = rs[ty][tx] + rs[ty + 1][tx] + rs[ty + 2][tx];
      __syncthreads();
      return v;
    };
    double sb = plane_s2(z0 - 1);
    double sc = plane_s2(z0);
    double uc = ld(x, y, z0);
    for (int z = z0; z < z1; ++z) {
      const double sa = plane_s2(z + 1);
      const double ua = ld(x, y, z + 1);
      if (in) {
        const double box = (sb + sc) + sa;
        double a = fma(op.wc + 1.0, uc, -box);  // 26 u - (box - u) with wc = 26
        double ucc = uc;
        if constexpr (EPI == EP_MPK_FIRST && !SCALE) {
          a *= e.M.dinv_u;
          ucc *= e.M.dinv_u;
        }
        epilogue<EPI>(e, (int64_t)z * pxy + (int64_t)y * nx + x, a, ucc, red);
      }
      sb = sc;
      sc = sa;
      uc = ua;
    }
  } else {
    stage(0, z0 - 1);
    stage(1, z0);
    for (int z = z0; z < z1; ++z) {
      const int sm = (z - z0) % 3, s0 = (z - z0 + 1) % 3, sp = (z - z0 + 2) % 3;
      stage(sp, z + 1);
      __syncthreads();
      if (in) {
        double a = 0.0;
        int k = 0;
        const int slots[3] = {sm, s0, sp};
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
          for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) a = fma(op.w[k++], pl[slots[dz]][ty + dy][tx + dx], a);
        double ucc = pl[s0][ty + 1][tx + 1];
        if constexpr (EPI == EP_MPK_FIRST && !SCALE) {
          a *= e.M.dinv_u;
          ucc *= e.M.dinv_u;
        }
        epilogue<EPI>(e, (int64_t)z * pxy + (int64_t)y * nx + x, a, ucc, red);
      }
      __syncthreads();
    }
  }
  reduce_and_finish<EPI>(e, red);
}

// ---------------------------------------------------------------- CSR

constexpr int kCsrCtasPerSm = 8;

template <int EPI, bool SCALE>
__global__ void __launch_bounds__(kThreads) k_csr(CsrOp A, EpiArgs e) {
  if (skip<EPI>(e)) return;
  double red[2] = {0.0, 0.0};
  const double* __restrict__ u = e.u;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k0 = __ldg(A.rowptr + i), k1 = __ldg(A.rowptr + i + 1);
    double a = 0.0;
    for (int64_t k = k0; k < k1; ++k) {
      const int32_t c = __ldg(A.colind + k);
      double v = __ldg(u + c);
      if constexpr (SCALE) v *= __ldg(e.M.dinv + c);
      a = fma(__ldg(A.vals + k), v, a);
    }
    double uc = __ldg(u + i);
    if constexpr (SCALE) uc *= __ldg(e.M.dinv + i);
    if constexpr (EPI == EP_MPK_FIRST && !SCALE) {
      a *= e.M.dinv_u;
      uc *= e.M.dinv_u;
    }
    epilogue<EPI>(e, i, a, uc, red);
  }
  reduce_and_finish<EPI>(e, red);
}

// ---------------------------------------------------------------- FP32 MPK step (mixed path)

template <int PTS, bool POISSON>
__device__ __forceinline__ float stencil7_point_f(const MpkF32Args& e, const float (*p)[TX + 2],
                                                  int tx, int ty, float ub, float uc, float ua) {
  if constexpr (POISSON) {
    float s = (p[ty + 1][tx] + p[ty + 1][tx + 2]) + (p[ty][tx + 1] + p[ty + 2][tx + 1]);
    if constexpr (PTS == 7) s += ub + ua;
    return fmaf(e.wc, uc, -s);
  } else if constexpr (PTS == 7) {
    float a = e.w[0] * ub;
    a = fmaf(e.w[1], p[ty][tx + 1], a);
    a = fmaf(e.w[2], p[ty + 1][tx], a);
    a = fmaf(e.w[3], uc, a);
    a = fmaf(e.w[4], p[ty + 1][tx + 2], a);
    a = fmaf(e.w[5], p[ty + 2][tx + 1], a);
    return fmaf(e.w[6], ua, a);
  } else {
    float a = e.w[0] * p[ty][tx + 1];
    a = fmaf(e.w[1], p[ty + 1][tx], a);
    a = fmaf(e.w[2], uc, a);
    a = fmaf(e.w[3], p[ty + 1][tx + 2], a);
    return fmaf(e.w[4], p[ty + 2][tx + 1], a);
  }
}

// The 2.5D body of k_stencil7 with FP32 values: half the bytes per point, and the FP32 pipe
// (64x the FP64 one on this part) does the arithmetic, so the step is bound by HBM.
template <int PTS, bool POISSON, bool FIRST, bool SCALE, bool PAP = false>
__global__ void __launch_bounds__(TX * TY) k_stencil7f(StencilOp op, MpkF32Args e, int zc) {
  if (e.ctrl && e.ctrl->done) return;
  float ph[1] = {0.0f}, pl[1] = {0.0f};  // PAP: p^T (A p)
  __shared__ float t[2][2][TY + 2][TX + 2];
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const int x = blockIdx.x * TX + tx, y = blockIdx.y * TY + ty;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
  const int64_t pxy = (int64_t)nx * ny;
  const bool in = x < nx && y < ny;
  const int64_t col = (int64_t)y * nx + x;
  const int hx = tx == 0 ? -1 : (tx == TX - 1 ? 1 : 0);
  const int hy = ty == 0 ? -1 : (ty == TY - 1 ? 1 : 0);
  const bool hxok = hx != 0 && x + hx >= 0 && x + hx < nx && y < ny;
  const bool hyok = hy != 0 && y + hy >= 0 && y + hy < ny && x < nx;
  const int64_t hxoff = col + hx, hyoff = col + (int64_t)hy * nx;
  auto ld = [&](int64_t off, int zz, bool ok) -> float {
    if (!ok || zz < 0 || zz >= nz) return 0.0f;
    const int64_t idx = off + (int64_t)zz * pxy;
    float v = __ldg(e.u + idx);
    if constexpr (SCALE) v *= __ldg(e.dinv + idx);
    return v;
  };
  float ub = ld(col, z0 - 1, in), uc = ld(col, z0, in);
  float ua = ld(col, z0 + 1, in), ua2 = ld(col, z0 + 2, in);
  float hx0 = ld(hxoff, z0, hxok), hx1 = ld(hxoff, z0 + 1, hxok);
  float hy0 = ld(hyoff, z0, hyok), hy1 = ld(hyoff, z0 + 1, hyok);
  int set = 0;
  for (int z = z0; z < z1; z += 2) {
    float (*P0)[TX + 2] = t[set][0];
    float (*P1)[TX + 2] = t[set][1];
    P0[ty + 1][tx + 1] = uc;
    P1[ty + 1][tx + 1] = ua;
    if (hx) {
      P0[ty + 1][tx + 1 + hx] = hx0;
      P1[ty + 1][tx + 1 + hx] = hx1;
    }
    if (hy) {
      P0[ty + 1 + hy][tx + 1] = hy0;
      P1[ty + 1 + hy][tx + 1] = hy1;
    }
    const float n3 = ld(col, z + 3, in), n4 = ld(col, z + 4, in);
    const float nhx0 = ld(hxoff, z + 2, hxok), nhx1 = ld(hxoff, z + 3, hxok);
    const float nhy0 = ld(hyoff, z + 2, hyok), nhy1 = ld(hyoff, z + 3, hyok);
    __syncthreads();
    if (in) {
      float a0 = stencil7_point_f<PTS, POISSON>(e, P0, tx, ty, ub, uc, ua), c0 = uc;
      if constexpr (FIRST && !SCALE) {
        a0 *= e.dinv_u;
        c0 *= e.dinv_u;
      }
      mpk_f32_epilogue(e, (int64_t)z * pxy + col, a0, c0, FIRST);
      if constexpr (PAP) df_acc_prod(ph[0], pl[0], c0, a0);
      if (z + 1 < z1) {
        float a1 = stencil7_point_f<PTS, POISSON>(e, P1, tx, ty, uc, ua, ua2), c1 = ua;
        if constexpr (FIRST && !SCALE) {
          a1 *= e.dinv_u;
          c1 *= e.dinv_u;
        }
        mpk_f32_epilogue(e, (int64_t)(z + 1) * pxy + col, a1, c1, FIRST);
        if constexpr (PAP) df_acc_prod(ph[0], pl[0], c1, a1);
      }
    }
    ub = ua;
    uc = ua2;
    ua = n3;
    ua2 = n4;
    hx0 = nhx0;
    hx1 = nhx1;
    hy0 = nhy0;
    hy1 = nhy1;
    set ^= 1;
  }
  if constexpr (PAP) pap_finish(e, ph, pl);
}

// FP32 MPK step for 7-point stencils with nx a multiple of 4 and a uniform M^{-1}: each thread
// owns four consecutive x points (16-byte loads and stores), a CTA a 64 x 16 tile of a z
// chunk, marching in z with the planes z-1, z, z+1 in registers and plane z staged in shared
// memory (two buffers, one barrier per plane) for the y and cross-vector x neighbours.  Four
// points share one set of index computations, which bounded the scalar kernel.
constexpr int TX4 = 16, TY4 = 16;  // threads: 16 float4 columns x 16 rows
constexpr int kRow4 = 4 * TX4 + 8;  // floats per staged row: 4 pad | 64 values | 4 pad

template <bool POISSON, bool FIRST, bool PAP = false>
__global__ void __launch_bounds__(TX4 * TY4) k_stencil7f4(StencilOp op, MpkF32Args e, int zc) {
  if (e.ctrl && e.ctrl->done) return;
  float ph[1] = {0.0f}, pl[1] = {0.0f};  // PAP: p^T (A p)
  __shared__ __align__(16) float sm[2][TY4 + 2][kRow4];
  const int tx = threadIdx.x % TX4, ty = threadIdx.x / TX4;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const int x0 = (blockIdx.x * TX4 + tx) * 4, y = blockIdx.y * TY4 + ty;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
  const int64_t pxy = (int64_t)nx * ny;
  const bool in = x0 < nx && y < ny;          // nx % 4 == 0: the whole vector is inside
  const int64_t col = (int64_t)y * nx + x0;
  const int hy = ty == 0 ? -1 : (ty == TY4 - 1 ? 1 : 0);
  const bool hyok = hy != 0 && x0 < nx && y + hy >= 0 && y + hy < ny;
  const int64_t hycol = col + (int64_t)hy * nx;
  // x halos: the point left of the tile (thread tx = 0) and right of it (tx = TX4 - 1)
  const int hx = tx == 0 ? -1 : (tx == TX4 - 1 ? 4 : 0);
  const bool hxok = hx != 0 && y < ny && x0 + hx >= 0 && x0 + hx < nx;
  const int64_t hxcol = col + hx;
  const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  auto ld4 = [&](int64_t c, int zz, bool ok) -> float4 {
    if (!ok || zz < 0 || zz >= nz) return zero4;
    return __ldg(reinterpret_cast<const float4*>(e.u + c + (int64_t)zz * pxy));
  };
  auto ld1 = [&](int64_t c, int zz, bool ok) -> float {
    if (!ok || zz < 0 || zz >= nz) return 0.0f;
    return __ldg(e.u + c + (int64_t)zz * pxy);
  };
  float4 ub = ld4(col, z0 - 1, in), uc = ld4(col, z0, in), ua = ld4(col, z0 + 1, in);
  float4 ua2 = ld4(col, z0 + 2, in);
  float4 hyv = ld4(hycol, z0, hyok);
  float hxv = ld1(hxcol, z0, hxok);
  const float wc = e.wc, a1 = e.c1 * e.dinv_u, c2 = e.c2;
  // z_{q-1} at this thread's points of the current plane, requested a plane ahead
  const bool zpv_on = in && e.znext && e.zprev;
  float4 zp = zpv_on ? __ldg(reinterpret_cast<const float4*>(e.zprev + (int64_t)z0 * pxy + col))
                     : zero4;
  int set = 0;
  for (int z = z0; z < z1; ++z) {
    float (*P)[kRow4] = sm[set];
    *reinterpret_cast<float4*>(&P[ty + 1][4 + 4 * tx]) = uc;
    if (hy) *reinterpret_cast<float4*>(&P[ty + 1 + hy][4 + 4 * tx]) = hyv;
    if (hx < 0) P[ty + 1][3] = hxv;
    if (hx > 0) P[ty + 1][4 + 4 * TX4] = hxv;
    // values of the planes ahead in flight during the barrier and the arithmetic: u two planes
    // ahead (z + 3), its halo and z_{q-1} one plane ahead
    const float4 nz4 = ld4(col, z + 3, in);
    const float4 nhy = ld4(hycol, z + 1, hyok);
    const float nhx = ld1(hxcol, z + 1, hxok);
    const float4 nzp = (zpv_on && z + 1 < z1)
                           ? __ldg(reinterpret_cast<const float4*>(e.zprev + (int64_t)(z + 1) * pxy + col))
                           : zero4;
    __syncthreads();
    if (in) {
      const float4 ym = *reinterpret_cast<const float4*>(&P[ty][4 + 4 * tx]);
      const float4 yp = *reinterpret_cast<const float4*>(&P[ty + 2][4 + 4 * tx]);
      const float xl = P[ty + 1][3 + 4 * tx], xr = P[ty + 1][8 + 4 * tx];
      const float xm[4] = {xl, uc.x, uc.y, uc.z}, xp[4] = {uc.y, uc.z, uc.w, xr};
      const float c[4] = {uc.x, uc.y, uc.z, uc.w}, dn[4] = {ub.x, ub.y, ub.z, ub.w};
      const float up[4] = {ua.x, ua.y, ua.z, ua.w};
      const float yM[4] = {ym.x, ym.y, ym.z, ym.w}, yP[4] = {yp.x, yp.y, yp.z, yp.w};
      float av[4], cv[4];
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        float a;
        if constexpr (POISSON) {
          float s = (xm[l] + xp[l]) + (yM[l] + yP[l]);
          s += dn[l] + up[l];
          a = fmaf(wc, c[l], -s);
        } else {  // weights in the order -z, -y, -x, centre, +x, +y, +z
          a = e.w[0] * dn[l];
          a = fmaf(e.w[1], yM[l], a);
          a = fmaf(e.w[2], xm[l], a);
          a = fmaf(e.w[3], c[l], a);
          a = fmaf(e.w[4], xp[l], a);
          a = fmaf(e.w[5], yP[l], a);
          a = fmaf(e.w[6], up[l], a);
        }
        float cc = c[l];
        if constexpr (FIRST) {  // uniform M^{-1}: A (d r) = d (A r)
          a *= e.dinv_u;
          cc *= e.dinv_u;
        }
        av[l] = a;
        cv[l] = cc;
      }
      const int64_t i = (int64_t)z * pxy + col;
      if constexpr (PAP) {
#pragma unroll
        for (int l = 0; l < 4; ++l) df_acc_prod(ph[0], pl[0], cv[l], av[l]);
      }
      if constexpr (FIRST) *reinterpret_cast<float4*>(e.z1 + i) = make_float4(cv[0], cv[1], cv[2], cv[3]);
      *reinterpret_cast<float4*>(e.y + i) = make_float4(av[0], av[1], av[2], av[3]);
      if (e.znext) {
        const float zpv[4] = {zp.x, zp.y, zp.z, zp.w};
        float zn[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) zn[l] = fmaf(a1, av[l], fmaf(-c2, cv[l], -zpv[l]));
        *reinterpret_cast<float4*>(e.znext + i) = make_float4(zn[0], zn[1], zn[2], zn[3]);
      }
    }
    ub = uc;
    uc = ua;
    ua = ua2;
    ua2 = nz4;
    hyv = nhy;
    hxv = nhx;
    zp = nzp;
    set ^= 1;
  }
  if constexpr (PAP) pap_finish(e, ph, pl);
}

// The same FP32 steps (MPK with a uniform M^{-1}, and the PCG product) with the u planes brought
// in by the tensor-memory accelerator.  A CTA owns the same 64 x 16 tile and z chunk as
// k_stencil7f4; one thread keeps up to kS7 planes of u in flight, each a 72 x 18 box (x from 4
// left of the tile, so that the x coordinate stays a multiple of 16 bytes; y from 1 below)
// that lands on its stage's mbarrier.  The copy zero-fills whatever lies outside the grid: the
// eliminated Dirichlet boundary.  Plane z reads stages z-1, z, z+1 straight from shared memory,
// so the depth of the pipeline costs shared memory, not registers (the register-fed kernel held
// two planes ahead and waited about one memory latency per plane).  The arithmetic is
// k_stencil7f4's, operation for operation.  Every wait is bounded: a copy that never lands
// stops the solve with SSTEP_ERR_TIMEOUT instead of hanging.
constexpr int S7W = 4 * TX4 + 8, S7H = TY4 + 2;  // box: 72 x 18 floats
constexpr int kS7 = 8;                           // pipeline stages (z planes)
constexpr int kS7Stage = 1312;                   // floats per stage: 1296 used, 5248 bytes (41 x 128)
constexpr uint32_t kS7Bytes = S7W * S7H * 4;
constexpr int kS7MaxCols = kMaxS + 1;

struct __align__(128) St7Smem {
  float u[kS7][kS7Stage];
  unsigned long long full[kS7];
};

template <bool POISSON, bool FIRST, bool PAP = false>
__global__ void __launch_bounds__(TX4 * TY4) k_stencil7f4_tma(const __grid_constant__ CUtensorMap mu,
                                                             StencilOp op, MpkF32Args e, int zc) {
  if (e.ctrl && e.ctrl->done) return;
  __shared__ St7Smem sh;
  float ph[1] = {0.0f}, pl[1] = {0.0f};  // PAP: p^T (A p)
  const int tid = threadIdx.x, tx = tid % TX4, ty = tid / TX4;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const int bx = blockIdx.x * (4 * TX4), by = blockIdx.y * TY4;
  const int x0 = bx + 4 * tx, y = by + ty;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
  const int nzc = z1 - z0;
  const int np = nzc + 2;  // stage p holds plane z0 - 1 + p
  const int64_t pxy = (int64_t)nx * ny;
  const bool in = x0 < nx && y < ny;  // nx % 4 == 0: the whole vector is inside
  int issued = 0;                     // stages issued (thread 0's count)
  auto issue = [&](int p) {
    const uint32_t bar = tma::smem_addr(&sh.full[p % kS7]);
    tma::mbar_expect_tx(bar, kS7Bytes);
    tma::load_3d(tma::smem_addr(sh.u[p % kS7]), &mu, bx - 4, by - 1, z0 - 1 + p, bar);
    issued = p + 1;
  };
  if (tid == 0) {
    for (int i = 0; i < kS7; ++i) tma::mbar_init(tma::smem_addr(&sh.full[i]), 1);
    tma::mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0)
    for (int p = 0; p < min(kS7, np); ++p) issue(p);
  int waited = 0;  // stages 0 .. waited-1 have landed
  bool lost = false;
  auto wait_stage = [&](int p) {
    if (!lost && !tma::mbar_wait(tma::smem_addr(&sh.full[p % kS7]), (uint32_t)(p / kS7) & 1u))
      lost = true;
    if (!lost) waited = p + 1;
  };
  const float wc = e.wc, a1 = e.c1 * e.dinv_u, c2 = e.c2;
  const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const bool zpv_on = in && e.znext && e.zprev;
  int64_t idx = (int64_t)z0 * pxy + (int64_t)y * nx + x0;
  float4 zp = zpv_on ? __ldg(reinterpret_cast<const float4*>(e.zprev + idx)) : zero4;
  const int r = (ty + 1) * S7W + 4 + 4 * tx;  // this thread's first point in a staged plane
  wait_stage(0);
  wait_stage(1);
  bool stop = false;
  for (int i = 0; i < nzc; ++i) {
    // z_{q-1} of the next plane, requested a plane ahead
    const float4 nzp = (zpv_on && i + 1 < nzc)
                           ? __ldg(reinterpret_cast<const float4*>(e.zprev + idx + pxy))
                           : zero4;
    wait_stage(i + 2);
    // every thread is done with plane i - 1's stage: refill its slot kS7 stages ahead
    stop = __syncthreads_or(lost);
    if (stop) break;
    if (tid == 0 && i >= 1 && i - 1 + kS7 < np) issue(i - 1 + kS7);
    if (in) {
      const float* Pm = sh.u[i % kS7];
      const float* Pc = sh.u[(i + 1) % kS7];
      const float* Pp = sh.u[(i + 2) % kS7];
      const float4 uc = *reinterpret_cast<const float4*>(Pc + r);
      const float4 ym = *reinterpret_cast<const float4*>(Pc + r - S7W);
      const float4 yp = *reinterpret_cast<const float4*>(Pc + r + S7W);
      const float4 ub = *reinterpret_cast<const float4*>(Pm + r);
      const float4 ua = *reinterpret_cast<const float4*>(Pp + r);
      const float xl = Pc[r - 1], xr = Pc[r + 4];
      const float xm[4] = {xl, uc.x, uc.y, uc.z}, xp[4] = {uc.y, uc.z, uc.w, xr};
      const float c[4] = {uc.x, uc.y, uc.z, uc.w}, dn[4] = {ub.x, ub.y, ub.z, ub.w};
      const float up[4] = {ua.x, ua.y, ua.z, ua.w};
      const float yM[4] = {ym.x, ym.y, ym.z, ym.w}, yP[4] = {yp.x, yp.y, yp.z, yp.w};
      float av[4], cv[4];
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        float a;
        if constexpr (POISSON) {
          float s = (xm[l] + xp[l]) + (yM[l] + yP[l]);
          s += dn[l] + up[l];
          a = fmaf(wc, c[l], -s);
        } else {  // weights in the order -z, -y, -x, centre, +x, +y, +z
          a = e.w[0] * dn[l];
          a = fmaf(e.w[1], yM[l], a);
          a = fmaf(e.w[2], xm[l], a);
          a = fmaf(e.w[3], c[l], a);
          a = fmaf(e.w[4], xp[l], a);
          a = fmaf(e.w[5], yP[l], a);
          a = fmaf(e.w[6], up[l], a);
        }
        float cc = c[l];
        if constexpr (FIRST) {  // uniform M^{-1}: A (d r) = d (A r)
          a *= e.dinv_u;
          cc *= e.dinv_u;
        }
        av[l] = a;
        cv[l] = cc;
      }
      if constexpr (PAP) {
#pragma unroll
        for (int l = 0; l < 4; ++l) df_acc_prod(ph[0], pl[0], cv[l], av[l]);
      }
      if constexpr (FIRST) *reinterpret_cast<float4*>(e.z1 + idx) = make_float4(cv[0], cv[1], cv[2], cv[3]);
      *reinterpret_cast<float4*>(e.y + idx) = make_float4(av[0], av[1], av[2], av[3]);
      if (e.znext) {
        const float zpv[4] = {zp.x, zp.y, zp.z, zp.w};
        float zn[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) zn[l] = fmaf(a1, av[l], fmaf(-c2, cv[l], -zpv[l]));
        *reinterpret_cast<float4*>(e.znext + idx) = make_float4(zn[0], zn[1], zn[2], zn[3]);
      }
    }
    zp = nzp;
    idx += pxy;
  }
  if (stop && tid == 0) {
    // let the copies still in flight land before the CTA's shared memory is released
    for (int p = waited; p < issued; ++p)
      tma::mbar_wait(tma::smem_addr(&sh.full[p % kS7]), (uint32_t)(p / kS7) & 1u);
    if (e.ctrl) {
      e.ctrl->status = SSTEP_ERR_TIMEOUT;
      e.ctrl->done = 1;
    }
  }
  if constexpr (PAP) pap_finish(e, ph, pl);  // every thread: stop is uniform over the CTA
}

template <bool FIRST, bool SCALE, bool PAP = false>
__global__ void __launch_bounds__(kThreads) k_csrf(CsrOp A, MpkF32Args e) {
  if (e.ctrl && e.ctrl->done) return;
  float ph[1] = {0.0f}, pl[1] = {0.0f};  // PAP: p^T (A p)
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < A.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k0 = __ldg(A.rowptr + i), k1 = __ldg(A.rowptr + i + 1);
    float a = 0.0f;
    for (int64_t k = k0; k < k1; ++k) {
      const int32_t c = __ldg(A.colind + k);
      float v = __ldg(e.u + c);
      if constexpr (SCALE) v *= __ldg(e.dinv + c);
      a = fmaf(__ldg(e.valsf + k), v, a);
    }
    float uc = __ldg(e.u + i);
    if constexpr (SCALE) uc *= __ldg(e.dinv + i);
    if constexpr (FIRST && !SCALE) {
      a *= e.dinv_u;
      uc *= e.dinv_u;
    }
    mpk_f32_epilogue(e, i, a, uc, FIRST);
    if constexpr (PAP) df_acc_prod(ph[0], pl[0], uc, a);
  }
  if constexpr (PAP) pap_finish(e, ph, pl);
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

struct StencilGrid {
  dim3 grid;
  int zc;
};

StencilGrid stencil_grid(const StencilOp& op) {
  const int gx = (op.nx + TX - 1) / TX, gy = (op.ny + TY - 1) / TY;
  const int64_t txy = (int64_t)gx * gy;
  // Aim for about 16 CTAs per SM in total while keeping z chunks of >= 8 planes.
  int64_t want_z = std::max<int64_t>(1, (int64_t)num_sms() * 16 / std::max<int64_t>(1, txy));
  want_z = std::min<int64_t>(want_z, std::max(1, op.nz / 8));
  int zc = (int)((op.nz + want_z - 1) / want_z);
  if (zc < 1) zc = 1;
  if (zc > 1 && (zc & 1)) ++zc;  // the 5/7-point kernel advances two planes per iteration
  int gz = (op.nz + zc - 1) / zc;
  return {dim3(gx, gy, gz), zc};
}

// FP64 MPK step (EP_MPK, EP_MPK_FIRST) for 7-point stencils with nx even and a uniform M^{-1}:
// each thread owns two consecutive x points (16-byte loads and stores), a CTA a 64 x 8 tile of
// a z chunk, marching in z with planes z-1, z, z+1 in registers and plane z staged in shared
// memory (two buffers, one barrier per plane).  Two points share one set of index and staging
// instructions, which leaves more of the issue slots to the FP64 pipe.
constexpr int TX2 = 32, TY2 = 8;
constexpr int kRow2 = 2 * TX2 + 4;  // doubles per staged row: 2 pad | 64 values | 2 pad

template <bool POISSON, int EPI>
__global__ void __launch_bounds__(TX2 * TY2) k_stencil7_x2(StencilOp op, EpiArgs e, int gx,
                                                           int64_t items) {
  if (skip<EPI>(e)) return;
  __shared__ __align__(16) double sm[2][TY2 + 2][kRow2];
  const int tx = threadIdx.x % TX2, ty = threadIdx.x / TX2;
  const int nx = op.nx, ny = op.ny, nz = op.nz;
  const int64_t pxy = (int64_t)nx * ny;
  const double2 zero2 = make_double2(0.0, 0.0);
  double red[2] = {0.0, 0.0};  // the reducing epilogues' sums
  // this CTA's share of the (tile, z plane) items in tile-major order: one launch wave of
  // CTAs with equal shares (to a plane), marched as one or more z segments of whole tiles
  const int64_t it0 = items * blockIdx.x / gridDim.x, it1 = items * (blockIdx.x + 1) / gridDim.x;
  int set = 0;
  for (int64_t it = it0; it < it1;) {
    const int64_t tile = it / nz;
    const int z0 = (int)(it % nz);
    const int z1 = (int)std::min<int64_t>(nz, z0 + (it1 - it));
    it += z1 - z0;
    const int bx = (int)(tile % gx), by = (int)(tile / gx);
    const int x0 = (bx * TX2 + tx) * 2, y = by * TY2 + ty;
    const bool in = x0 < nx && y < ny;  // nx even: both points inside
    const int64_t col = (int64_t)y * nx + x0;
    const int hy = ty == 0 ? -1 : (ty == TY2 - 1 ? 1 : 0);
    const bool hyok = hy != 0 && x0 < nx && y + hy >= 0 && y + hy < ny;
    const int64_t hycol = col + (int64_t)hy * nx;
    const int hx = tx == 0 ? -1 : (tx == TX2 - 1 ? 2 : 0);
    const bool hxok = hx != 0 && y < ny && x0 + hx >= 0 && x0 + hx < nx;
    const int64_t hxcol = col + hx;
    auto ld2 = [&](int64_t c, int zz, bool ok) -> double2 {
      if (!ok || zz < 0 || zz >= nz) return zero2;
      return __ldg(reinterpret_cast<const double2*>(e.u + c + (int64_t)zz * pxy));
    };
    auto ld1 = [&](int64_t c, int zz, bool ok) -> double {
      if (!ok || zz < 0 || zz >= nz) return 0.0;
      return __ldg(e.u + c + (int64_t)zz * pxy);
    };
    double2 ub = ld2(col, z0 - 1, in), uc = ld2(col, z0, in), ua = ld2(col, z0 + 1, in);
    double2 hyv = ld2(hycol, z0, hyok);
    double hxv = ld1(hxcol, z0, hxok);
    for (int z = z0; z < z1; ++z) {
      double (*P)[kRow2] = sm[set];
      *reinterpret_cast<double2*>(&P[ty + 1][2 + 2 * tx]) = uc;
      if (hy) *reinterpret_cast<double2*>(&P[ty + 1 + hy][2 + 2 * tx]) = hyv;
      if (hx < 0) P[ty + 1][1] = hxv;
      if (hx > 0) P[ty + 1][2 + 2 * TX2] = hxv;
      const double2 nz2 = ld2(col, z + 2, in);
      const double2 nhy = ld2(hycol, z + 1, hyok);
      const double nhx = ld1(hxcol, z + 1, hxok);
      __syncthreads();
      if (in) {
        const double2 ym = *reinterpret_cast<const double2*>(&P[ty][2 + 2 * tx]);
        const double2 yp = *reinterpret_cast<const double2*>(&P[ty + 2][2 + 2 * tx]);
        const double xl = P[ty + 1][1 + 2 * tx], xr = P[ty + 1][4 + 2 * tx];
        const double xm[2] = {xl, uc.x}, xp[2] = {uc.y, xr};
        const double c[2] = {uc.x, uc.y}, dn[2] = {ub.x, ub.y}, up[2] = {ua.x, ua.y};
        const double yM[2] = {ym.x, ym.y}, yP[2] = {yp.x, yp.y};
        double av[2], cv[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
          double a;
          if constexpr (POISSON) {
            double s = (xm[l] + xp[l]) + (yM[l] + yP[l]);
            s += dn[l] + up[l];
            a = fma(op.wc, c[l], -s);
          } else {  // weights in the order -z, -y, -x, centre, +x, +y, +z
            a = op.w[0] * dn[l];
            a = fma(op.w[1], yM[l], a);
            a = fma(op.w[2], xm[l], a);
            a = fma(op.w[3], c[l], a);
            a = fma(op.w[4], xp[l], a);
            a = fma(op.w[5], yP[l], a);
            a = fma(op.w[6], up[l], a);
          }
          double cc = c[l];
          if constexpr (EPI == EP_MPK_FIRST) {  // uniform M^{-1}: A (d r) = d (A r)
            a *= e.M.dinv_u;
            cc *= e.M.dinv_u;
          }
          av[l] = a;
          cv[l] = cc;
        }
        const int64_t i = (int64_t)z * pxy + col;
        if constexpr (EPI == EP_MPK || EPI == EP_MPK_FIRST) {
          if constexpr (EPI == EP_MPK_FIRST) *reinterpret_cast<double2*>(e.z1 + i) = make_double2(cv[0], cv[1]);
          *reinterpret_cast<double2*>(e.y + i) = make_double2(av[0], av[1]);
          if (e.znext) {
            double2 zp = zero2;
            if (e.zprev) zp = __ldg(reinterpret_cast<const double2*>(e.zprev + i));
            const double t0 = e.c3 == 1.0 ? -zp.x : -e.c3 * zp.x;
            const double t1 = e.c3 == 1.0 ? -zp.y : -e.c3 * zp.y;
            *reinterpret_cast<double2*>(e.znext + i) =
                make_double2(fma(e.a1u, av[0], fma(-e.c2, cv[0], t0)),
                             fma(e.a1u, av[1], fma(-e.c2, cv[1], t1)));
          }
        } else {  // the other epilogues, point by point (PCG product, residuals)
          epilogue<EPI>(e, i, av[0], cv[0], red);
          epilogue<EPI>(e, i + 1, av[1], cv[1], red);
        }
      }
      ub = uc;
      uc = ua;
      ua = nz2;
      hyv = nhy;
      hxv = nhx;
      set ^= 1;
    }
  }
  reduce_and_finish<EPI>(e, red);
}

template <int EPI, bool SCALE>
cudaError_t launch_stencil(const StencilOp& op, const EpiArgs& e, cudaStream_t st) {
  // the middle MPK steps (with its three outputs the first step runs faster in the scalar
  // kernel), the PCG product and the residuals
  if constexpr ((EPI == EP_MPK || EPI == EP_PCG_AP || EPI == EP_RR || EPI == EP_RESID ||
                 EPI == EP_TRUERES) && !SCALE) {
    auto a16 = [](const void* p) { return ((uintptr_t)p & 15) == 0; };  // null passes
    const bool aligned = a16(e.u) && a16(e.y) && a16(e.znext) && a16(e.zprev) && a16(e.z1);
    if (op.points == 7 && op.nx % 2 == 0 && (EPI != EP_MPK || e.M.dinv == nullptr) && aligned) {
      // one wave: the SM count times the resident CTAs per SM, each with an equal share of
      // the (tile, plane) items (at least 8 planes per CTA)
      const int gx = (op.nx + 2 * TX2 - 1) / (2 * TX2), gy = (op.ny + TY2 - 1) / TY2;
      const int64_t items = (int64_t)gx * gy * op.nz;
      auto wave = [&](auto kernel, int& per_sm) -> int {
        if (!per_sm &&
            (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, TX2 * TY2, 0) !=
                 cudaSuccess ||
             per_sm < 1))
          per_sm = 1;
        return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * per_sm, items / 8));
      };
      static int occ_p = 0, occ_g = 0;
      if (op.poisson) {
        const int ctas = wave(k_stencil7_x2<true, EPI>, occ_p);
        k_stencil7_x2<true, EPI><<<ctas, TX2 * TY2, 0, st>>>(op, e, gx, items);
      } else {
        const int ctas = wave(k_stencil7_x2<false, EPI>, occ_g);
        k_stencil7_x2<false, EPI><<<ctas, TX2 * TY2, 0, st>>>(op, e, gx, items);
      }
      return cudaGetLastError();
    }
  }
  StencilGrid g = stencil_grid(op);
  const int threads = TX * TY;
  if (op.points == 27) {
    if (op.poisson) k_stencil27<true, EPI, SCALE><<<g.grid, threads, 0, st>>>(op, e, g.zc);
    else k_stencil27<false, EPI, SCALE><<<g.grid, threads, 0, st>>>(op, e, g.zc);
  } else if (op.points == 7) {
    if (op.poisson) k_stencil7<7, true, EPI, SCALE><<<g.grid, threads, 0, st>>>(op, e, g.zc);
    else k_stencil7<7, false, EPI, SCALE><<<g.grid, threads, 0, st>>>(op, e, g.zc);
  } else {
    if (op.poisson) k_stencil7<5, true, EPI, SCALE><<<g.grid, threads, 0, st>>>(op, e, g.zc);
    else k_stencil7<5, false, EPI, SCALE><<<g.grid, threads, 0, st>>>(op, e, g.zc);
  }
  return cudaGetLastError();
}

int csr_ctas(int64_t n) {
  int64_t want = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * kCsrCtasPerSm));
}

template <int EPI, bool SCALE>
cudaError_t launch_csr(const CsrOp& A, const EpiArgs& e, cudaStream_t st) {
  k_csr<EPI, SCALE><<<csr_ctas(A.n), kThreads, 0, st>>>(A, e);
  return cudaGetLastError();
}

template <int EPI>
cudaError_t dispatch(const OpDesc& A, const EpiArgs& e, cudaStream_t st) {
  // Per-entry scaling by M^{-1} is needed only when the first MPK step applies a
  // non-uniform M^{-1} before the operator.
  const bool scale = (EPI == EP_MPK_FIRST) && e.M.dinv != nullptr;
  if (A.kind == SSTEP_MATRIX_STENCIL) {
    return scale ? launch_stencil<EPI, true>(A.st, e, st) : launch_stencil<EPI, false>(A.st, e, st);
  }
  return scale ? launch_csr<EPI, true>(A.csr, e, st) : launch_csr<EPI, false>(A.csr, e, st);
}

}  // namespace

int operator_grid_ctas(const OpDesc& A) {
  if (A.kind == SSTEP_MATRIX_Q1) return q1_grid_ctas(A.q1);
  if (A.kind == SSTEP_MATRIX_STENCIL) {
    StencilGrid g = stencil_grid(A.st);
    return (int)(g.grid.x * g.grid.y * g.grid.z);
  }
  return csr_ctas(A.csr.n);
}

cudaError_t launch_operator(const OpDesc& A, const EpiArgs& e, cudaStream_t st) {
  if (A.kind == SSTEP_MATRIX_Q1) return launch_q1_operator(A.q1, e, st);
  switch (e.epi) {
    case EP_SPMV: return dispatch<EP_SPMV>(A, e, st);
    case EP_MPK: return dispatch<EP_MPK>(A, e, st);
    case EP_MPK_FIRST: return dispatch<EP_MPK_FIRST>(A, e, st);
    case EP_RESID: return dispatch<EP_RESID>(A, e, st);
    case EP_POWER: return dispatch<EP_POWER>(A, e, st);
    case EP_PCG_AP: return dispatch<EP_PCG_AP>(A, e, st);
    case EP_TRUERES: return dispatch<EP_TRUERES>(A, e, st);
    case EP_RR: return dispatch<EP_RR>(A, e, st);
    default: return cudaErrorInvalidValue;
  }
}

struct St7TmaMaps {
  int ncols;
  const float* col[kS7MaxCols];
  CUtensorMap mu[kS7MaxCols];
};

namespace {

// The tensor map of the vector u, or null when u has none.
const CUtensorMap* st7_map(const StencilOp& op, const float* u) {
  if (!op.tma) return nullptr;
  for (int c = 0; c < op.tma->ncols; ++c)
    if (op.tma->col[c] == u) return &op.tma->mu[c];
  return nullptr;
}

// One wave of resident CTAs, each marching a z chunk of at least 8 planes: the pipeline fill
// is paid once per CTA.
template <bool POISSON, bool FIRST, bool PAP>
cudaError_t launch_st7_tma(const CUtensorMap* m, const StencilOp& op, const MpkF32Args& e,
                           cudaStream_t st) {
  static int per_sm = 0;
  if (!per_sm) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, k_stencil7f4_tma<POISSON, FIRST, PAP>, TX4 * TY4, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  const int gx = (op.nx + 4 * TX4 - 1) / (4 * TX4), gy = (op.ny + TY4 - 1) / TY4;
  int64_t gz = std::max<int64_t>(1, (int64_t)num_sms() * per_sm / std::max(1, gx * gy));
  gz = std::min<int64_t>(gz, std::max(1, op.nz / 8));
  const int zc = (int)((op.nz + gz - 1) / gz);
  const dim3 grid(gx, gy, (op.nz + zc - 1) / zc);
  k_stencil7f4_tma<POISSON, FIRST, PAP><<<grid, TX4 * TY4, 0, st>>>(*m, op, e, zc);
  return cudaGetLastError();
}

}  // namespace

St7TmaMaps* st7_tma_build(const StencilOp& op, const float* const* cols, int ncols) {
  // rows must be 16-byte multiples (nx % 4 == 0); boxes no larger than the grid
  if (op.points != 7 || op.nx % 4 != 0 || op.nx < S7W || op.ny < S7H || ncols < 1 ||
      ncols > kS7MaxCols)
    return nullptr;
  auto* m = new St7TmaMaps{};
  m->ncols = ncols;
  bool ok = true;
  for (int c = 0; ok && c < ncols; ++c) {
    m->col[c] = cols[c];
    ok = tma::encode_3d(&m->mu[c], cols[c], (uint64_t)op.nx, (uint64_t)op.ny, (uint64_t)op.nz,
                        (uint64_t)op.nx, S7W, S7H);
  }
  if (!ok) {
    delete m;
    return nullptr;
  }
  return m;
}

void st7_tma_free(St7TmaMaps* m) { delete m; }

cudaError_t launch_mpk_f32(const OpDesc& A, const MpkF32Args& e, cudaStream_t st) {
  if (e.pap) {  // FP32 PCG product step: y = A p with p^T A p (no recurrence)
    if (e.first || e.znext || !e.ctrl || !e.partials) return cudaErrorInvalidValue;
    if (A.kind == SSTEP_MATRIX_STENCIL) {
      const StencilOp& op = A.st;
      if (op.points == 27) return cudaErrorNotSupported;
      if (const CUtensorMap* m = op.points == 7 ? st7_map(op, e.u) : nullptr) {
        if (op.poisson) return launch_st7_tma<true, false, true>(m, op, e, st);
        return launch_st7_tma<false, false, true>(m, op, e, st);
      }
      if (op.points == 7 && op.nx % 4 == 0) {
        const int gx = (op.nx + 4 * TX4 - 1) / (4 * TX4), gy = (op.ny + TY4 - 1) / TY4;
        int64_t gz = std::max<int64_t>(1, (int64_t)num_sms() * 4 / std::max(1, gx * gy));
        gz = std::min<int64_t>(gz, std::max(1, op.nz / 8));
        const int zc = (int)((op.nz + gz - 1) / gz);
        const dim3 grid(gx, gy, (op.nz + zc - 1) / zc);
        if (op.poisson) k_stencil7f4<true, false, true><<<grid, TX4 * TY4, 0, st>>>(op, e, zc);
        else k_stencil7f4<false, false, true><<<grid, TX4 * TY4, 0, st>>>(op, e, zc);
        return cudaGetLastError();
      }
      StencilGrid g = stencil_grid(op);
      const int threads = TX * TY;
      if (op.points == 7) {
        if (op.poisson) k_stencil7f<7, true, false, false, true><<<g.grid, threads, 0, st>>>(op, e, g.zc);
        else k_stencil7f<7, false, false, false, true><<<g.grid, threads, 0, st>>>(op, e, g.zc);
      } else {
        if (op.poisson) k_stencil7f<5, true, false, false, true><<<g.grid, threads, 0, st>>>(op, e, g.zc);
        else k_stencil7f<5, false, false, false, true><<<g.grid, threads, 0, st>>>(op, e, g.zc);
      }
      return cudaGetLastError();
    }
    if (A.kind == SSTEP_MATRIX_CSR) {
      k_csrf<false, false, true><<<csr_ctas(A.csr.n), kThreads, 0, st>>>(A.csr, e);
      return cudaGetLastError();
    }
    if (A.kind == SSTEP_MATRIX_Q1) return launch_q1_mpk_f32(A.q1, e, st);
    return cudaErrorNotSupported;
  }
  if (A.kind == SSTEP_MATRIX_Q1) return launch_q1_mpk_f32(A.q1, e, st);
  const bool scale = e.first && e.dinv != nullptr;
  if (A.kind == SSTEP_MATRIX_STENCIL) {
    const StencilOp& op = A.st;
    if (op.points == 27) return cudaErrorNotSupported;  // the mixed path takes 27 points as CSR
    const CUtensorMap* m = op.points == 7 && e.dinv == nullptr ? st7_map(op, e.u) : nullptr;
    if (m) {
      if (e.first) {
        if (op.poisson) return launch_st7_tma<true, true, false>(m, op, e, st);
        return launch_st7_tma<false, true, false>(m, op, e, st);
      }
      if (op.poisson) return launch_st7_tma<true, false, false>(m, op, e, st);
      return launch_st7_tma<false, false, false>(m, op, e, st);
    }
    if (op.points == 7 && op.nx % 4 == 0 && !scale && e.dinv == nullptr) {
      // vector kernel: about four 256-thread CTAs per SM, z chunks of at least 8 planes
      const int gx = (op.nx + 4 * TX4 - 1) / (4 * TX4), gy = (op.ny + TY4 - 1) / TY4;
      int64_t gz = std::max<int64_t>(1, (int64_t)num_sms() * 4 / std::max(1, gx * gy));
      gz = std::min<int64_t>(gz, std::max(1, op.nz / 8));
      const int zc = (int)((op.nz + gz - 1) / gz);
      const dim3 grid(gx, gy, (op.nz + zc - 1) / zc);
      if (e.first) {
        if (op.poisson) k_stencil7f4<true, true><<<grid, TX4 * TY4, 0, st>>>(op, e, zc);
        else k_stencil7f4<false, true><<<grid, TX4 * TY4, 0, st>>>(op, e, zc);
      } else {
        if (op.poisson) k_stencil7f4<true, false><<<grid, TX4 * TY4, 0, st>>>(op, e, zc);
        else k_stencil7f4<false, false><<<grid, TX4 * TY4, 0, st>>>(op, e, zc);
      }
      return cudaGetLastError();
    }
    StencilGrid g = stencil_grid(op);
    const int threads = TX * TY;
#define L7(P, POI)                                                                           \
  do {                                                                                       \
    if (e.first) {                                                                           \
      if (scale) k_stencil7f<P, POI, true, true><<<g.grid, threads, 0, st>>>(op, e, g.zc);    \
      else k_stencil7f<P, POI, true, false><<<g.grid, threads, 0, st>>>(op, e, g.zc);         \
    } else {                                                                                 \
      k_stencil7f<P, POI, false, false><<<g.grid, threads, 0, st>>>(op, e, g.zc);             \
    }                                                                                        \
  } while (0)
    if (op.points == 7) {
      if (op.poisson) L7(7, true);
      else L7(7, false);
    } else {
      if (op.poisson) L7(5, true);
      else L7(5, false);
    }
#undef L7
    return cudaGetLastError();
  }
  const int grid = csr_ctas(A.csr.n);
  if (e.first) {
    if (scale) k_csrf<true, true><<<grid, kThreads, 0, st>>>(A.csr, e);
    else k_csrf<true, false><<<grid, kThreads, 0, st>>>(A.csr, e);
  } else {
    k_csrf<false, false><<<grid, kThreads, 0, st>>>(A.csr, e);
  }
  return cudaGetLastError();
}

}  // namespace sstep
