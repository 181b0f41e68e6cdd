// k_adjoint.cu -- device kernels of the differentiated Q1 diffusion solve: the conductivity
// field from the log-conductivity, the assembled CSR values of the Q1 operator as a function
// of the conductivities, and the gradient of a loss with respect to the conductivities (or
// their logarithms) from the adjoint solution.
//
// The operator: trilinear (Q1) finite elements on unit cells, one conductivity kappa_c per
// cell (cell cx + (nx+1)(cy + (ny+1) cz)), unknowns at the nx*ny*nz interior vertices (vertex
// i + nx (j + ny k) sits at grid point (i+1, j+1, k+1)), Dirichlet boundary vertices
// eliminated.  A = sum_c kappa_c P_c^T K_ref P_c with the 8 x 8 element stiffness
// K_ref = K1 x M1 x M1 + M1 x K1 x M1 + M1 x M1 x K1 (K1 = [[1,-1],[-1,1]],
// M1 = [[1,1/2],[1/2,1]]/3; local vertex lx + 2 ly + 4 lz).  For x = A^{-1} b and a loss L(x),
// with the adjoint A^T lambda = dL/dx (A is symmetric):
//   dL/dkappa_c = -lambda_c^T K_ref x_c        (lambda_c, x_c: the cell's 8 vertex values,
//                                               0 at boundary vertices),
//   dL/dtheta_c = kappa_c dL/dkappa_c          for kappa = exp(theta).
// The paper has no differentiated form; this is the adjoint of a linear solve.
#include <algorithm>

#include "common.cuh"

namespace sstep {

namespace {

// K_ref[a][b], formed in the same operation order as the input generator's Kronecker products
// ((Mz My) Kx + (Mz Ky) Mx) + (Kz My) Mx, with rounded multiplies and adds (no contraction),
// so that assembled values agree with the generator's bit for bit.
__device__ __forceinline__ double kref(int a, int b) {
  const double third = 1.0 / 3.0, sixth = 0.5 / 3.0;
  const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
  const int bx = b & 1, by = (b >> 1) & 1, bz = b >> 2;
  const double Mx = ax == bx ? third : sixth, My = ay == by ? third : sixth,
               Mz = az == bz ? third : sixth;
  const double Kx = ax == bx ? 1.0 : -1.0, Ky = ay == by ? 1.0 : -1.0, Kz = az == bz ? 1.0 : -1.0;
  const double t1 = __dmul_rn(__dmul_rn(Mz, My), Kx);
  const double t2 = __dmul_rn(__dmul_rn(Mz, Ky), Mx);
  const double t3 = __dmul_rn(__dmul_rn(Kz, My), Mx);
  return __dadd_rn(__dadd_rn(t1, t2), t3);
}

__global__ void __launch_bounds__(kThreads) k_q1_exp(int64_t ncell, const double* theta,
                                                     double* kappa) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x)
    kappa[c] = exp(__ldg(theta + c));
}

// One thread per row: entry (i, j) = sum over the cells shared by vertices i and j of
// kappa_c K_ref[l_i, l_j], the cells visited in the input generator's order (x offset outer,
// then y, then z; lower corner offsets -1 before 0).  *bad is set when a column is not one of
// the 27 neighbours of its row.
__global__ void __launch_bounds__(kThreads) k_q1_assemble(int nx, int ny, int nz,
                                                          const double* kappa, int64_t n,
                                                          const int64_t* rowptr,
                                                          const int32_t* colind, double* vals,
                                                          int* bad) {
  const int64_t cx1 = nx + 1, cxy = (int64_t)(nx + 1) * (ny + 1);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((int64_t)nx * ny));
    for (int64_t k = __ldg(rowptr + i); k < __ldg(rowptr + i + 1); ++k) {
      const int64_t j = __ldg(colind + k);
      const int jx = (int)(j % nx), jy = (int)((j / nx) % ny), jz = (int)(j / ((int64_t)nx * ny));
      const int dx = jx - ix, dy = jy - iy, dz = jz - iz;
      if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) {
        atomicExch(bad, 1);
        vals[k] = 0.0;
        continue;
      }
      double v = 0.0;
      for (int ox = -1; ox <= 0; ++ox)
        for (int oy = -1; oy <= 0; ++oy)
          for (int oz = -1; oz <= 0; ++oz) {
            const int lvx = -ox, lvy = -oy, lvz = -oz;  // vertex i in the cell
            const int lwx = lvx + dx, lwy = lvy + dy, lwz = lvz + dz;
            if (lwx < 0 || lwx > 1 || lwy < 0 || lwy > 1 || lwz < 0 || lwz > 1) continue;
            const int64_t cell = (int64_t)(iz + 1 + oz) * cxy + (int64_t)(iy + 1 + oy) * cx1 +
                                 (ix + 1 + ox);
            const double kv = kref(lvx + 2 * lvy + 4 * lvz, lwx + 2 * lwy + 4 * lwz);
            v = __dadd_rn(v, __dmul_rn(kv, __ldg(kappa + cell)));
          }
      vals[k] = v;
    }
  }
}

// One thread per cell: g_c = -lambda_c^T K_ref x_c (times kappa_c for the log-conductivity).
__global__ void __launch_bounds__(kThreads) k_q1_grad(int nx, int ny, int nz, const double* kappa,
                                                      const double* lam, const double* x,
                                                      double* grad, int wrt_log,
                                                      int accumulate) {
  __shared__ double K[64];
  for (int e = threadIdx.x; e < 64; e += blockDim.x) K[e] = kref(e >> 3, e & 7);
  __syncthreads();
  const int64_t cx1 = nx + 1, cy1 = ny + 1;
  const int64_t ncell = cx1 * cy1 * (nz + 1);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int cx = (int)(c % cx1), cy = (int)((c / cx1) % cy1), cz = (int)(c / (cx1 * cy1));
    double lv[8], xv[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      // corner (lx, ly, lz) of cell (cx, cy, cz) is grid point (cx+lx, ...), interior vertex
      // (cx+lx-1, ...) when inside 0..n-1 on every axis
      const int vx = cx + (a & 1) - 1, vy = cy + ((a >> 1) & 1) - 1, vz = cz + (a >> 2) - 1;
      const bool in = vx >= 0 && vx < nx && vy >= 0 && vy < ny && vz >= 0 && vz < nz;
      const int64_t v = ((int64_t)vz * ny + vy) * nx + vx;
      lv[a] = in ? __ldg(lam + v) : 0.0;
      xv[a] = in ? __ldg(x + v) : 0.0;
    }
    double g = 0.0;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      double kx = 0.0;
#pragma unroll
      for (int b = 0; b < 8; ++b) kx = fma(K[a * 8 + b], xv[b], kx);
      g = fma(lv[a], kx, g);
    }
    g = -g;
    if (wrt_log) g *= __ldg(kappa + c);
    grad[c] = accumulate ? grad[c] + g : g;
  }
}

// One CTA per problem p: out[2p] = lam_p^T x_p and out[2p+1] = lam_p^T (N x_p), N the sum of
// the six axis neighbours inside the grid (the off-diagonal part of a 7-point stencil with unit
// weights).  For A = wc I + wo N, dA/dwc = I and dA/dwo = N.  Fixed-order block reduction.
__global__ void __launch_bounds__(kThreads) k_stencil7_bilinear(const Bil7Prob* probs,
                                                                 double* out) {
  const Bil7Prob p = probs[blockIdx.x];
  const int64_t pxy = (int64_t)p.nx * p.ny, n = pxy * p.nz;
  double v[2] = {0.0, 0.0};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const int ix = (int)(i % p.nx), iy = (int)((i / p.nx) % p.ny), iz = (int)(i / pxy);
    double nb = 0.0;
    if (ix > 0) nb += __ldg(p.x + i - 1);
    if (ix + 1 < p.nx) nb += __ldg(p.x + i + 1);
    if (iy > 0) nb += __ldg(p.x + i - p.nx);
    if (iy + 1 < p.ny) nb += __ldg(p.x + i + p.nx);
    if (iz > 0) nb += __ldg(p.x + i - pxy);
    if (iz + 1 < p.nz) nb += __ldg(p.x + i + pxy);
    const double l = __ldg(p.lam + i);
    v[0] = fma(l, __ldg(p.x + i), v[0]);
    v[1] = fma(l, nb, v[1]);
  }
  __shared__ double sh[2 * 32];
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = v[0];
    out[2 * blockIdx.x + 1] = v[1];
  }
}

// out[g * w + k] = scale * sum_{r < per} in[(g * per + r) * w + k], r in increasing order.
__global__ void k_sum_groups(const double* in, int groups, int per, int w, double scale,
                             double* out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < groups * w; e += gridDim.x * blockDim.x) {
    const int g = e / w, k = e % w;
    double v = 0.0;
    for (int r = 0; r < per; ++r) v += in[((int64_t)g * per + r) * w + k];
    out[e] = scale * v;
  }
}

int grid_for(int64_t n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  const int64_t need = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 8));
}

}  // namespace

cudaError_t launch_q1_exp(int64_t ncell, const double* theta, double* kappa, cudaStream_t st) {
  k_q1_exp<<<grid_for(ncell), kThreads, 0, st>>>(ncell, theta, kappa);
  return cudaGetLastError();
}

cudaError_t launch_q1_assemble(int nx, int ny, int nz, const double* kappa, int64_t n,
                               const int64_t* rowptr, const int32_t* colind, double* vals,
                               int* bad, cudaStream_t st) {
  k_q1_assemble<<<grid_for(n), kThreads, 0, st>>>(nx, ny, nz, kappa, n, rowptr, colind, vals, bad);
  return cudaGetLastError();
}

cudaError_t launch_stencil7_bilinear(const Bil7Prob* probs_dev, int nprob, double* out,
                                     cudaStream_t st) {
  k_stencil7_bilinear<<<nprob, kThreads, 0, st>>>(probs_dev, out);
  return cudaGetLastError();
}

cudaError_t launch_sum_groups(const double* in, int groups, int per, int w, double scale,
                              double* out, cudaStream_t st) {
  const int total = groups * w;
  k_sum_groups<<<std::max(1, (total + kThreads - 1) / kThreads), kThreads, 0, st>>>(
      in, groups, per, w, scale, out);
  return cudaGetLastError();
}

cudaError_t launch_q1_grad(int nx, int ny, int nz, const double* kappa, const double* lam,
                           const double* x, double* grad, int wrt_log, int accumulate,
                           cudaStream_t st) {
  const int64_t ncell = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  k_q1_grad<<<grid_for(ncell), kThreads, 0, st>>>(nx, ny, nz, kappa, lam, x, grad, wrt_log,
                                                  accumulate);
  return cudaGetLastError();
}

}  // namespace sstep
