// k_q1.cu -- the Q1 (trilinear finite-element) diffusion operator, matrix-free from the
// per-cell conductivities: y = A u with the same fused epilogues as the stencil and CSR
// kernels (one Matrix-Powers-Kernel step of Algorithm 2, residuals, power-method step, PCG
// product), in FP64, and the FP32 MPK step of the FP32-basis path.
//
// Operator.  The element stiffness of the unit cube with conductivity kappa_e is
// kappa_e (K1 x M1 x M1 + M1 x K1 x M1 + M1 x M1 x K1) (K1 = [[1,-1],[-1,1]],
// M1 = [[1/3,1/6],[1/6,1/3]]): 1/3 on the diagonal, 0 between corners one edge apart, -1/12
// between corners two or three edges apart.  Summed over the eight cells around an interior
// vertex v:
//   a_vv = (1/3) sum of the 8 kappa,
//   face diagonal (two offsets of +-1): -(1/12) (sum of the 2 kappa sharing that face diagonal),
//   body diagonal (three offsets of +-1): -(1/12) (kappa of the one cell between them),
//   axis neighbours: 0.
// So a row holds 21 entries.  The FP32 MPK step forms them on the fly and reads one
// conductivity per cell and one value per vertex (8 bytes per vertex) where the assembled CSR
// matrix reads about 170; the FP64 kernels, bound by the FP64 pipe rather than by HBM, read
// the 13 vertex coefficients the set-up pass stored (22 FP64 operations per vertex, not 38).
//
// Tiling.  A CTA owns 32 x 8 vertices of the xy plane and marches through a chunk of z planes:
// u planes z-1, z, z+1 (one-vertex xy halo) and cell planes z, z+1 are staged in shared memory
// (four u slots and three cell slots, so one barrier per plane suffices), and the next plane is
// loaded into registers before the arithmetic of the current one.  The middle steps of the
// FP32 MPK (the bulk of the FP32-basis solve) instead bring every plane in with tensor-memory-
// accelerator copies several planes ahead (k_q1f_tma), when the grid allows it.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "common.cuh"
#include "epilogue.cuh"
#include "tma.cuh"

namespace sstep {

namespace {

constexpr int QX = 32, QY = 8, QT = QX * QY;  // vertex tile, threads per CTA
constexpr int UW = QX + 2, UH = QY + 2;       // staged u plane with its halo
constexpr int KW = QX + 1, KH = QY + 1;       // staged cell plane (cells x0..x0+QX)
constexpr int kUPer = (UW * UH + QT - 1) / QT;  // staged u values per thread
constexpr int kKPer = (KW * KH + QT - 1) / QT;  // staged conductivities per thread

// The library's Q1 operator data is one FP64 allocation: the (nx+1)(ny+1)(nz+1) conductivities,
// then (from this offset, 256-byte aligned) 13 arrays of n vertex coefficients written by the
// set-up pass (k_q1_setup) and read by the FP64 operator kernels: k = 0..3 the face diagonals
// with dz = 0 at (dx, dy) = (-1,-1), (1,-1), (-1,1), (1,1); k = 4..7 those with dy = 0 at
// (dx, dz); k = 8..11 those with dx = 0 at (dy, dz), each -1/12 of the two conductivities that
// share the diagonal; k = 12: a_vv = (1/3) sum of the eight around v.
__host__ __device__ __forceinline__ int64_t q1_coef_offset(const Q1Op& A) {
  const int64_t ncell = (int64_t)(A.nx + 1) * (A.ny + 1) * (A.nz + 1);
  return (ncell + 31) / 32 * 32;
}

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmaT(float a, float b, float c) { return fmaf(a, b, c); }

template <typename T>
struct Q1Smem {
  T u[4][UH * UW];
  T k[3][KH * KW];
};

// (A u)_v from the staged planes.  Um, Uc, Up: u planes z-1, z, z+1; K0, K1: cell planes z and
// z+1 (the cells below and above the vertex plane).  Cell (a, b, c) of the vertex is
// (x + a, y + b, z + c): the neighbour at offset (dx, dy, dz) lies in the cells with
// a = (dx + 1) / 2 (any a when dx = 0), and so on.
template <typename T>
__device__ __forceinline__ T q1_vertex(const T* Um, const T* Uc, const T* Up, const T* K0,
                                       const T* K1, int tx, int ty, T& uc) {
  auto U = [&](const T* P, int dx, int dy) -> T { return P[(ty + 1 + dy) * UW + tx + 1 + dx]; };
  auto C = [&](const T* P, int a, int b) -> T { return P[(ty + b) * KW + tx + a]; };
  const T k000 = C(K0, 0, 0), k100 = C(K0, 1, 0), k010 = C(K0, 0, 1), k110 = C(K0, 1, 1);
  const T k001 = C(K1, 0, 0), k101 = C(K1, 1, 0), k011 = C(K1, 0, 1), k111 = C(K1, 1, 1);
  // face-diagonal couplings: the two cells that share each diagonal
  const T z00 = k000 + k001, z10 = k100 + k101, z01 = k010 + k011, z11 = k110 + k111;  // dz = 0
  const T y00 = k000 + k010, y10 = k100 + k110, y01 = k001 + k011, y11 = k101 + k111;  // dy = 0
  const T x00 = k000 + k100, x10 = k010 + k110, x01 = k001 + k101, x11 = k011 + k111;  // dx = 0
  const T k8 = (z00 + z10) + (z01 + z11);
  T s = z00 * U(Uc, -1, -1);
  s = fmaT(z10, U(Uc, 1, -1), s);
  s = fmaT(z01, U(Uc, -1, 1), s);
  s = fmaT(z11, U(Uc, 1, 1), s);
  s = fmaT(y00, U(Um, -1, 0), s);
  s = fmaT(y10, U(Um, 1, 0), s);
  s = fmaT(y01, U(Up, -1, 0), s);
  s = fmaT(y11, U(Up, 1, 0), s);
  s = fmaT(x00, U(Um, 0, -1), s);
  s = fmaT(x10, U(Um, 0, 1), s);
  s = fmaT(x01, U(Up, 0, -1), s);
  s = fmaT(x11, U(Up, 0, 1), s);
  s = fmaT(k000, U(Um, -1, -1), s);
  s = fmaT(k100, U(Um, 1, -1), s);
  s = fmaT(k010, U(Um, -1, 1), s);
  s = fmaT(k110, U(Um, 1, 1), s);
  s = fmaT(k001, U(Up, -1, -1), s);
  s = fmaT(k101, U(Up, 1, -1), s);
  s = fmaT(k011, U(Up, -1, 1), s);
  s = fmaT(k111, U(Up, 1, 1), s);
  uc = U(Uc, 0, 0);
  const T third = T(1) / T(3), twelfth = T(1) / T(12);
  return fmaT(k8 * third, uc, -(s * twelfth));
}

// The z march shared by the FP64 and FP32 kernels.  load_u(idx) returns the (possibly
// M^{-1}-scaled) input at vertex idx; vertex(Um, Uc, Up, K0, K1, tx, ty, i, uc) forms (A u)_i
// from the staged planes; at(i, y, uc, in) consumes the vertex of plane z.
template <typename T, class LoadU, class Vertex, class At>
__device__ __forceinline__ void q1_march(const Q1Op& A, const T* __restrict__ kap, int kpitch,
                                         int zc, Q1Smem<T>& sh, LoadU load_u, Vertex vertex,
                                         At at) {
  const int tid = threadIdx.x, tx = tid % QX, ty = tid / QX;
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const int x0 = blockIdx.x * QX, y0 = blockIdx.y * QY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
  const int64_t pxy = (int64_t)nx * ny;
  const int64_t cpxy = (int64_t)kpitch * (ny + 1);
  // the staged elements of this thread: u tile element j = tid + p QT, cell tile likewise
  int64_t uoff[kUPer], koff[kKPer];
  bool uok[kUPer], kok[kKPer];
#pragma unroll
  for (int p = 0; p < kUPer; ++p) {
    const int j = tid + p * QT;
    const int gx = x0 - 1 + j % UW, gy = y0 - 1 + j / UW;
    uok[p] = j < UW * UH && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    uoff[p] = (int64_t)gy * nx + gx;
  }
#pragma unroll
  for (int p = 0; p < kKPer; ++p) {
    const int j = tid + p * QT;
    const int cx = x0 + j % KW, cy = y0 + j / KW;
    kok[p] = j < KW * KH && cx <= nx && cy <= ny;
    koff[p] = (int64_t)cy * kpitch + cx;
  }
  auto ldu = [&](int p, int zz) -> T {
    if (!uok[p] || zz < 0 || zz >= nz) return T(0);
    return load_u(uoff[p] + (int64_t)zz * pxy);
  };
  auto ldk = [&](int p, int cz) -> T {
    if (!kok[p] || cz > nz) return T(0);
    return __ldg(kap + koff[p] + (int64_t)cz * cpxy);
  };
  auto put_u = [&](int slot, int p, T v) {
    const int j = tid + p * QT;
    if (j < UW * UH) sh.u[slot][j] = v;
  };
  auto put_k = [&](int slot, int p, T v) {
    const int j = tid + p * QT;
    if (j < KW * KH) sh.k[slot][j] = v;
  };
  // u plane zz lives in slot (zz - z0 + 1) & 3, cell plane cz in slot (cz - z0) % 3
  T nu[kUPer], nk[kKPer];
#pragma unroll
  for (int p = 0; p < kUPer; ++p) {
    put_u(0, p, ldu(p, z0 - 1));
    put_u(1, p, ldu(p, z0));
    nu[p] = ldu(p, z0 + 1);
  }
#pragma unroll
  for (int p = 0; p < kKPer; ++p) {
    put_k(0, p, ldk(p, z0));
    nk[p] = ldk(p, z0 + 1);
  }
  const int x = x0 + tx, y = y0 + ty;
  const bool in = x < nx && y < ny;
  int ks = 0;  // slot of cell plane z
  for (int z = z0; z < z1; ++z) {
    const int iu = z - z0;
    const int ks1 = ks == 2 ? 0 : ks + 1;
#pragma unroll
    for (int p = 0; p < kUPer; ++p) put_u((iu + 2) & 3, p, nu[p]);
#pragma unroll
    for (int p = 0; p < kKPer; ++p) put_k(ks1, p, nk[p]);
    __syncthreads();
    if (z + 1 < z1) {
#pragma unroll
      for (int p = 0; p < kUPer; ++p) nu[p] = ldu(p, z + 2);
#pragma unroll
      for (int p = 0; p < kKPer; ++p) nk[p] = ldk(p, z + 2);
    }
    T uc = T(0), yv = T(0);
    const int64_t i = (int64_t)z * pxy + (int64_t)y * nx + x;
    if (in)
      yv = vertex(sh.u[iu & 3], sh.u[(iu + 1) & 3], sh.u[(iu + 2) & 3], sh.k[ks], sh.k[ks1], tx,
                  ty, i, uc);
    at(i, yv, uc, in);
    ks = ks1;
  }
}

// (A u)_v in FP64 from the vertex's precomputed coefficients (a_vv and the twelve face-diagonal
// entries, -1/12 of a pair sum each, written by k_q1_setup) and the staged planes; the body diagonals
// take the conductivities of the staged cell planes.  22 FP64 operations per vertex instead of
// the 38 of q1_vertex: the FP64 kernels are bound by the FP64 pipe, HBM has room for the
// 104 bytes of coefficients.
__device__ __forceinline__ double q1_vertex_coef(const double* __restrict__ c, int64_t n,
                                                 const double* Um, const double* Uc,
                                                 const double* Up, const double* K0,
                                                 const double* K1, int tx, int ty, int64_t i,
                                                 double& uc) {
  auto U = [&](const double* P, int dx, int dy) -> double {
    return P[(ty + 1 + dy) * UW + tx + 1 + dx];
  };
  auto C = [&](const double* P, int a, int b) -> double { return P[(ty + b) * KW + tx + a]; };
  double cf[13];
#pragma unroll
  for (int k = 0; k < 13; ++k) cf[k] = __ldg(c + k * n + i);
  uc = U(Uc, 0, 0);
  double y = cf[12] * uc;
  y = fma(cf[0], U(Uc, -1, -1), y);  // face diagonals in the plane (dz = 0)
  y = fma(cf[1], U(Uc, 1, -1), y);
  y = fma(cf[2], U(Uc, -1, 1), y);
  y = fma(cf[3], U(Uc, 1, 1), y);
  y = fma(cf[4], U(Um, -1, 0), y);   // dy = 0
  y = fma(cf[5], U(Um, 1, 0), y);
  y = fma(cf[6], U(Up, -1, 0), y);
  y = fma(cf[7], U(Up, 1, 0), y);
  y = fma(cf[8], U(Um, 0, -1), y);   // dx = 0
  y = fma(cf[9], U(Um, 0, 1), y);
  y = fma(cf[10], U(Up, 0, -1), y);
  y = fma(cf[11], U(Up, 0, 1), y);
  double b = C(K0, 0, 0) * U(Um, -1, -1);  // body diagonals: one cell each
  b = fma(C(K0, 1, 0), U(Um, 1, -1), b);
  b = fma(C(K0, 0, 1), U(Um, -1, 1), b);
  b = fma(C(K0, 1, 1), U(Um, 1, 1), b);
  b = fma(C(K1, 0, 0), U(Up, -1, -1), b);
  b = fma(C(K1, 1, 0), U(Up, 1, -1), b);
  b = fma(C(K1, 0, 1), U(Up, -1, 1), b);
  b = fma(C(K1, 1, 1), U(Up, 1, 1), b);
  return fma(-1.0 / 12.0, b, y);
}

template <int EPI, bool SCALE>
__global__ void __launch_bounds__(QT) k_q1(Q1Op A, EpiArgs e, int zc) {
  if (skip<EPI>(e)) return;
  __shared__ Q1Smem<double> sh;
  double red[2] = {0.0, 0.0};
  const double* __restrict__ u = e.u;
  const int64_t n = (int64_t)A.nx * A.ny * A.nz;
  auto load_u = [&](int64_t idx) -> double {
    double v = __ldg(u + idx);
    if constexpr (SCALE) v *= __ldg(e.M.dinv + idx);
    return v;
  };
  auto vertex = [&](const double* Um, const double* Uc, const double* Up, const double* K0,
                    const double* K1, int tx, int ty, int64_t i, double& uc) -> double {
    return q1_vertex_coef(A.kappa + q1_coef_offset(A), n, Um, Uc, Up, K0, K1, tx, ty, i, uc);
  };
  q1_march<double>(A, A.kappa, A.nx + 1, zc, sh, load_u, vertex, [&](int64_t i, double yv, double uc, bool in) {
    if (!in) return;
    if constexpr (EPI == EP_MPK_FIRST && !SCALE) {
      yv *= e.M.dinv_u;
      uc *= e.M.dinv_u;
    }
    epilogue<EPI>(e, i, yv, uc, red);
  });
  reduce_and_finish<EPI>(e, red);
}

// PAP: the FP32 PCG product step (u = p, y = A p, no recurrence): p^T (A p) is accumulated in
// double-float and the last CTA forms alpha (pap_finish).
template <bool FIRST, bool SCALE, bool PAP = false>
__global__ void __launch_bounds__(QT) k_q1f(Q1Op A, MpkF32Args e, int zc) {
  if (e.ctrl && e.ctrl->done) return;
  __shared__ Q1Smem<float> sh;
  float ph[1] = {0.0f}, pl[1] = {0.0f};
  const float* __restrict__ u = e.u;
  auto load_u = [&](int64_t idx) -> float {
    float v = __ldg(u + idx);
    if constexpr (SCALE) v *= __ldg(e.dinv + idx);
    return v;
  };
  auto vertex = [&](const float* Um, const float* Uc, const float* Up, const float* K0,
                    const float* K1, int tx, int ty, int64_t, float& uc) -> float {
    return q1_vertex<float>(Um, Uc, Up, K0, K1, tx, ty, uc);
  };
  q1_march<float>(A, A.kappaf, A.kpitch, zc, sh, load_u, vertex, [&](int64_t i, float yv, float uc, bool in) {
    if (!in) return;
    if constexpr (FIRST && !SCALE) {
      yv *= e.dinv_u;
      uc *= e.dinv_u;
    }
    mpk_f32_epilogue(e, i, yv, uc, FIRST);
    if constexpr (PAP) df_acc_prod(ph[0], pl[0], uc, yv);
  });
  if constexpr (PAP) pap_finish(e, ph, pl);
}

// ---------------------------------------------------------------- TMA-fed FP32 MPK step

// Middle MPK steps of the FP32 path (input not scaled by M^{-1}).  A CTA owns 64 x 8 vertices
// (two x-adjacent vertices per thread) and marches a z chunk.  One thread issues, per z plane,
// a 3D tiled copy of the u plane with its halo (a 72 x 10 box that starts 4 vertices left of
// the tile, so that the x coordinate stays a multiple of 16 bytes) and one of the conductivity
// plane (68 x 9 cells); both complete on the stage's mbarrier.  The copy zero-fills whatever
// lies outside the grid, which is exactly the eliminated Dirichlet boundary.  Each thread reads
// a landed plane from shared memory once into a register window that serves three vertex
// planes (u) or two (cells), after which the slot is refilled kNS planes ahead.  Every wait is
// bounded: a copy that never lands stops the solve with SSTEP_ERR_TIMEOUT instead of hanging.
constexpr int TBX = 64;            // vertices per CTA along x (two per thread)
constexpr int TUW = 72, TUH = 10;  // u box (vertices)
constexpr int TKW = 68, TKH = 9;   // conductivity box (cells)
constexpr int kNS = 6;             // pipeline stages (z planes)
constexpr int kUStage = 736;       // floats per u stage: 720 used, 2944 bytes (23 x 128)
constexpr int kKStage = 640;       // floats per cell stage: 612 used, 2560 bytes (20 x 128)
constexpr uint32_t kStageBytes = (TUW * TUH + TKW * TKH) * 4;

struct __align__(128) TmaSmem {
  float u[kNS][kUStage];
  float k[kNS][kKStage];
  unsigned long long full[kNS];
};

// Register window of one staged plane for a thread's two vertices (x and x + 1): u at rows
// y-1..y+1 and columns x-1..x+2 (v[dy + 1][c]); the conductivities of cells x..x+2 at rows
// y, y+1 (k[b][a]) with their in-plane pair sums.
struct UWin2 {
  float v[3][4];
};
struct KWin2 {
  float k[2][3];
  float ya[3];     // ya[a] = k[0][a] + k[1][a]: the pair along y of cell column a
  float xb[2][2];  // xb[d][b] = k[b][d] + k[b][d + 1]: the pair along x of vertex d, row b
};

__device__ __forceinline__ void read_plane2(const float* P, const float* K, int tx, int ty,
                                            UWin2& w, KWin2& c) {
  // vertex x0 + 2 tx is column 2 tx + 4 of the u box and column 2 tx of the cell box
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float* row = P + (ty + r) * TUW + 2 * tx + 3;
    w.v[r][0] = row[0];
    const float2 mid = *reinterpret_cast<const float2*>(row + 1);
    w.v[r][1] = mid.x;
    w.v[r][2] = mid.y;
    w.v[r][3] = row[3];
  }
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const float* row = K + (ty + b) * TKW + 2 * tx;
    const float2 lo = *reinterpret_cast<const float2*>(row);
    c.k[b][0] = lo.x;
    c.k[b][1] = lo.y;
    c.k[b][2] = row[2];
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) c.ya[a] = c.k[0][a] + c.k[1][a];
#pragma unroll
  for (int d = 0; d < 2; ++d)
#pragma unroll
    for (int b = 0; b < 2; ++b) c.xb[d][b] = c.k[b][d] + c.k[b][d + 1];
}

// q1_vertex's arithmetic, term for term, for vertex D of the pair: m, c, p = u planes z-1, z,
// z+1; k0, k1 = cell planes z, z+1.
template <int D>
__device__ __forceinline__ float q1_vertex_win(const UWin2& m, const UWin2& c, const UWin2& p,
                                               const KWin2& k0, const KWin2& k1, float& uc) {
  auto U = [](const UWin2& w, int dx, int dy) -> float { return w.v[dy + 1][D + 1 + dx]; };
  const float k000 = k0.k[0][D], k100 = k0.k[0][D + 1], k010 = k0.k[1][D], k110 = k0.k[1][D + 1];
  const float k001 = k1.k[0][D], k101 = k1.k[0][D + 1], k011 = k1.k[1][D], k111 = k1.k[1][D + 1];
  const float z00 = k000 + k001, z10 = k100 + k101, z01 = k010 + k011, z11 = k110 + k111;
  const float k8 = (z00 + z10) + (z01 + z11);
  float s = z00 * U(c, -1, -1);
  s = fmaf(z10, U(c, 1, -1), s);
  s = fmaf(z01, U(c, -1, 1), s);
  s = fmaf(z11, U(c, 1, 1), s);
  s = fmaf(k0.ya[D], U(m, -1, 0), s);      // y00
  s = fmaf(k0.ya[D + 1], U(m, 1, 0), s);   // y10
  s = fmaf(k1.ya[D], U(p, -1, 0), s);      // y01
  s = fmaf(k1.ya[D + 1], U(p, 1, 0), s);   // y11
  s = fmaf(k0.xb[D][0], U(m, 0, -1), s);   // x00
  s = fmaf(k0.xb[D][1], U(m, 0, 1), s);    // x10
  s = fmaf(k1.xb[D][0], U(p, 0, -1), s);   // x01
  s = fmaf(k1.xb[D][1], U(p, 0, 1), s);    // x11
  s = fmaf(k000, U(m, -1, -1), s);
  s = fmaf(k100, U(m, 1, -1), s);
  s = fmaf(k010, U(m, -1, 1), s);
  s = fmaf(k110, U(m, 1, 1), s);
  s = fmaf(k001, U(p, -1, -1), s);
  s = fmaf(k101, U(p, 1, -1), s);
  s = fmaf(k011, U(p, -1, 1), s);
  s = fmaf(k111, U(p, 1, 1), s);
  uc = U(c, 0, 0);
  return fmaf(k8 * (1.0f / 3.0f), uc, -(s * (1.0f / 12.0f)));
}

// PAP: the FP32 PCG product step, as in k_q1f.
template <bool PAP = false>
__global__ void __launch_bounds__(QT, 3) k_q1f_tma(const __grid_constant__ CUtensorMap mu,
                                                 const __grid_constant__ CUtensorMap mk, Q1Op A,
                                                 MpkF32Args e, int zc) {
  if (e.ctrl && e.ctrl->done) return;
  __shared__ TmaSmem sh;
  float pah[1] = {0.0f}, pal[1] = {0.0f};  // PAP: p^T (A p)
  const int tid = threadIdx.x, tx = tid % QX, ty = tid / QX;
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const int x0 = blockIdx.x * TBX, y0 = blockIdx.y * QY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, nz);
  const int nzc = z1 - z0;
  const int np = nzc + 2;  // stage p holds u plane and cell plane z0 - 1 + p
  const int64_t pxy = (int64_t)nx * ny;
  int issued = 0;          // stages issued (thread 0's count)
  auto issue = [&](int p) {
    const int slot = p % kNS;
    const uint32_t bar = tma::smem_addr(&sh.full[slot]);
    tma::mbar_expect_tx(bar, kStageBytes);
    tma::load_3d(tma::smem_addr(sh.u[slot]), &mu, x0 - 4, y0 - 1, z0 - 1 + p, bar);
    tma::load_3d(tma::smem_addr(sh.k[slot]), &mk, x0, y0, z0 - 1 + p, bar);
    issued = p + 1;
  };
  if (tid == 0) {
    for (int i = 0; i < kNS; ++i) tma::mbar_init(tma::smem_addr(&sh.full[i]), 1);
    tma::mbar_init_fence();
  }
  __syncthreads();
  if (tid == 0)
    for (int p = 0; p < min(kNS, np); ++p) issue(p);
  const int x = x0 + 2 * tx, y = y0 + ty;
  const bool in = x < nx && y < ny;  // nx is even: x + 1 < nx too
  int waited = 0;                    // stages 0 .. waited-1 have landed
  bool lost = false;
  auto wait_stage = [&](int slot, uint32_t parity) {
    if (!lost && !tma::mbar_wait(tma::smem_addr(&sh.full[slot]), parity)) lost = true;
    if (!lost) ++waited;
  };
  UWin2 uw[3];  // stage p in uw[p % 3]
  KWin2 kw[2];  // stage p in kw[p % 2]
  int64_t idx = (int64_t)z0 * pxy + (int64_t)y * nx + x;  // even: 8-byte aligned pairs
  float2 dv = make_float2(e.dinv_u, e.dinv_u), zp = make_float2(0.0f, 0.0f);
  if (in) {
    if (e.dinv) dv = __ldg(reinterpret_cast<const float2*>(e.dinv + idx));
    if (e.zprev) zp = __ldg(reinterpret_cast<const float2*>(e.zprev + idx));
  }
  wait_stage(0, 0);
  wait_stage(1, 0);
  if (!lost) {
    read_plane2(sh.u[0], sh.k[0], tx, ty, uw[0], kw[0]);
    read_plane2(sh.u[1], sh.k[1], tx, ty, uw[1], kw[1]);
  }
  bool stop = __syncthreads_or(lost);
  if (!stop && tid == 0)
    for (int p = kNS; p < min(kNS + 2, np); ++p) issue(p);
  uint32_t ph = 0;  // phase parity of the stages in the current round of kNS
  // unrolled by kNS (a multiple of both window periods): slots and windows are constants
  for (int i0 = 0; i0 < nzc && !stop; i0 += kNS, ph ^= 1u) {
#pragma unroll
    for (int j = 0; j < kNS; ++j) {
      const int i = i0 + j;
      if (i >= nzc || stop) break;
      float2 dvn = make_float2(e.dinv_u, e.dinv_u), zpn = make_float2(0.0f, 0.0f);
      if (in && i + 1 < nzc) {  // next plane's epilogue inputs, requested early
        if (e.dinv) dvn = __ldg(reinterpret_cast<const float2*>(e.dinv + idx + pxy));
        if (e.zprev) zpn = __ldg(reinterpret_cast<const float2*>(e.zprev + idx + pxy));
      }
      constexpr int kFill = 2;  // stage i + 2 enters the windows in iteration i
      wait_stage((j + kFill) % kNS, ph ^ (uint32_t)((j + kFill) / kNS));
      if (!lost)
        read_plane2(sh.u[(j + kFill) % kNS], sh.k[(j + kFill) % kNS], tx, ty, uw[(j + 2) % 3],
                    kw[j % 2]);
      // every thread has its copy of stage i + 2: refill that slot kNS stages ahead
      stop = __syncthreads_or(lost);
      if (stop) break;
      if (tid == 0 && i + kFill + kNS < np) issue(i + kFill + kNS);
      if (in) {
        float2 yv, uc;
        yv.x = q1_vertex_win<0>(uw[j % 3], uw[(j + 1) % 3], uw[(j + 2) % 3], kw[(j + 1) % 2],
                                kw[j % 2], uc.x);
        yv.y = q1_vertex_win<1>(uw[j % 3], uw[(j + 1) % 3], uw[(j + 2) % 3], kw[(j + 1) % 2],
                                kw[j % 2], uc.y);
        *reinterpret_cast<float2*>(e.y + idx) = yv;  // A z_q
        if constexpr (PAP) {
          df_acc_prod(pah[0], pal[0], uc.x, yv.x);
          df_acc_prod(pah[0], pal[0], uc.y, yv.y);
        }
        if (e.znext) {
          const float2 t = e.zprev ? make_float2(-zp.x, -zp.y) : make_float2(0.0f, 0.0f);
          float2 zn;
          zn.x = fmaf(e.c1 * dv.x, yv.x, fmaf(-e.c2, uc.x, t.x));
          zn.y = fmaf(e.c1 * dv.y, yv.y, fmaf(-e.c2, uc.y, t.y));
          *reinterpret_cast<float2*>(e.znext + idx) = zn;
        }
      }
      dv = dvn;
      zp = zpn;
      idx += pxy;
    }
  }
  if (stop && tid == 0) {
    // let the copies still in flight land before the CTA's shared memory is released
    for (int p = waited; p < issued; ++p)
      tma::mbar_wait(tma::smem_addr(&sh.full[p % kNS]), (uint32_t)(p / kNS) & 1u);
    if (e.ctrl) {
      e.ctrl->status = SSTEP_ERR_TIMEOUT;
      e.ctrl->done = 1;
    }
  }
  if constexpr (PAP) pap_finish(e, pah, pal);  // every thread: stop is uniform over the CTA
}

// FP32 conductivities with rows padded to kpitch (padding zero).
__global__ void k_q1_kappaf(Q1Op A, float* out) {
  const int64_t rows = (int64_t)(A.ny + 1) * (A.nz + 1);
  const int64_t total = rows * A.kpitch;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = c / A.kpitch;
    const int cx = (int)(c % A.kpitch);
    out[c] = cx <= A.nx ? (float)A.kappa[row * (A.nx + 1) + cx] : 0.0f;
  }
}

int sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

struct Q1Grid {
  dim3 grid;
  int zc;
};

// xy tiles x z chunks: about eight CTAs per SM, z chunks of at least 8 planes.
Q1Grid q1_grid(const Q1Op& A) {
  const int gx = (A.nx + QX - 1) / QX, gy = (A.ny + QY - 1) / QY;
  int64_t gz = std::max<int64_t>(1, (int64_t)sms() * 8 / std::max(1, gx * gy));
  gz = std::min<int64_t>(gz, std::max(1, A.nz / 8));
  const int zc = (int)((A.nz + gz - 1) / gz);
  return {dim3(gx, gy, (A.nz + zc - 1) / zc), zc};
}

template <int EPI>
cudaError_t launch_epi(const Q1Op& A, const EpiArgs& e, cudaStream_t st) {
  const Q1Grid g = q1_grid(A);
  if (EPI == EP_MPK_FIRST && e.M.dinv != nullptr)
    k_q1<EPI, true><<<g.grid, QT, 0, st>>>(A, e, g.zc);
  else
    k_q1<EPI, false><<<g.grid, QT, 0, st>>>(A, e, g.zc);
  return cudaGetLastError();
}

// Set-up pass: one vertex per thread, conductivities read from global memory.
__global__ void __launch_bounds__(kThreads) k_q1_setup(Q1Op A, int jacobi, double* dinv,
                                                       double* out_min, int* bad) {
  __shared__ double sh[kThreads];
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t ncell = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t c = t0; c < ncell; c += stride) {
    const double k = A.kappa[c];
    if (!(k > 0.0) || !(k < 1.79e308)) *bad = 1;
  }
  double lo = 1.0e308;
  for (int64_t i = t0; i < n; i += stride) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
    auto kap = [&](int a, int b, int c) -> double {
      return A.kappa[((int64_t)(z + c) * (ny + 1) + (y + b)) * (nx + 1) + (x + a)];
    };
    double k8 = 0.0, off = 0.0;
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) k8 += kap(a, b, c);
    {  // the FP64 kernels' vertex coefficients (layout at q1_coef_offset)
      double* o = const_cast<double*>(A.kappa) + q1_coef_offset(A) + i;
      const double w = -1.0 / 12.0;
      o[0 * n] = w * (kap(0, 0, 0) + kap(0, 0, 1));
      o[1 * n] = w * (kap(1, 0, 0) + kap(1, 0, 1));
      o[2 * n] = w * (kap(0, 1, 0) + kap(0, 1, 1));
      o[3 * n] = w * (kap(1, 1, 0) + kap(1, 1, 1));
      o[4 * n] = w * (kap(0, 0, 0) + kap(0, 1, 0));
      o[5 * n] = w * (kap(1, 0, 0) + kap(1, 1, 0));
      o[6 * n] = w * (kap(0, 0, 1) + kap(0, 1, 1));
      o[7 * n] = w * (kap(1, 0, 1) + kap(1, 1, 1));
      o[8 * n] = w * (kap(0, 0, 0) + kap(1, 0, 0));
      o[9 * n] = w * (kap(0, 1, 0) + kap(1, 1, 0));
      o[10 * n] = w * (kap(0, 0, 1) + kap(1, 0, 1));
      o[11 * n] = w * (kap(0, 1, 1) + kap(1, 1, 1));
      o[12 * n] = k8 / 3.0;
    }
    // interior neighbours at offsets with two or three non-zero components
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int nnzc = (dx != 0) + (dy != 0) + (dz != 0);
          if (nnzc < 2) continue;
          if (x + dx < 0 || x + dx >= nx || y + dy < 0 || y + dy >= ny || z + dz < 0 ||
              z + dz >= nz)
            continue;
          double w = 0.0;  // sum of the conductivities of the cells holding both vertices
          for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
              for (int a = 0; a < 2; ++a) {
                if (dx != 0 && a != (dx + 1) / 2) continue;
                if (dy != 0 && b != (dy + 1) / 2) continue;
                if (dz != 0 && c != (dz + 1) / 2) continue;
                w += kap(a, b, c);
              }
          off += w / 12.0;
        }
    const double d = k8 / 3.0;
    if (dinv) dinv[i] = 1.0 / d;
    lo = fmin(lo, jacobi ? 1.0 - off / d : d - off);
  }
  sh[threadIdx.x] = lo;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out_min[blockIdx.x] = sh[0];
}

}  // namespace

constexpr int kMaxCols = 16;

struct Q1TmaMaps {
  int ncols;
  const float* col[kMaxCols];
  CUtensorMap mu[kMaxCols];
  CUtensorMap mk;
};

int q1_grid_ctas(const Q1Op& A) {
  const Q1Grid g = q1_grid(A);
  return (int)(g.grid.x * g.grid.y * g.grid.z);
}

cudaError_t launch_q1_operator(const Q1Op& A, const EpiArgs& e, cudaStream_t st) {
  switch (e.epi) {
    case EP_SPMV: return launch_epi<EP_SPMV>(A, e, st);
    case EP_MPK: return launch_epi<EP_MPK>(A, e, st);
    case EP_MPK_FIRST: return launch_epi<EP_MPK_FIRST>(A, e, st);
    case EP_RESID: return launch_epi<EP_RESID>(A, e, st);
    case EP_POWER: return launch_epi<EP_POWER>(A, e, st);
    case EP_PCG_AP: return launch_epi<EP_PCG_AP>(A, e, st);
    case EP_TRUERES: return launch_epi<EP_TRUERES>(A, e, st);
    case EP_RR: return launch_epi<EP_RR>(A, e, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_q1_mpk_f32(const Q1Op& A, const MpkF32Args& e, cudaStream_t st) {
  if (!A.kappaf) return cudaErrorInvalidValue;
  const Q1Grid g = q1_grid(A);
  if (!e.first && A.tma) {
    for (int c = 0; c < A.tma->ncols; ++c)
      if (A.tma->col[c] == e.u) {
        // one wave of resident CTAs, each marching a long z chunk: the pipeline fill (the
        // first two planes' latency) is paid once per CTA
        static int per_sm = 0;
        if (!per_sm) {
          if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_q1f_tma<false>, QT, 0) !=
                  cudaSuccess ||
              per_sm < 1)
            per_sm = 1;
        }
        const int gx = (A.nx + TBX - 1) / TBX, gy = (A.ny + QY - 1) / QY;
        int64_t gz = std::max<int64_t>(1, (int64_t)sms() * per_sm / std::max(1, gx * gy));
        gz = std::min<int64_t>(gz, std::max(1, A.nz / 8));
        const int zc = (int)((A.nz + gz - 1) / gz);
        const dim3 grid(gx, gy, (A.nz + zc - 1) / zc);
        if (e.pap) k_q1f_tma<true><<<grid, QT, 0, st>>>(A.tma->mu[c], A.tma->mk, A, e, zc);
        else k_q1f_tma<false><<<grid, QT, 0, st>>>(A.tma->mu[c], A.tma->mk, A, e, zc);
        return cudaGetLastError();
      }
  }
  if (e.pap) {
    if (e.first) return cudaErrorInvalidValue;
    k_q1f<false, false, true><<<g.grid, QT, 0, st>>>(A, e, g.zc);
    return cudaGetLastError();
  }
  if (e.first) {
    if (e.dinv) k_q1f<true, true><<<g.grid, QT, 0, st>>>(A, e, g.zc);
    else k_q1f<true, false><<<g.grid, QT, 0, st>>>(A, e, g.zc);
  } else {
    k_q1f<false, false><<<g.grid, QT, 0, st>>>(A, e, g.zc);
  }
  return cudaGetLastError();
}


Q1TmaMaps* q1_tma_build(const Q1Op& A, const float* const* cols, int ncols) {
  // rows of u must be 16-byte multiples (nx % 4 == 0); boxes no larger than the grid
  if (A.nx % 4 != 0 || A.nx < TUW || A.ny < TUH || A.nx + 1 < TKW || !A.kappaf ||
      A.kpitch % 4 != 0 || ncols < 1 || ncols > kMaxCols)
    return nullptr;
  auto* m = new Q1TmaMaps{};
  m->ncols = ncols;
  bool ok = tma::encode_3d(&m->mk, A.kappaf, (uint64_t)A.nx + 1, (uint64_t)A.ny + 1,
                      (uint64_t)A.nz + 1, (uint64_t)A.kpitch, TKW, TKH);
  for (int c = 0; ok && c < ncols; ++c) {
    m->col[c] = cols[c];
    ok = tma::encode_3d(&m->mu[c], cols[c], (uint64_t)A.nx, (uint64_t)A.ny, (uint64_t)A.nz,
                   (uint64_t)A.nx, TUW, TUH);
  }
  if (!ok) {
    delete m;
    return nullptr;
  }
  return m;
}

void q1_tma_free(Q1TmaMaps* m) { delete m; }

cudaError_t launch_q1_kappaf(const Q1Op& A, float* kappaf, cudaStream_t st) {
  const int64_t total = (int64_t)(A.ny + 1) * (A.nz + 1) * A.kpitch;
  const int64_t want = (total + kThreads - 1) / kThreads;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms() * 8));
  k_q1_kappaf<<<grid, kThreads, 0, st>>>(A, kappaf);
  return cudaGetLastError();
}

int q1_setup_ctas(int64_t n) {
  const int64_t want = (n + kThreads - 1) / kThreads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms() * 4));
}

cudaError_t launch_q1_setup(const Q1Op& A, int jacobi, double* dinv, double* out_min, int* bad,
                            cudaStream_t st) {
  const int64_t n = (int64_t)A.nx * A.ny * A.nz;
  k_q1_setup<<<q1_setup_ctas(n), kThreads, 0, st>>>(A, jacobi, dinv, out_min, bad);
  return cudaGetLastError();
}

}  // namespace sstep
