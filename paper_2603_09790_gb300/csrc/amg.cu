// amg.cu -- aggregation AMG preconditioner (M^{-1} = one V-cycle) for CSR operators.
//
// The paper treats M^{-1} as a black box and uses an external AMG (Section 5); this library's
// AMG is defined as follows (set-up on the host, application on the device):
//  * coupling strength w_ij = -a_ij / sqrt(a_ii a_jj); greedy pairwise matching over rows in
//    increasing order, each unmatched row taking its unmatched neighbour of largest w_ij > 0
//    (ties: lower index), singletons otherwise; aggregates numbered by their lowest row;
//  * two matchings per level (pairs of pairs), unsmoothed piecewise-constant prolongation P;
//  * Galerkin A_c = P^T A P summed in a fixed order (coarse row J visits the rows of aggregate
//    J in increasing order, each row's entries in stored order; the first contribution
//    initialises an entry), coarse rows stored with increasing columns, so the hierarchy is
//    reproducible bit for bit;
//  * l1-Jacobi smoothing D = diag(sum_j |a_ij|), one sweep before and after the coarse
//    correction; coarsening stops at n <= coarse_max, where A^{-1} is applied as a dense
//    matrix (formed from its Cholesky factor at set-up).
// V-cycle on level l for b: x = D^{-1} b; r = b - A x; x_c = V_{l+1}(P^T r); t = x + P x_c;
// x = t + D^{-1}(b - A t).  Every reduction is a fixed-order loop: results are deterministic.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace sstep {

struct AmgLevel {
  int64_t n = 0, nnz = 0, nc = 0;
  // host copies (kept for inspection)
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> v;
  std::vector<int32_t> agg;
  // device
  int64_t* rowptr = nullptr;
  int32_t* colind = nullptr;
  double* vals = nullptr;
  double* dinv = nullptr;     // 1 / (l1 row sum)
  int32_t* dagg = nullptr;    // fine row -> aggregate
  int64_t* mptr = nullptr;    // aggregate members (increasing rows), CSR-like
  int32_t* mem = nullptr;
  double *x = nullptr, *b = nullptr, *r = nullptr;  // work vectors (x, b unused on level 0)
};

struct AmgHier {
  std::vector<AmgLevel> lev;
  double* cinv = nullptr;  // dense A_coarsest^{-1}, n_c x n_c row-major
  int64_t ncoarse = 0;
};

namespace {

struct HostCsr {
  int64_t n = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> v;
};

// Greedy pairwise matching; returns the number of aggregates, or -1 for a non-positive diagonal.
int64_t pair_match(const HostCsr& A, std::vector<int32_t>& agg) {
  const int64_t n = A.n;
  std::vector<double> d(n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k)
      if (A.ci[k] == i) d[i] = A.v[k];
    if (!(d[i] > 0.0)) return -1;
  }
  std::vector<int64_t> mate(n, -1);
  for (int64_t i = 0; i < n; ++i) {
    if (mate[i] >= 0) continue;
    int64_t best = -1;
    double wb = 0.0;
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
      const int64_t j = A.ci[k];
      if (j == i || mate[j] >= 0) continue;
      const double w = -A.v[k] / std::sqrt(d[i] * d[j]);
      if (w > wb || (w == wb && best >= 0 && j < best)) {
        best = j;
        wb = w;
      }
    }
    if (best >= 0) {
      mate[i] = best;
      mate[best] = i;
    } else {
      mate[i] = i;
    }
  }
  agg.assign(n, -1);
  int64_t nc = 0;
  for (int64_t i = 0; i < n; ++i)
    if (i <= mate[i]) {
      agg[i] = (int32_t)nc;
      agg[mate[i]] = (int32_t)nc;
      ++nc;
    }
  return nc;
}

// Members of every aggregate in increasing row order.
void members(const std::vector<int32_t>& agg, int64_t nc, std::vector<int64_t>& mptr,
             std::vector<int32_t>& mem) {
  mptr.assign(nc + 1, 0);
  for (int32_t a : agg) mptr[a + 1] += 1;
  for (int64_t J = 0; J < nc; ++J) mptr[J + 1] += mptr[J];
  std::vector<int64_t> fill(mptr.begin(), mptr.end() - 1);
  mem.assign(agg.size(), 0);
  for (size_t i = 0; i < agg.size(); ++i) mem[fill[agg[i]]++] = (int32_t)i;
}

// P^T A P in the fixed order described at the top of the file.  Coarse rows are independent,
// so contiguous blocks of them are formed by host threads and concatenated in row order: the
// result does not depend on the number of threads.
void galerkin(const HostCsr& A, const std::vector<int32_t>& agg, int64_t nc, HostCsr& C) {
  std::vector<int64_t> mptr;
  std::vector<int32_t> mem;
  members(agg, nc, mptr, mem);
  C.n = nc;
  C.rp.assign(nc + 1, 0);
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int T = nc < 8192 ? 1 : std::min(16, hw);
  std::vector<std::vector<int32_t>> tci(T);
  std::vector<std::vector<double>> tv(T);
  std::vector<int64_t> cnt(nc, 0);
  auto work = [&](int t) {
    const int64_t J0 = nc * t / T, J1 = nc * (t + 1) / T;
    std::vector<int64_t> pos(nc, -1);
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t J = J0; J < J1; ++J) {
      row.clear();
      for (int64_t m = mptr[J]; m < mptr[J + 1]; ++m) {
        const int64_t i = mem[m];
        for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) {
          const int32_t Jc = agg[A.ci[k]];
          if (pos[Jc] < 0) {
            pos[Jc] = (int64_t)row.size();
            row.emplace_back(Jc, A.v[k]);
          } else {
            row[pos[Jc]].second += A.v[k];
          }
        }
      }
      for (auto& e : row) pos[e.first] = -1;
      std::sort(row.begin(), row.end(),
                [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                  return a.first < b.first;
                });
      for (auto& e : row) {
        tci[t].push_back(e.first);
        tv[t].push_back(e.second);
      }
      cnt[J] = (int64_t)row.size();
    }
  };
  if (T == 1) {
    work(0);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t) th.emplace_back(work, t);
    for (auto& x : th) x.join();
  }
  for (int64_t J = 0; J < nc; ++J) C.rp[J + 1] = C.rp[J] + cnt[J];
  C.ci.clear();
  C.v.clear();
  C.ci.reserve(C.rp[nc]);
  C.v.reserve(C.rp[nc]);
  for (int t = 0; t < T; ++t) {
    C.ci.insert(C.ci.end(), tci[t].begin(), tci[t].end());
    C.v.insert(C.v.end(), tv[t].begin(), tv[t].end());
  }
}

// Dense inverse of the SPD matrix A (n x n, row-major out) through its Cholesky factor.
bool dense_inverse(const HostCsr& A, std::vector<double>& inv) {
  const int64_t n = A.n;
  std::vector<double> L(n * n, 0.0);  // row-major, lower
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = A.rp[i]; k < A.rp[i + 1]; ++k) L[i * n + A.ci[k]] = A.v[k];
  for (int64_t j = 0; j < n; ++j) {
    double d = L[j * n + j];
    for (int64_t k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    L[j * n + j] = ljj;
    for (int64_t i = j + 1; i < n; ++i) {
      double s = L[i * n + j];
      for (int64_t k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = s / ljj;
    }
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) L[i * n + j] = 0.0;
  // Linv (lower) by forward substitution on the unit vectors; A^{-1} = Linv^T Linv
  std::vector<double> Li(n * n, 0.0);
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t i = c; i < n; ++i) {
      double s = i == c ? 1.0 : 0.0;
      for (int64_t k = c; k < i; ++k) s -= L[i * n + k] * Li[k * n + c];
      Li[i * n + c] = s / L[i * n + i];
    }
  }
  inv.assign(n * n, 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j <= i; ++j) {
      double s = 0.0;
      for (int64_t k = i; k < n; ++k) s += Li[k * n + i] * Li[k * n + j];
      inv[i * n + j] = s;
      inv[j * n + i] = s;
    }
  return true;
}

// ---------------------------------------------------------------- kernels

constexpr int kAmgThreads = 256;

int grid_for(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + kAmgThreads - 1) / kAmgThreads, 152 * 8));
}

// x = D^{-1} b; r = b - A x (x's neighbours formed on the fly)
__global__ void k_amg_pre(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const double* __restrict__ v, const double* __restrict__ dinv,
                          const double* __restrict__ b, double* __restrict__ x, double* __restrict__ r) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double ax = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
      const int32_t j = ci[k];
      ax = fma(v[k], b[j] * dinv[j], ax);
    }
    const double bi = b[i];
    x[i] = bi * dinv[i];
    r[i] = bi - ax;
  }
}

// b_c[J] = sum of r over the rows of aggregate J (increasing rows)
__global__ void k_amg_restrict(int64_t nc, const int64_t* __restrict__ mptr,
                               const int32_t* __restrict__ mem, const double* __restrict__ r,
                               double* __restrict__ bc) {
  for (int64_t J = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; J < nc;
       J += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t m = mptr[J]; m < mptr[J + 1]; ++m) s += r[mem[m]];
    bc[J] = s;
  }
}

// t = x + P x_c
__global__ void k_amg_prolong(int64_t n, const int32_t* __restrict__ agg, const double* __restrict__ x,
                              const double* __restrict__ xc, double* __restrict__ t) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    t[i] = x[i] + xc[agg[i]];
}

// x = t + D^{-1} (b - A t)
__global__ void k_amg_post(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ v, const double* __restrict__ dinv,
                           const double* __restrict__ b, const double* __restrict__ t,
                           double* __restrict__ x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double at = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) at = fma(v[k], t[ci[k]], at);
    x[i] = fma(b[i] - at, dinv[i], t[i]);
  }
}

// x = A_c^{-1} b on the coarsest level: one warp per row, fixed-order lane sums.
__global__ void k_amg_coarse(int64_t nc, const double* __restrict__ inv, const double* __restrict__ b,
                             double* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < nc; i += warps) {
    double s = 0.0;
    for (int64_t k = lane; k < nc; k += 32) s = fma(inv[i * nc + k], b[k], s);
    s = warp_sum(s);
    if (lane == 0) x[i] = s;
  }
}

// z_next = c1 t - c2 z_q - c3 z_prev (Chebyshev recurrence with M^{-1} applied to A z_q)
__global__ void k_cheb_combine(int64_t n, const double* __restrict__ t, const double* __restrict__ zq,
                               const double* __restrict__ zprev, double c1, double c2, double c3,
                               double* __restrict__ znext) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double z = fma(c1, t[i], -c2 * zq[i]);
    if (zprev) z = fma(-c3, zprev[i], z);
    znext[i] = z;
  }
}

cudaError_t upload(AmgLevel& L, bool coarsest, cudaStream_t st) {
  cudaError_t e;
  const int64_t n = L.n, nnz = L.nnz;
  if ((e = cudaMalloc(&L.rowptr, sizeof(int64_t) * (n + 1))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&L.colind, sizeof(int32_t) * std::max<int64_t>(nnz, 1))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&L.vals, sizeof(double) * std::max<int64_t>(nnz, 1))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&L.dinv, sizeof(double) * n)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&L.x, sizeof(double) * n)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&L.b, sizeof(double) * n)) != cudaSuccess) return e;
  if ((e = cudaMalloc(&L.r, sizeof(double) * n)) != cudaSuccess) return e;
  std::vector<double> d(n, 0.0);
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = L.rp[i]; k < L.rp[i + 1]; ++k) s += std::fabs(L.v[k]);
    d[i] = 1.0 / s;
  }
  if ((e = cudaMemcpyAsync(L.rowptr, L.rp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(L.colind, L.ci.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(L.vals, L.v.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(L.dinv, d.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if (!coarsest) {
    std::vector<int64_t> mptr;
    std::vector<int32_t> mem;
    members(L.agg, L.nc, mptr, mem);
    if ((e = cudaMalloc(&L.dagg, sizeof(int32_t) * n)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&L.mptr, sizeof(int64_t) * (L.nc + 1))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&L.mem, sizeof(int32_t) * n)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(L.dagg, L.agg.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(L.mptr, mptr.data(), sizeof(int64_t) * (L.nc + 1), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(L.mem, mem.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  }
  return cudaStreamSynchronize(st);  // the host vectors above must outlive the copies
}

cudaError_t vcycle(const AmgHier* H, size_t l, const double* b, double* x, cudaStream_t st) {
  const AmgLevel& L = H->lev[l];
  if (l + 1 == H->lev.size()) {
    k_amg_coarse<<<(int)std::min<int64_t>((L.n + 7) / 8, 1024), 256, 0, st>>>(L.n, H->cinv, b, x);
    return cudaGetLastError();
  }
  const AmgLevel& C = H->lev[l + 1];
  const int g = grid_for(L.n);
  k_amg_pre<<<g, kAmgThreads, 0, st>>>(L.n, L.rowptr, L.colind, L.vals, L.dinv, b, x, L.r);
  k_amg_restrict<<<grid_for(L.nc), kAmgThreads, 0, st>>>(L.nc, L.mptr, L.mem, L.r, C.b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = vcycle(H, l + 1, C.b, C.x, st)) != cudaSuccess) return e;
  k_amg_prolong<<<g, kAmgThreads, 0, st>>>(L.n, L.dagg, x, C.x, L.r);
  k_amg_post<<<g, kAmgThreads, 0, st>>>(L.n, L.rowptr, L.colind, L.vals, L.dinv, b, L.r, x);
  return cudaGetLastError();
}

}  // namespace

sstep_status amg_build(const int64_t* rowptr_dev, const int32_t* colind_dev, const double* vals_dev,
                       int64_t n, int64_t nnz, int64_t coarse_max, int max_levels,
                       cudaStream_t st, AmgHier** out) {
  *out = nullptr;
  if (coarse_max < 1 || coarse_max > 4096 || max_levels < 1 || max_levels > 32) {
    set_last_error("AMG coarse_max must be in 1..4096 and max_levels in 1..32");
    return SSTEP_ERR_INVALID;
  }
  HostCsr A;
  A.n = n;
  A.rp.resize(n + 1);
  A.ci.resize(nnz);
  A.v.resize(nnz);
  if (cudaMemcpyAsync(A.rp.data(), rowptr_dev, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(A.ci.data(), colind_dev, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(A.v.data(), vals_dev, sizeof(double) * nnz, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_last_error("AMG set-up: copying the operator to the host failed");
    return SSTEP_ERR_CUDA;
  }
  AmgHier* H = new AmgHier();
  auto bail = [&](sstep_status s, const char* msg) {
    set_last_error(msg);
    amg_free(H);
    return s;
  };
  HostCsr cur = std::move(A);
  for (int l = 0;; ++l) {
    H->lev.emplace_back();
    AmgLevel& L = H->lev.back();
    L.n = cur.n;
    L.nnz = cur.rp[cur.n];
    const bool last = cur.n <= coarse_max || l + 1 >= max_levels;
    if (!last) {
      std::vector<int32_t> a1, a2;
      const int64_t nc1 = pair_match(cur, a1);
      if (nc1 < 0) return bail(SSTEP_ERR_INVALID, "AMG needs a positive diagonal on every level");
      HostCsr B;
      galerkin(cur, a1, nc1, B);
      const int64_t nc = pair_match(B, a2);
      if (nc < 0) return bail(SSTEP_ERR_INVALID, "AMG needs a positive diagonal on every level");
      if (nc < cur.n) {
        L.agg.resize(cur.n);
        for (int64_t i = 0; i < cur.n; ++i) L.agg[i] = a2[a1[i]];
        L.nc = nc;
        HostCsr C;
        galerkin(cur, L.agg, nc, C);
        L.rp = std::move(cur.rp);
        L.ci = std::move(cur.ci);
        L.v = std::move(cur.v);
        if (upload(L, false, st) != cudaSuccess) return bail(SSTEP_ERR_OOM, "AMG: device allocation failed");
        cur = std::move(C);
        continue;
      }
      if (cur.n > 8 * coarse_max)
        return bail(SSTEP_ERR_UNSUPPORTED, "AMG coarsening stalled above the dense-solve size");
    }
    // coarsest level: dense inverse
    L.rp = std::move(cur.rp);
    L.ci = std::move(cur.ci);
    L.v = std::move(cur.v);
    HostCsr tmp;
    tmp.n = L.n;
    tmp.rp = L.rp;
    tmp.ci = L.ci;
    tmp.v = L.v;
    std::vector<double> inv;
    if (!dense_inverse(tmp, inv)) return bail(SSTEP_ERR_BREAKDOWN, "AMG coarsest matrix is not positive definite");
    if (upload(L, true, st) != cudaSuccess) return bail(SSTEP_ERR_OOM, "AMG: device allocation failed");
    H->ncoarse = L.n;
    if (cudaMalloc(&H->cinv, sizeof(double) * L.n * L.n) != cudaSuccess)
      return bail(SSTEP_ERR_OOM, "AMG: device allocation failed");
    if (cudaMemcpyAsync(H->cinv, inv.data(), sizeof(double) * L.n * L.n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return bail(SSTEP_ERR_CUDA, "AMG: upload failed");
    break;
  }
  *out = H;
  return SSTEP_OK;
}

cudaError_t amg_apply(const AmgHier* H, const double* b, double* x, cudaStream_t st) {
  return vcycle(H, 0, b, x, st);
}

int amg_kernels_per_apply(const AmgHier* H) { return 4 * ((int)H->lev.size() - 1) + 1; }

int amg_nlevels(const AmgHier* H) { return (int)H->lev.size(); }

sstep_status amg_level_copy(const AmgHier* H, int l, int64_t* n, int64_t* nnz, int64_t* rowptr,
                            int32_t* colind, double* vals, int32_t* agg) {
  if (l < 0 || l >= (int)H->lev.size()) return SSTEP_ERR_INVALID;
  const AmgLevel& L = H->lev[l];
  if (n) *n = L.n;
  if (nnz) *nnz = L.nnz;
  if (rowptr) std::memcpy(rowptr, L.rp.data(), sizeof(int64_t) * (L.n + 1));
  if (colind) std::memcpy(colind, L.ci.data(), sizeof(int32_t) * L.nnz);
  if (vals) std::memcpy(vals, L.v.data(), sizeof(double) * L.nnz);
  if (agg && !L.agg.empty()) std::memcpy(agg, L.agg.data(), sizeof(int32_t) * L.n);
  return SSTEP_OK;
}

void amg_free(AmgHier* H) {
  if (!H) return;
  for (AmgLevel& L : H->lev) {
    void* ps[] = {L.rowptr, L.colind, L.vals, L.dinv, L.dagg, L.mptr, L.mem, L.x, L.b, L.r};
    for (void* p : ps)
      if (p) cudaFree(p);
  }
  if (H->cinv) cudaFree(H->cinv);
  delete H;
}

cudaError_t launch_cheb_combine(int64_t n, const double* t, const double* zq, const double* zprev,
                                double c1, double c2, double c3, double* znext, cudaStream_t st) {
  k_cheb_combine<<<grid_for(n), kAmgThreads, 0, st>>>(n, t, zq, zprev, c1, c2, c3, znext);
  return cudaGetLastError();
}

namespace {
// Power method step with a general M (Section 2): t = M^{-1} A v was formed by the caller; here
// t *= 1/lambda_(l-1) (so that v_(l-1) is normalised), lambda_l = ||t||, and the stop rule.
__global__ void __launch_bounds__(kAmgThreads) k_power_scale(int64_t n, double* t, Ctrl* c,
                                                              double* partials) {
  if (c->power_done) return;
  const double sc = c->inv_scale;
  double a[1] = {0.0}, tot[1];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double y = sc * t[i];
    t[i] = y;
    a[0] = fma(y, y, a[0]);
  }
  if (grid_sum_last<1>(a, partials, &c->ticket[TK_NORM], tot) && threadIdx.x == 0) {
    const double lam = sqrt(tot[0]);
    c->power_iters += 1;
    const bool conv = c->power_iters > 1 && c->power_tol > 0.0 &&
                      fabs(lam - c->lam) < c->power_tol * fabs(lam);
    c->lam = lam;
    c->inv_scale = lam > 0.0 ? 1.0 / lam : 0.0;
    if (conv || c->power_iters >= c->power_max || !(lam > 0.0)) c->power_done = 1;
  }
}
}  // namespace

cudaError_t launch_power_scale(int64_t n, double* t, Ctrl* c, double* partials, cudaStream_t st) {
  k_power_scale<<<grid_for(n), kAmgThreads, 0, st>>>(n, t, c, partials);
  return cudaGetLastError();
}

}  // namespace sstep
