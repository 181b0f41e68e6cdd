// api.cu -- the C ABI of libsstep.so (declared in include/sstep.h).
//
// A handle owns a device copy of A, M^{-1}, the Chebyshev scalars of Section 2, the basis
// blocks Z, AZ, Q, AQ (column-major, leading dimension n rounded up to 32), the vectors x, r, b
// (and p, Ap for PCG), a device control block and a partial-sum buffer.  One outer iteration
// of PCG-S (s MPK launches, one Gram reduction whose last CTA solves the reduced systems, one
// fused update whose last CTA applies the stop test) is captured once into a CUDA graph and
// replayed.  The host reads the device stop flag every `check_every` iterations while the
// next batch is already queued; launches after convergence return at kernel entry.
#include <algorithm>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

using namespace sstep;

namespace {

thread_local std::string g_err;

sstep_status fail(sstep_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      return fail(e_ == cudaErrorMemoryAllocation ? SSTEP_ERR_OOM : SSTEP_ERR_CUDA,            \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                        \
    }                                                                                         \
  } while (0)

#define CKS(expr)                  \
  do {                             \
    sstep_status s_ = (expr);      \
    if (s_ != SSTEP_OK) return s_; \
  } while (0)

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace

struct sstep_ctx {
  OpDesc op{};
  int prec_kind = SSTEP_PREC_JACOBI;
  Prec M{};
  sstep_opts o{};
  cudaStream_t user_stream = nullptr;
  cudaStream_t st = nullptr;   // stream all work is ordered on (captures need a non-legacy one)
  bool own_stream = false;
  int64_t nlaunch = 0;         // kernel launches issued (graph replays count their nodes)
  int64_t graph_nodes[5] = {0, 0, 0, 0, 0};
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int64_t n = 0, ld = 0, nnz = 0;
  int s = 4;
  // device memory
  int64_t* rowptr = nullptr;
  int32_t* colind = nullptr;
  double* vals = nullptr;
  double* dinv = nullptr;
  double* kappa = nullptr;  // Q1 operator: cell conductivities, then the vertex coefficients
  int64_t ncell = 0;
  double q1_gersh = 0.0;    // Q1 operator: Gershgorin lower bound found at set-up
  Q1TmaMaps* q1tma = nullptr;  // Q1 operator, FP32 path: tensor maps of the basis columns
  St7TmaMaps* st7tma = nullptr;  // 7-point stencil, FP32 path: tensor maps of r_hi and Z, or p
  double *Z = nullptr, *AZ = nullptr, *Q = nullptr, *AQ = nullptr;
  double *x = nullptr, *r = nullptr, *b = nullptr, *p = nullptr, *Ap = nullptr;
  double* partials = nullptr;
  double* hist = nullptr;
  double* red = nullptr;  // the reduced systems of every outer iteration (diagnostics)
  Ctrl* ctrl = nullptr;
  Ctrl* hctrl = nullptr;  // pinned host mirror
  // basis info
  double lmin = 0.0, lmax = 0.0, c_alpha = 0.0, c_sigma = 0.0, c_gamma = 1.0;
  int power_run = 0;
  double ms_setup = 0.0;
  // mixed path (FP32 basis): blocks, FP32 copies of the operator, x/r increments
  bool mixed = false;
  int rr_period = 0;
  int64_t ldf = 0;
  float *Zf = nullptr, *AZf = nullptr, *Qf = nullptr, *AQf = nullptr;
  float *rhi = nullptr, *rlo = nullptr, *xhi = nullptr, *xlo = nullptr;
  float *valsf = nullptr, *dinvf = nullptr, *kappaf = nullptr;
  float *pf = nullptr, *Apf = nullptr;  // FP32 PCG: search direction and A p
  // graphs of one outer iteration, per algorithm (index 3: the mixed literal form, rr_period
  // outer iterations followed by a residual replacement; index 4: FP32 PCG, rr_period
  // iterations followed by a residual replacement)
  cudaGraphExec_t gexec[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t graph_nodes4 = 0;
  // host polling of the stop flag
  cudaEvent_t poll_ev[2] = {nullptr, nullptr};
  int* poll_flags = nullptr;  // pinned, 4 ints
  // batched persistent solver (nsys > 1 or opts.persistent): everything lives in here
  BatchCtx* batch = nullptr;
  // aggregation AMG preconditioner (kind SSTEP_PREC_AMG) and its MPK work vector
  AmgHier* amg = nullptr;
  double* t = nullptr;
  int amg_coarse_max = 512, amg_max_levels = 25;
};

namespace {

sstep_status alloc(double** p, int64_t count) {
  CK(cudaMalloc((void**)p, sizeof(double) * (size_t)std::max<int64_t>(count, 1)));
  return SSTEP_OK;
}

// ---------------------------------------------------------------- kernel sequences

// Every Gram block as computed (Algorithm 1), or the symmetric shortcut (opt-in, one-reduction
// form only: the literal form always forms W = Q^T AQ in full, as Algorithm 1 prints it).
int full_blocks(const sstep_ctx* h) {
  return (h->o.algo == SSTEP_ALGO_LITERAL || h->o.gram_solver == SSTEP_GRAM_CHOLESKY ||
          h->o.gram_blocks != SSTEP_GRAM_BLOCKS_SYM) ? 1 : 0;
}

EpiArgs epi_base(sstep_ctx* h, int epi) {
  EpiArgs e{};
  e.epi = epi;
  e.M = h->M;
  e.ctrl = h->ctrl;
  e.partials = h->partials;
  return e;
}

// Algorithm 2 on residual r: Z = [z_1..z_s], AZ = [A z_1 .. A z_s].
// AMG: M^{-1} is a V-cycle, so SpMV, M^{-1} and the recurrence run as separate launches:
// z_1 = M^{-1} r; A z_q; t = M^{-1}(A z_q); z_{q+1} = c1 t - c2 z_q - c3 z_{q-1}.
sstep_status run_mpk_amg(sstep_ctx* h, const double* r, double* Z, double* AZ, int s) {
  const int64_t ld = h->ld, n = h->n;
  const int per = amg_kernels_per_apply(h->amg);
  CK(amg_apply(h->amg, r, Z, h->st));
  h->nlaunch += per;
  for (int q = 1; q <= s; ++q) {
    EpiArgs e = epi_base(h, EP_SPMV);
    e.u = Z + (q - 1) * ld;
    e.y = AZ + (q - 1) * ld;
    CK(launch_operator(h->op, e, h->st));
    ++h->nlaunch;
    if (q == s) break;
    CK(amg_apply(h->amg, AZ + (q - 1) * ld, h->t, h->st));
    h->nlaunch += per;
    const double c1 = q == 1 ? h->c_alpha : 2.0 * h->c_alpha;
    const double c2 = q == 1 ? h->c_sigma : 2.0 * h->c_sigma;
    CK(launch_cheb_combine(n, h->t, Z + (q - 1) * ld, q == 1 ? nullptr : Z + (q - 2) * ld, c1, c2,
                           h->c_gamma, Z + q * ld, h->st));
    ++h->nlaunch;
  }
  return SSTEP_OK;
}

sstep_status run_mpk(sstep_ctx* h, const double* r, double* Z, double* AZ, int s, Ctrl* ctrl) {
  if (h->amg) return run_mpk_amg(h, r, Z, AZ, s);
  const int64_t ld = h->ld;
  for (int q = 1; q <= s; ++q) {
    EpiArgs e = epi_base(h, q == 1 ? EP_MPK_FIRST : EP_MPK);
    e.ctrl = ctrl;
    if (q == 1) {
      e.u = r;
      e.z1 = Z;
      e.zprev = nullptr;
      e.c1 = h->c_alpha;  // z_2 = c_alpha M^{-1} A z_1 - c_sigma z_1
      e.c2 = h->c_sigma;
      e.c3 = 0.0;
    } else {
      e.u = Z + (q - 1) * ld;
      e.zprev = Z + (q - 2) * ld;
      e.c1 = 2.0 * h->c_alpha;  // z_{q+1} = 2 c_alpha M^{-1} A z_q - 2 c_sigma z_q - c_gamma z_{q-1}
      e.c2 = 2.0 * h->c_sigma;
      e.c3 = h->c_gamma;
    }
    e.y = AZ + (q - 1) * ld;
    e.znext = q < s ? Z + q * ld : nullptr;
    e.a1u = e.c1 * h->M.dinv_u;
    CK(launch_operator(h->op, e, h->st));
    ++h->nlaunch;
  }
  return SSTEP_OK;
}

sstep_status run_gram(sstep_ctx* h, int mode) {
  const int s = h->s;
  const int64_t ld = h->ld;
  if (full_blocks(h)) {
    cudaError_t e = launch_gram_tiled(mode, s, h->n, ld, h->Q, h->AQ, h->Z, h->AZ, h->r, h->ctrl,
                                      h->partials, h->st);
    if (e == cudaSuccess) {
      ++h->nlaunch;
      return SSTEP_OK;
    }
    if (e != cudaErrorNotSupported) CK(e);
    cudaGetLastError();
  }
  GramArgs g{};
  g.n = h->n;
  g.mode = mode;
  g.ctrl = h->ctrl;
  g.partials = h->partials;
  int nl = 0, nr = 0;
  g.ne = gram_pairs(mode, s, full_blocks(h), g.pairs, &nl, &nr);
  g.nl = nl;
  g.nr = nr;
  auto cols = [&](const double* base, int k, const double** dst) {
    for (int j = 0; j < k; ++j) dst[j] = base + j * ld;
  };
  switch (mode) {
    case GM_ONESYNC_FIRST:
      cols(h->Z, s, g.L);
      cols(h->AZ, s, g.R);
      g.R[s] = h->r;
      break;
    case GM_LITERAL_W:
      cols(h->Q, s, g.L);
      cols(h->AQ, s, g.R);
      g.R[s] = h->r;
      break;
    case GM_LITERAL_B2:
      cols(h->Q, s, g.L);
      cols(h->AZ, s, g.R);
      break;
    case GM_ONESYNC:
      cols(h->Q, s, g.L);
      cols(h->Z, s, g.L + s);
      cols(h->AQ, s, g.R);
      cols(h->AZ, s, g.R + s);
      g.R[2 * s] = h->r;
      break;
  }
  CK(launch_gram(g, h->st));
  ++h->nlaunch;
  return SSTEP_OK;
}

sstep_status run_update(sstep_ctx* h, int mode) {
  UpdArgs u{};
  u.n = h->n;
  u.ld = h->ld;
  u.s = h->s;
  u.mode = mode;
  u.Z = h->Z;
  u.AZ = h->AZ;
  u.Q = h->Q;
  u.AQ = h->AQ;
  u.x = h->x;
  u.r = h->r;
  u.alpha = h->ctrl->alpha;
  u.beta = (mode == UM_FIRST || mode == UM_XR || mode == UM_R) ? nullptr : h->ctrl->beta;
  u.ctrl = h->ctrl;
  u.partials = h->partials;
  u.ticket = &h->ctrl->ticket[TK_UPDATE];
  u.hist = h->hist;
  CK(launch_update(u, h->st));
  ++h->nlaunch;
  return SSTEP_OK;
}

// Direction-block update, Eq. (blockdirupdate) (Q <- Z + Q beta, AQ <- AZ + AQ beta; first
// block: Q <- Z, AQ <- AZ) followed by the step system of Section 2 (W = Q^T AQ, b1 = Q^T r,
// alpha = FGS(W, b1)).  Fused in one pass for s <= 8.
sstep_status run_upd_w(sstep_ctx* h, bool first) {
  UpdGramArgs a{h->n, h->ld, h->Z, h->AZ, h->Q, h->AQ, h->r, h->ctrl, h->partials, h->x};
  cudaError_t e = launch_upd_gram(a, h->s, first, h->st);
  if (e == cudaSuccess) {
    ++h->nlaunch;
    return SSTEP_OK;
  }
  if (e != cudaErrorNotSupported) CK(e);
  cudaGetLastError();
  if (first) {
    CK(cudaMemcpyAsync(h->Q, h->Z, sizeof(double) * h->ld * h->s, cudaMemcpyDeviceToDevice, h->st));
    CK(cudaMemcpyAsync(h->AQ, h->AZ, sizeof(double) * h->ld * h->s, cudaMemcpyDeviceToDevice, h->st));
  } else {
    CKS(run_update(h, UM_QAQ));
  }
  return run_gram(h, GM_LITERAL_W);
}

// ---------------------------------------------------------------- FP32-basis path

constexpr int kAlgoMixed = 3;    // graph index of the mixed literal form
constexpr int kAlgoPcgF32 = 4;   // graph index of FP32 PCG with FP64 residual replacement

int solve_algo(const sstep_ctx* h) {
  if (!h->mixed) return h->o.algo;
  return h->o.algo == SSTEP_ALGO_PCG ? kAlgoPcgF32 : kAlgoMixed;
}

MixedArgs mixed_args(sstep_ctx* h) {
  MixedArgs a{};
  a.n = h->n;
  a.ld = h->ldf;
  a.Z = h->Zf;
  a.AZ = h->AZf;
  a.Q = h->Qf;
  a.AQ = h->AQf;
  a.rhi = h->rhi;
  a.rlo = h->rlo;
  a.xhi = h->xhi;
  a.xlo = h->xlo;
  a.ctrl = h->ctrl;
  a.partials = h->partials;
  a.hist = h->hist;
  return a;
}

// Algorithm 2 in FP32 from r_hi (the FP32 value nearest r).
sstep_status run_mpk_f32(sstep_ctx* h) {
  const int64_t ld = h->ldf;
  const int s = h->s;
  MpkF32Args e{};
  e.dinv = h->dinvf;
  e.dinv_u = (float)h->M.dinv_u;
  e.valsf = h->valsf;
  e.ctrl = h->ctrl;
  if (h->op.kind == SSTEP_MATRIX_STENCIL) {
    for (int k = 0; k < h->op.st.points; ++k) e.w[k] = (float)h->op.st.w[k];
    e.wc = (float)h->op.st.wc;
  }
  for (int q = 1; q <= s; ++q) {
    e.first = q == 1;
    if (q == 1) {
      e.u = h->rhi;
      e.z1 = h->Zf;
      e.zprev = nullptr;
      e.c1 = (float)h->c_alpha;
      e.c2 = (float)h->c_sigma;
    } else {
      e.u = h->Zf + (q - 1) * ld;
      e.z1 = nullptr;
      e.zprev = h->Zf + (q - 2) * ld;
      e.c1 = (float)(2.0 * h->c_alpha);
      e.c2 = (float)(2.0 * h->c_sigma);
    }
    e.y = h->AZf + (q - 1) * ld;
    e.znext = q < s ? h->Zf + q * ld : nullptr;
    CK(launch_mpk_f32(h->op, e, h->st));
    ++h->nlaunch;
  }
  return SSTEP_OK;
}

// x += xhi + xlo (increments zeroed) after the pending step Q alpha of the FP32 s-step form.
cudaError_t fold_x(sstep_ctx* h) {
  const bool pcg = h->o.algo == SSTEP_ALGO_PCG;
  return launch_fold_x(h->x, h->xhi, h->xlo, h->n, h->ctrl, pcg ? nullptr : h->Qf, h->ldf,
                       pcg ? 0 : h->s, h->st);
}

// Residual replacement in FP64: x += xhi + xlo (increments zeroed), r = b - A x split into
// rhi + rlo, ||r||^2 and the stop test on it.
sstep_status run_rr(sstep_ctx* h) {
  CK(fold_x(h));
  EpiArgs e = epi_base(h, EP_RR);
  e.u = h->x;
  e.y = nullptr;
  e.b = h->b;
  e.rhi = h->rhi;
  e.rlo = h->rlo;
  CK(launch_operator(h->op, e, h->st));
  h->nlaunch += 2;
  return SSTEP_OK;
}

// One outer iteration of the mixed literal form (basis, conjugation, direction update with the
// previous step's x update, then step system, r update and stop test).
sstep_status mixed_outer(sstep_ctx* h) {
  const MixedArgs a = mixed_args(h);
  CKS(run_mpk_f32(h));
  CK(launch_gram_b2_f32(a, h->s, h->st));
  CK(launch_upd_gram_f32(a, h->s, false, h->st));
  CK(launch_update_xr_f32(a, h->s, h->st));
  h->nlaunch += h->s > 4 ? 4 : 3;
  return SSTEP_OK;
}

// First outer iteration of the mixed form: first block Q_0 = Z_0, step system, r update, stop test.
sstep_status mixed_first(sstep_ctx* h) {
  const MixedArgs a = mixed_args(h);
  CKS(run_mpk_f32(h));
  CK(launch_upd_gram_f32(a, h->s, true, h->st));
  CK(launch_update_xr_f32(a, h->s, h->st));
  h->nlaunch += h->s > 4 ? 3 : 2;
  return SSTEP_OK;
}

PcgF32Args pcgf_args(sstep_ctx* h) {
  PcgF32Args a{};
  a.n = h->n;
  a.p = h->pf;
  a.Ap = h->Apf;
  a.xhi = h->xhi;
  a.xlo = h->xlo;
  a.rhi = h->rhi;
  a.rlo = h->rlo;
  a.dinv = h->dinvf;
  a.dinv_u = (float)h->M.dinv_u;
  a.ctrl = h->ctrl;
  a.partials = h->partials;
  a.hist = h->hist;
  return a;
}

// FP32 PCG: A p in FP32 with p^T A p and alpha in the operator kernel's last CTA.
sstep_status pcgf_product(sstep_ctx* h) {
  MpkF32Args e{};
  e.u = h->pf;
  e.y = h->Apf;
  e.valsf = h->valsf;
  e.ctrl = h->ctrl;
  e.pap = 1;
  e.partials = h->partials;
  if (h->op.kind == SSTEP_MATRIX_STENCIL) {
    for (int k = 0; k < h->op.st.points; ++k) e.w[k] = (float)h->op.st.w[k];
    e.wc = (float)h->op.st.wc;
  }
  CK(launch_mpk_f32(h->op, e, h->st));
  ++h->nlaunch;
  return SSTEP_OK;
}

// One FP32 PCG iteration; `replace`: FP64 residual replacement before the direction update.
sstep_status pcgf_iteration(sstep_ctx* h, bool replace) {
  const PcgF32Args a = pcgf_args(h);
  CKS(pcgf_product(h));
  CK(launch_pcgf_update(a, h->st));
  ++h->nlaunch;
  if (replace) {
    CKS(run_rr(h));
    CK(launch_pcgf_rz(a, 0, h->st));
    ++h->nlaunch;
  }
  CK(launch_pcgf_pdir(a, 0, h->st));
  ++h->nlaunch;
  return SSTEP_OK;
}

// One outer iteration k >= 1 of each algorithm (what the graph captures).
sstep_status outer_iteration(sstep_ctx* h, int algo) {
  if (algo == kAlgoMixed) {
    for (int k = 0; k < h->rr_period; ++k) CKS(mixed_outer(h));
    CKS(run_rr(h));
  } else if (algo == kAlgoPcgF32) {
    for (int k = 0; k < h->rr_period; ++k) CKS(pcgf_iteration(h, k == h->rr_period - 1));
  } else if (algo == SSTEP_ALGO_ONESYNC) {
    CKS(run_mpk(h, h->r, h->Z, h->AZ, h->s, h->ctrl));
    CKS(run_gram(h, GM_ONESYNC));
    CKS(run_update(h, UM_FUSED));
  } else if (algo == SSTEP_ALGO_LITERAL) {
    // One outer iteration of Algorithm 1 starting at the new basis (the first update ran before):
    CKS(run_mpk(h, h->r, h->Z, h->AZ, h->s, h->ctrl));  // basis of r^(k+1) (Algorithm 2)
    CKS(run_gram(h, GM_LITERAL_B2));                     // conjugation: b2 = -Q^T AZ, beta
    CKS(run_upd_w(h, false));                            // Q, AQ update, then W, b1, alpha
    CKS(run_update(h, UM_R));                            // r update, stop test (x: pending)
  } else {
    EpiArgs e = epi_base(h, EP_PCG_AP);
    e.u = h->p;
    e.y = h->Ap;
    CK(launch_operator(h->op, e, h->st));
    PcgArgs a{h->n, h->x, h->r, h->p, h->Ap, h->M, h->ctrl, h->partials, h->hist};
    CK(launch_pcg_update(a, h->st));
    CK(launch_pcg_pdir(a, h->st));
    h->nlaunch += 3;
  }
  return SSTEP_OK;
}

sstep_status ensure_graph(sstep_ctx* h, int algo) {
  if (h->gexec[algo]) return SSTEP_OK;
  cudaGraph_t graph = nullptr;
  const int64_t before = h->nlaunch;
  CK(cudaStreamBeginCapture(h->st, cudaStreamCaptureModeRelaxed));
  sstep_status st = outer_iteration(h, algo);
  cudaError_t e = cudaStreamEndCapture(h->st, &graph);
  h->graph_nodes[algo] = h->nlaunch - before;  // captured, not executed
  h->nlaunch = before;
  if (st != SSTEP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return fail(SSTEP_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->gexec[algo], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->gexec[algo] = nullptr;
    return fail(SSTEP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  return SSTEP_OK;
}

sstep_status reset_ctrl(sstep_ctx* h) {
  Ctrl* c = h->hctrl;
  std::memset(c, 0, sizeof(Ctrl));
  c->rtol2 = h->o.rtol * h->o.rtol;
  c->status = SSTEP_NOT_CONVERGED;
  c->max_iters = h->o.max_outer;
  c->s = h->s;
  c->nu = h->o.sweeps;
  c->solver = h->o.gram_solver;
  // the FP32-basis path applies the FGS sweeps in operator form (s <= 8, all it supports): one
  // P_nu(W_k) serves alpha_k and beta_k, and the chain of the reduced solve is O(log nu)
  if (h->o.precision == SSTEP_PRECISION_FP32_RR && c->solver == SSTEP_GRAM_FGS && h->s <= 8)
    c->solver = SSTEP_GRAM_FGS_OPERATOR;
  c->full_gram = full_blocks(h);
  c->power_tol = h->o.power_tol;
  c->power_max = h->o.power_iters;
  c->red = h->red;
  c->red_max = h->o.max_outer + 1;
  c->red_stride = red_stride_for(h->s);
  CK(cudaMemcpyAsync(h->ctrl, c, sizeof(Ctrl), cudaMemcpyHostToDevice, h->st));
  return SSTEP_OK;
}

sstep_status read_ctrl(sstep_ctx* h) {
  CK(cudaMemcpyAsync(h->hctrl, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  return SSTEP_OK;
}

// Power method of Section 2 on M^{-1}A, entirely on the device (x and r serve as buffers).
sstep_status power_method(sstep_ctx* h) {
  CKS(reset_ctrl(h));
  if (h->o.power_v0) {
    CK(cudaMemcpyAsync(h->x, h->o.power_v0, sizeof(double) * h->n, cudaMemcpyDefault, h->st));
  } else {
    CK(launch_fill_splitmix(h->x, h->n, 1ull, h->st));
  }
  CK(launch_norm2(h->x, h->n, h->ctrl, h->partials, 0, h->st));
  if (h->amg) {  // t = M^{-1} A v by a V-cycle, then the scaling and the stop rule
    double* v = h->x;
    double* t = h->b;
    for (int it = 0; it < h->o.power_iters; ++it) {
      EpiArgs e = epi_base(h, EP_SPMV);
      e.u = v;
      e.y = h->r;
      CK(launch_operator(h->op, e, h->st));
      CK(amg_apply(h->amg, h->r, t, h->st));
      CK(launch_power_scale(h->n, t, h->ctrl, h->partials, h->st));
      std::swap(v, t);
    }
    CKS(read_ctrl(h));
    h->lmax = h->hctrl->lam;
    h->power_run = h->hctrl->power_iters;
    if (!(h->lmax > 0.0) || h->lmax != h->lmax)
      return fail(SSTEP_ERR_INVALID, "power method produced no positive estimate of lambda_max");
    return SSTEP_OK;
  }
  double* buf[2] = {h->x, h->r};
  for (int it = 0; it < h->o.power_iters; ++it) {
    EpiArgs e = epi_base(h, EP_POWER);
    e.u = buf[it & 1];
    e.y = buf[(it + 1) & 1];
    CK(launch_operator(h->op, e, h->st));
  }
  CKS(read_ctrl(h));
  h->lmax = h->hctrl->lam;
  h->power_run = h->hctrl->power_iters;
  if (!(h->lmax > 0.0) || h->lmax != h->lmax)
    return fail(SSTEP_ERR_INVALID, "power method produced no positive estimate of lambda_max");
  return SSTEP_OK;
}

double stencil_gershgorin(const StencilOp& st, int jacobi) {
  // Minimum over row classes (first / interior / last index per dimension) of d - sum|w_nb|.
  const int nd[3] = {st.nx, st.ny, st.nz};
  std::vector<int> offs;  // (dx, dy, dz) of each weight
  double lo = 1e308;
  for (int cz = 0; cz < 3; ++cz)
    for (int cy = 0; cy < 3; ++cy)
      for (int cx = 0; cx < 3; ++cx) {
        const int cls[3] = {cx, cy, cz};
        bool exists = true;
        for (int d = 0; d < 3; ++d) {
          const int N = nd[d];
          if (cls[d] == 1 && N < 3) exists = false;  // interior needs N >= 3
          if (cls[d] == 2 && N < 2) exists = false;  // distinct last needs N >= 2
        }
        if (!exists) continue;
        double off = 0.0;
        int k = 0;
        for (int dz = -1; dz <= 1; ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              bool used;
              if (st.points == 27) used = true;
              else if (st.points == 7) used = (std::abs(dx) + std::abs(dy) + std::abs(dz) <= 1);
              else used = (dz == 0 && std::abs(dx) + std::abs(dy) <= 1);
              if (!used) continue;
              const double w = st.w[k++];
              if (dx == 0 && dy == 0 && dz == 0) continue;
              const int dd[3] = {dx, dy, dz};
              bool present = true;
              for (int d = 0; d < 3; ++d) {
                const int N = nd[d];
                const int idx = cls[d] == 0 ? 0 : (cls[d] == 1 ? 1 : N - 1);
                const int j = idx + dd[d];
                if (j < 0 || j >= N) present = false;
              }
              if (present) off += std::fabs(w);
            }
        const double b = jacobi ? 1.0 - off / st.wc : st.wc - off;
        lo = std::min(lo, b);
      }
  return lo > 0.0 ? lo : 0.0;
}

sstep_status validate_opts(const sstep_opts* o) {
  if (o->s < 1 || o->s > kMaxS) return fail(SSTEP_ERR_INVALID, "s must be in 1..16");
  if (o->sweeps < 0) return fail(SSTEP_ERR_INVALID, "sweeps must be >= 0");
  if (!(o->rtol >= 0.0)) return fail(SSTEP_ERR_INVALID, "rtol must be >= 0");
  if (o->max_outer < 0) return fail(SSTEP_ERR_INVALID, "max_outer must be >= 0");
  if (o->algo < 0 || o->algo > 2) return fail(SSTEP_ERR_INVALID, "unknown algo");
  if (o->gram_solver < 0 || o->gram_solver > 2) return fail(SSTEP_ERR_INVALID, "unknown gram_solver");
  if (o->gram_solver == SSTEP_GRAM_FGS_OPERATOR && o->s > 8)
    return fail(SSTEP_ERR_UNSUPPORTED, "the FGS operator form takes s <= 8");
  if (o->power_iters < 1 && !(o->lambda_max > 0.0))
    return fail(SSTEP_ERR_INVALID, "power_iters must be >= 1 when lambda_max is not given");
  if (o->precision != SSTEP_PRECISION_FP64 && o->precision != SSTEP_PRECISION_FP32_RR)
    return fail(SSTEP_ERR_INVALID, "unknown precision");
  if (o->precision == SSTEP_PRECISION_FP32_RR) {
    if (o->algo != SSTEP_ALGO_LITERAL && o->algo != SSTEP_ALGO_PCG)
      return fail(SSTEP_ERR_UNSUPPORTED,
                  "the FP32-basis path implements the literal form and classical PCG");
    if (o->s > 8) return fail(SSTEP_ERR_UNSUPPORTED, "the FP32-basis path supports s <= 8");
    if (o->gram_solver == SSTEP_GRAM_CHOLESKY)
      return fail(SSTEP_ERR_UNSUPPORTED, "the FP32-basis path uses FGS reduced solves");
  }
  return SSTEP_OK;
}

void destroy(sstep_ctx* h) {
  if (!h) return;
  if (h->batch) batch_free(h->batch);
  if (h->amg) amg_free(h->amg);
  if (h->q1tma) q1_tma_free(h->q1tma);
  if (h->st7tma) st7_tma_free(h->st7tma);
  if (h->t) cudaFree(h->t);
  if (h->st) cudaStreamSynchronize(h->st);
  for (auto& g : h->gexec)
    if (g) cudaGraphExecDestroy(g);
  void* fbufs[] = {h->Zf,  h->AZf, h->Qf,    h->AQf,   h->rhi,   h->rlo, h->xhi,
                   h->xlo, h->valsf, h->dinvf, h->kappaf, h->pf,    h->Apf};
  for (void* p : fbufs)
    if (p) cudaFree(p);
  void* bufs[] = {h->rowptr, h->colind, h->vals, h->dinv, h->Z, h->AZ, h->Q, h->AQ, h->x, h->r,
                  h->b, h->p, h->Ap, h->partials, h->hist, h->ctrl, h->red,
                  h->kappa};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (h->hctrl) cudaFreeHost(h->hctrl);
  if (h->poll_flags) cudaFreeHost(h->poll_flags);
  for (auto& e : h->poll_ev)
    if (e) cudaEventDestroy(e);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->st && h->own_stream) cudaStreamDestroy(h->st);
  delete h;
}

// Q1 set-up pass: conductivities finite and positive, M^{-1} = 1 / a_ii into h->dinv (when
// allocated), and the Gershgorin lower bound of M^{-1} A (Jacobi) or A into h->q1_gersh.
sstep_status q1_setup(sstep_ctx* h) {
  const int g = q1_setup_ctas(h->n);
  int* bad = nullptr;
  CK(cudaMallocAsync((void**)&bad, sizeof(int), h->st));
  CK(cudaMemsetAsync(bad, 0, sizeof(int), h->st));
  CK(launch_q1_setup(h->op.q1, h->prec_kind == SSTEP_PREC_JACOBI, h->dinv, h->partials, bad,
                     h->st));
  std::vector<double> mins(g);
  int hbad = 0;
  CK(cudaMemcpyAsync(mins.data(), h->partials, sizeof(double) * g, cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, h->st));
  CK(cudaFreeAsync(bad, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (hbad) return fail(SSTEP_ERR_INVALID, "Q1 conductivities must be finite and positive");
  double lo = 1e308;
  for (double v : mins) lo = std::min(lo, v);
  h->q1_gersh = lo;
  return SSTEP_OK;
}

sstep_status setup_impl(const sstep_matrix* A, int nsys, const sstep_precond* M,
                        const sstep_opts* o, void* stream, sstep_ctx* h) {
  const double t0 = now_ms();
  if (!A || !o) return fail(SSTEP_ERR_INVALID, "null matrix or options");
  if (nsys != 1) return fail(SSTEP_ERR_UNSUPPORTED, "nsys must be 1");
  CKS(validate_opts(o));
  h->o = *o;
  h->s = o->s;
  if (o->check_every <= 0) h->o.check_every = 0;
  h->prec_kind = M ? M->kind : SSTEP_PREC_JACOBI;
  if (h->prec_kind != SSTEP_PREC_NONE && h->prec_kind != SSTEP_PREC_JACOBI &&
      h->prec_kind != SSTEP_PREC_AMG)
    return fail(SSTEP_ERR_INVALID, "unknown preconditioner kind");
  if (h->prec_kind == SSTEP_PREC_AMG) {
    if (A->kind != SSTEP_MATRIX_CSR)
      return fail(SSTEP_ERR_UNSUPPORTED, "the AMG preconditioner takes CSR operators");
    if (o->algo == SSTEP_ALGO_PCG || o->precision != SSTEP_PRECISION_FP64)
      return fail(SSTEP_ERR_UNSUPPORTED, "the AMG preconditioner serves the FP64 s-step forms");
    if (M->amg_coarse_max) h->amg_coarse_max = M->amg_coarse_max;
    if (M->amg_max_levels) h->amg_max_levels = M->amg_max_levels;
  }
  h->user_stream = (cudaStream_t)stream;
  // Work runs on the caller's stream when one is given (so the caller's CUDA events bracket
  // the kernels).  The legacy default stream cannot be captured, so NULL gets a private
  // *blocking* stream: it stays ordered with the caller's work on the legacy default stream
  // (for example the kernels that produced b or the CSR values).
  if (h->user_stream) {
    h->st = h->user_stream;
    h->own_stream = false;
  } else {
    CK(cudaStreamCreateWithFlags(&h->st, cudaStreamDefault));
    h->own_stream = true;
  }
  CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));

  // ---- operator
  h->op.kind = A->kind;
  if (A->kind == SSTEP_MATRIX_STENCIL) {
    StencilOp& st = h->op.st;
    st.nx = A->nx;
    st.ny = A->ny;
    st.nz = A->nz;
    st.points = A->points;
    if (!(A->points == 5 || A->points == 7 || A->points == 27))
      return fail(SSTEP_ERR_INVALID, "stencil points must be 5, 7 or 27");
    if (A->nx < 1 || A->ny < 1 || A->nz < 1) return fail(SSTEP_ERR_INVALID, "stencil dims must be >= 1");
    if (A->points == 5 && A->nz != 1) return fail(SSTEP_ERR_INVALID, "5-point stencil needs nz = 1");
    const int cidx = A->points == 5 ? 2 : (A->points == 7 ? 3 : 13);
    if (A->weights) {
      for (int k = 0; k < A->points; ++k) st.w[k] = A->weights[k];
    } else {
      for (int k = 0; k < A->points; ++k) st.w[k] = -1.0;
      st.w[cidx] = A->points == 5 ? 4.0 : (A->points == 7 ? 6.0 : 26.0);
    }
    st.wc = st.w[cidx];
    st.poisson = 1;
    for (int k = 0; k < A->points; ++k)
      if (k != cidx && st.w[k] != -1.0) st.poisson = 0;
    h->n = (int64_t)A->nx * A->ny * A->nz;
    if (A->n != 0 && A->n != h->n) return fail(SSTEP_ERR_INVALID, "stencil n != nx*ny*nz");
    if (h->prec_kind == SSTEP_PREC_JACOBI && !(st.wc > 0.0))
      return fail(SSTEP_ERR_INVALID, "Jacobi needs a positive diagonal");
    h->M.dinv = nullptr;
    h->M.dinv_u = h->prec_kind == SSTEP_PREC_JACOBI ? 1.0 / st.wc : 1.0;
  } else if (A->kind == SSTEP_MATRIX_CSR) {
    if (A->n < 1 || A->nnz < 1 || !A->rowptr || !A->colind || !A->vals)
      return fail(SSTEP_ERR_INVALID, "CSR needs n, nnz and three arrays");
    if (A->n >= ((int64_t)1 << 31)) return fail(SSTEP_ERR_UNSUPPORTED, "CSR with n >= 2^31");
    h->n = A->n;
    CK(cudaMalloc(&h->rowptr, sizeof(int64_t) * (A->n + 1)));
    CK(cudaMalloc(&h->colind, sizeof(int32_t) * A->nnz));
    CK(cudaMalloc(&h->vals, sizeof(double) * A->nnz));
    CK(cudaMemcpyAsync(h->rowptr, A->rowptr, sizeof(int64_t) * (A->n + 1), cudaMemcpyDefault, h->st));
    CK(cudaMemcpyAsync(h->colind, A->colind, sizeof(int32_t) * A->nnz, cudaMemcpyDefault, h->st));
    CK(cudaMemcpyAsync(h->vals, A->vals, sizeof(double) * A->nnz, cudaMemcpyDefault, h->st));
    h->op.csr = CsrOp{A->n, h->rowptr, h->colind, h->vals};
    h->nnz = A->nnz;
    {
      int* bad = nullptr;
      CK(cudaMalloc(&bad, sizeof(int)));
      CK(cudaMemsetAsync(bad, 0, sizeof(int), h->st));
      CK(launch_csr_check(h->op.csr, A->nnz, bad, h->st));
      int hbad = 0;
      CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      cudaFree(bad);
      if (hbad) return fail(SSTEP_ERR_INVALID, "CSR arrays are inconsistent (row pointers or column indices)");
    }
  } else if (A->kind == SSTEP_MATRIX_Q1) {
    if (A->nx < 1 || A->ny < 1 || A->nz < 1 || !A->weights)
      return fail(SSTEP_ERR_INVALID, "Q1 needs nx, ny, nz >= 1 and the cell conductivities");
    h->n = (int64_t)A->nx * A->ny * A->nz;
    if (A->n != 0 && A->n != h->n) return fail(SSTEP_ERR_INVALID, "Q1 n != nx*ny*nz");
    h->ncell = (int64_t)(A->nx + 1) * (A->ny + 1) * (A->nz + 1);
    // conductivities, then (256-byte aligned) the 13 x n vertex coefficients that the set-up
    // pass writes for the FP64 kernels
    CK(cudaMalloc(&h->kappa, sizeof(double) * (round_up(h->ncell, 32) + 13 * h->n)));
    CK(cudaMemcpyAsync(h->kappa, A->weights, sizeof(double) * h->ncell, cudaMemcpyDefault, h->st));
    h->op.q1 = Q1Op{A->nx, A->ny, A->nz, h->kappa, nullptr, (int)round_up(A->nx + 1, 4),
                    nullptr};
  } else {
    return fail(SSTEP_ERR_INVALID, "unknown matrix kind");
  }
  h->op.n = h->n;
  h->ld = round_up(h->n, 32);

  // ---- buffers
  const int64_t ld = h->ld;
  const int s = h->s;
  CKS(alloc(&h->Z, ld * s));
  CKS(alloc(&h->AZ, ld * s));
  CKS(alloc(&h->Q, ld * s));
  CKS(alloc(&h->AQ, ld * s));
  CKS(alloc(&h->x, ld));
  CKS(alloc(&h->r, ld));
  CKS(alloc(&h->b, ld));
  if (h->o.algo == SSTEP_ALGO_PCG) {
    CKS(alloc(&h->p, ld));
    CKS(alloc(&h->Ap, ld));
  }
  CK(cudaMemsetAsync(h->Q, 0, sizeof(double) * ld * s, h->st));
  CK(cudaMemsetAsync(h->AQ, 0, sizeof(double) * ld * s, h->st));
  const int64_t part = std::max<int64_t>(
      {(int64_t)operator_grid_ctas(h->op) * 2, (int64_t)gram_ctas() * kMaxEntries,
       (int64_t)update_ctas(h->n), (int64_t)pcg_ctas(h->n) * 2, (int64_t)gershgorin_ctas(h->n) + 1,
       (int64_t)4096});
  CKS(alloc(&h->partials, part));
  CKS(alloc(&h->hist, (int64_t)h->o.max_outer + 2));
  CKS(alloc(&h->red, ((int64_t)h->o.max_outer + 2) * red_stride_for(s)));
  CK(cudaMalloc(&h->ctrl, sizeof(Ctrl)));
  CK(cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->st));
  CK(cudaMallocHost(&h->hctrl, sizeof(Ctrl)));
  std::memset(h->hctrl, 0, sizeof(Ctrl));
  CK(cudaMallocHost(&h->poll_flags, sizeof(int) * 4));
  CK(cudaEventCreateWithFlags(&h->poll_ev[0], cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&h->poll_ev[1], cudaEventDisableTiming));
  CK(gram_init());

  // ---- Q1: check the conductivities, Jacobi M^{-1} and the Gershgorin bound in one pass
  if (A->kind == SSTEP_MATRIX_Q1) {
    if (h->prec_kind == SSTEP_PREC_JACOBI) CKS(alloc(&h->dinv, ld));
    CKS(q1_setup(h));
    h->M.dinv = h->dinv;
    h->M.dinv_u = h->dinv ? 0.0 : 1.0;
  }

  // ---- Jacobi M^{-1} for CSR
  if (A->kind == SSTEP_MATRIX_CSR) {
    if (h->prec_kind == SSTEP_PREC_AMG) {
      CKS(amg_build(h->rowptr, h->colind, h->vals, h->n, h->nnz, h->amg_coarse_max,
                    h->amg_max_levels, h->st, &h->amg));
      CKS(alloc(&h->t, ld));
      h->M.dinv = nullptr;
      h->M.dinv_u = 1.0;
    } else if (h->prec_kind == SSTEP_PREC_JACOBI) {
      CKS(alloc(&h->dinv, ld));
      int* bad = nullptr;
      CK(cudaMalloc(&bad, sizeof(int)));
      CK(cudaMemsetAsync(bad, 0, sizeof(int), h->st));
      CK(launch_jacobi_csr(h->op.csr, h->dinv, bad, h->st));
      int hbad = 0;
      CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      cudaFree(bad);
      if (hbad) return fail(SSTEP_ERR_INVALID, "Jacobi needs a positive diagonal entry in every row");
      h->M.dinv = h->dinv;
      h->M.dinv_u = 0.0;
    } else {
      h->M.dinv = nullptr;
      h->M.dinv_u = 1.0;
    }
  }

  // ---- Chebyshev interval (Section 2)
  const int jac = h->prec_kind == SSTEP_PREC_JACOBI;
  if (o->lambda_min < 0.0 && h->amg) {
    h->lmin = 0.0;  // no cheap bound for a V-cycle: Section 2's 0
  } else if (o->lambda_min < 0.0) {
    if (A->kind == SSTEP_MATRIX_STENCIL) {
      h->lmin = stencil_gershgorin(h->op.st, jac);
    } else if (A->kind == SSTEP_MATRIX_Q1) {
      h->lmin = h->q1_gersh > 0.0 ? h->q1_gersh : 0.0;
    } else {
      const int g = gershgorin_ctas(h->n);
      CK(launch_gershgorin_csr(h->op.csr, jac, h->partials, h->st));
      std::vector<double> mins(g);
      CK(cudaMemcpyAsync(mins.data(), h->partials, sizeof(double) * g, cudaMemcpyDeviceToHost, h->st));
      CK(cudaStreamSynchronize(h->st));
      double lo = 1e308;
      for (double v : mins) lo = std::min(lo, v);
      h->lmin = lo > 0.0 ? lo : 0.0;
    }
  } else {
    h->lmin = o->lambda_min;
  }
  if (o->lambda_max > 0.0) {
    h->lmax = o->lambda_max;
    h->power_run = 0;
  } else {
    CKS(power_method(h));
  }
  if (!(h->lmax > h->lmin)) return fail(SSTEP_ERR_INVALID, "lambda_max must exceed lambda_min");
  h->c_alpha = 2.0 / (h->lmax - h->lmin);
  h->c_sigma = (h->lmax + h->lmin) / (h->lmax - h->lmin);
  h->c_gamma = 1.0;

  // ---- FP32-basis path: FP32 blocks and increments, FP32 copies of the operator
  if (h->o.precision == SSTEP_PRECISION_FP32_RR) {
    const bool pcg = h->o.algo == SSTEP_ALGO_PCG;
    h->mixed = true;
    // PCG: one replacement per 16 iterations by default, the spacing in CG steps of the
    // s-step form's default (every s outer iterations of s steps each, s = 4)
    h->rr_period = h->o.rr_period > 0 ? h->o.rr_period : (pcg ? 16 : h->s);
    h->ldf = round_up(h->n, 64);
    const int64_t lf = h->ldf;
    auto fal = [&](float** p, int64_t count) -> cudaError_t {
      return cudaMalloc((void**)p, sizeof(float) * (size_t)std::max<int64_t>(count, 1));
    };
    if (pcg) {
      CK(fal(&h->pf, lf));
      CK(fal(&h->Apf, lf));
    } else {
      CK(fal(&h->Zf, lf * s));
      CK(fal(&h->AZf, lf * s));
      CK(fal(&h->Qf, lf * s));
      CK(fal(&h->AQf, lf * s));
    }
    CK(fal(&h->rhi, lf));
    CK(fal(&h->rlo, lf));
    CK(fal(&h->xhi, lf));
    CK(fal(&h->xlo, lf));
    if (A->kind == SSTEP_MATRIX_CSR) {
      CK(fal(&h->valsf, A->nnz));
      CK(launch_d2f(h->vals, h->valsf, A->nnz, h->st));
      if (h->dinv) {
        CK(fal(&h->dinvf, lf));
        CK(launch_d2f(h->dinv, h->dinvf, h->n, h->st));
      }
    } else if (A->kind == SSTEP_MATRIX_Q1) {
      CK(fal(&h->kappaf, (int64_t)h->op.q1.kpitch * (A->ny + 1) * (A->nz + 1)));
      h->op.q1.kappaf = h->kappaf;
      CK(launch_q1_kappaf(h->op.q1, h->kappaf, h->st));
      // the vectors the TMA-fed kernel reads: the basis columns, or PCG's direction p
      std::vector<const float*> cols;
      if (pcg) cols.push_back(h->pf);
      else
        for (int c = 0; c < s; ++c) cols.push_back(h->Zf + c * lf);
      // null (or SSTEP_Q1_TMA=0 in the environment): the plain-load kernel serves every step
      const char* tma_env = std::getenv("SSTEP_Q1_TMA");
      if (!(tma_env && tma_env[0] == '0'))
        h->q1tma = q1_tma_build(h->op.q1, cols.data(), (int)cols.size());
      h->op.q1.tma = h->q1tma;
      if (h->dinv) {
        CK(fal(&h->dinvf, lf));
        CK(launch_d2f(h->dinv, h->dinvf, h->n, h->st));
      }
    } else if (A->points == 27) {
      return fail(SSTEP_ERR_UNSUPPORTED, "the FP32-basis path takes 27-point operators as CSR");
    }
    if (A->kind == SSTEP_MATRIX_STENCIL && A->points == 7) {
      // the vectors the TMA-fed 7-point steps read: r_hi and the basis columns, or PCG's p
      std::vector<const float*> cols;
      if (pcg) {
        cols.push_back(h->pf);
      } else {
        cols.push_back(h->rhi);
        for (int c = 0; c < s; ++c) cols.push_back(h->Zf + c * lf);
      }
      // null (or SSTEP_STENCIL_TMA=0 in the environment): the register-fed kernel serves them
      const char* tma_env = std::getenv("SSTEP_STENCIL_TMA");
      if (!(tma_env && tma_env[0] == '0'))
        h->st7tma = st7_tma_build(h->op.st, cols.data(), (int)cols.size());
      h->op.st.tma = h->st7tma;
    }
  }
  CK(cudaStreamSynchronize(h->st));
  h->ms_setup = now_ms() - t0;
  return SSTEP_OK;
}

int auto_check_every(const sstep_ctx* h) {
  if (h->o.check_every > 0) return h->o.check_every;
  // Roughly one host poll per millisecond of device work.
  const double us_per_iter = 3.0 * (h->o.algo == SSTEP_ALGO_PCG ? 3 : h->s + 2) +
                             (double)h->n * (h->o.algo == SSTEP_ALGO_PCG ? 1.0 : h->s) * 2e-5;
  int b = (int)(1000.0 / us_per_iter);
  return std::max(1, std::min(32, b));
}

sstep_status solve_impl(sstep_ctx* h, const double* b, double* x, sstep_info* info) {
  const double t0 = now_ms();
  const int64_t n = h->n;
  const int algo = solve_algo(h);
  // Order against the caller's stream: inputs produced there are complete before we read.
  CK(cudaEventRecord(h->ev_in, h->user_stream));
  CK(cudaStreamWaitEvent(h->st, h->ev_in, 0));
  CK(cudaMemcpyAsync(h->b, b, sizeof(double) * n, cudaMemcpyDefault, h->st));
  CK(cudaMemcpyAsync(h->x, x, sizeof(double) * n, cudaMemcpyDefault, h->st));
  if (h->mixed) {
    CK(cudaMemsetAsync(h->xhi, 0, sizeof(float) * n, h->st));
    CK(cudaMemsetAsync(h->xlo, 0, sizeof(float) * n, h->st));
  }
  CKS(reset_ctrl(h));
  const int64_t launches0 = h->nlaunch;
  // initial residual r^(0) = b - A x^(0); ||b||^2, ||r||^2 (mixed path: r kept as FP32 hi + lo)
  {
    EpiArgs e = epi_base(h, EP_RESID);
    e.u = h->x;
    e.y = h->mixed ? nullptr : h->r;
    e.b = h->b;
    e.rhi = h->mixed ? h->rhi : nullptr;
    e.rlo = h->mixed ? h->rlo : nullptr;
    CK(launch_operator(h->op, e, h->st));
    ++h->nlaunch;
  }
  // first outer iteration (not captured: it differs from the rest)
  const int maxit = h->o.max_outer;
  if (algo == kAlgoMixed) {
    if (maxit > 0) CKS(mixed_first(h));
  } else if (algo == kAlgoPcgF32) {
    const PcgF32Args a = pcgf_args(h);
    CK(launch_pcgf_rz(a, 1, h->st));
    CK(launch_pcgf_pdir(a, 1, h->st));
    h->nlaunch += 2;
  } else if (algo == SSTEP_ALGO_ONESYNC) {
    if (maxit > 0) {
      CKS(run_mpk(h, h->r, h->Z, h->AZ, h->s, h->ctrl));
      CKS(run_gram(h, GM_ONESYNC_FIRST));
      CKS(run_update(h, UM_FIRST));
    }
  } else if (algo == SSTEP_ALGO_LITERAL) {
    if (maxit > 0) {
      CKS(run_mpk(h, h->r, h->Z, h->AZ, h->s, h->ctrl));  // basis of r^(0)
      CKS(run_upd_w(h, true));                            // Q_0 = Z_0; W, b1, alpha
      CKS(run_update(h, UM_R));                           // r update and stop test
    }
  } else {
    PcgArgs a{h->n, h->x, h->r, h->p, h->Ap, h->M, h->ctrl, h->partials, h->hist};
    CK(launch_pcg_init(a, h->st));
    ++h->nlaunch;
  }
  CKS(ensure_graph(h, algo));
  // Replay the captured outer iteration; poll the stop flag one batch behind.
  const int B = auto_check_every(h);
  // PCG-S ran its first outer iteration above
  int launched = (algo == SSTEP_ALGO_PCG || algo == kAlgoPcgF32) ? 0 : 1;
  // outer iterations per replay
  const int per_graph = (algo == kAlgoMixed || algo == kAlgoPcgF32) ? h->rr_period : 1;
  bool finished = false;
  Ctrl* hc = h->hctrl;
  int* flags = h->poll_flags;
  flags[0] = flags[1] = flags[2] = flags[3] = 0;
  int pending = -1;  // batch whose poll is outstanding
  int batch = 0;
  sstep_status st = SSTEP_OK;
  while (!finished) {
    const int todo = std::min(B, (maxit - launched + per_graph - 1) / per_graph);
    if (todo > 0) {
      for (int k = 0; k < todo; ++k) {
        cudaError_t e = cudaGraphLaunch(h->gexec[algo], h->st);
        if (e != cudaSuccess) {
          st = fail(SSTEP_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
          break;
        }
      }
      if (st != SSTEP_OK) break;
      launched += todo * per_graph;
      h->nlaunch += (int64_t)todo * h->graph_nodes[algo];
      const int slot = batch & 1;
      CK(cudaMemcpyAsync(flags + 2 * slot, &h->ctrl->done, sizeof(int), cudaMemcpyDeviceToHost, h->st));
      CK(cudaEventRecord(h->poll_ev[slot], h->st));
    }
    if (pending >= 0) {
      const int ps = pending & 1;
      CK(cudaEventSynchronize(h->poll_ev[ps]));
      if (flags[2 * ps]) finished = true;
    }
    if (todo <= 0) finished = true;  // nothing left to launch
    pending = (todo > 0) ? batch : -1;
    ++batch;
  }
  CK(cudaStreamSynchronize(h->st));
  if (st != SSTEP_OK) return st;
  if (h->mixed) {  // fold the last increments (and the pending step) into the FP64 solution
    CK(fold_x(h));
    ++h->nlaunch;
  } else if (h->o.algo == SSTEP_ALGO_LITERAL) {  // the step x += Q alpha still pending
    CK(launch_flush_x(h->x, h->Q, n, h->ld, h->s, h->ctrl, h->st));
    ++h->nlaunch;
  }
  CKS(read_ctrl(h));
  // b = 0: x = 0
  if (hc->nb2 == 0.0) CK(cudaMemsetAsync(h->x, 0, sizeof(double) * n, h->st));
  // true residual ||b - A x|| (reported, not used to stop)
  {
    EpiArgs e = epi_base(h, EP_TRUERES);
    e.u = h->x;
    e.b = h->b;
    CK(launch_operator(h->op, e, h->st));
    ++h->nlaunch;
  }
  double true_rr = 0.0;
  CK(cudaMemcpyAsync(&true_rr, &h->ctrl->sums[0], sizeof(double), cudaMemcpyDeviceToHost, h->st));
  CK(cudaMemcpyAsync(x, h->x, sizeof(double) * n, cudaMemcpyDefault, h->st));
  CK(cudaStreamSynchronize(h->st));
  CK(cudaEventRecord(h->ev_out, h->st));
  CK(cudaStreamWaitEvent(h->user_stream, h->ev_out, 0));
  const sstep_status result = (sstep_status)hc->status;
  if (info) {
    info->status = result;
    info->outer_iters = hc->iters;
    info->inner_equiv = h->o.algo == SSTEP_ALGO_PCG ? hc->iters : hc->iters * h->s;
    const double nb = std::sqrt(hc->nb2);
    info->relres = nb > 0.0 ? std::sqrt(hc->rr) / nb : 0.0;
    info->relres_true = nb > 0.0 ? std::sqrt(true_rr) / nb : 0.0;
    info->lambda_max = h->lmax;
    info->lambda_min = h->lmin;
    info->ms_setup = h->ms_setup;
    info->ms_solve = now_ms() - t0;
    info->launches = h->nlaunch - launches0;
  }
  if (result != SSTEP_OK && result != SSTEP_NOT_CONVERGED)
    g_err = std::string("solve ended with ") + sstep_status_string(result);
  return result;
}

}  // namespace

void sstep::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

// ================================================================== C ABI

extern "C" {

void sstep_default_opts(sstep_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->s = 4;
  o->sweeps = 2;
  o->rtol = 1e-8;
  o->max_outer = 10000;
  o->algo = SSTEP_ALGO_LITERAL;
  o->gram_solver = SSTEP_GRAM_FGS;
  o->power_iters = 50;
  o->power_tol = 1e-3;
  o->lambda_min = 0.0;
  o->lambda_max = 0.0;
  o->power_v0 = nullptr;
  o->check_every = 0;
  o->gram_blocks = SSTEP_GRAM_BLOCKS_FULL;
  o->precision = SSTEP_PRECISION_FP64;
  o->rr_period = 0;
  o->persistent = 0;
  o->cluster = 0;
  o->block_threads = 0;
}

sstep_status sstep_setup(const sstep_matrix* A, int nsys, const sstep_precond* M,
                         const sstep_opts* o, void* stream, sstep_handle* out) {
  g_err.clear();
  if (!out) return fail(SSTEP_ERR_INVALID, "out is null");
  *out = nullptr;
  sstep_ctx* h = new (std::nothrow) sstep_ctx();
  if (!h) return fail(SSTEP_ERR_OOM, "host allocation failed");
  if (o && (nsys > 1 || o->persistent)) {
    g_err.clear();
    sstep_status st = batch_setup(A, nsys, M, o, (cudaStream_t)stream, &h->batch);
    if (st != SSTEP_OK) {
      delete h;
      return st;
    }
    *out = h;
    return SSTEP_OK;
  }
  sstep_status st = setup_impl(A, nsys, M, o, stream, h);
  if (st != SSTEP_OK) {
    std::string keep = g_err;
    destroy(h);
    cudaGetLastError();
    g_err = keep;
    return st;
  }
  *out = h;
  return SSTEP_OK;
}

sstep_status sstep_solve(sstep_handle h, const double* b, double* x, sstep_info* info) {
  g_err.clear();
  if (!h || !b || !x) return fail(SSTEP_ERR_INVALID, "null handle, b or x");
  if (h->batch) return fail(SSTEP_ERR_INVALID, "a batched handle solves through sstep_solve_batched");
  return solve_impl(h, b, x, info);
}

sstep_status sstep_solve_batched(sstep_handle h, int nrhs, const double* const* b,
                                 double* const* x, sstep_info* infos) {
  g_err.clear();
  if (!h || nrhs < 0 || (nrhs > 0 && (!b || !x))) return fail(SSTEP_ERR_INVALID, "bad arguments");
  if (h->batch) return batch_solve(h->batch, nrhs, b, x, infos);
  sstep_status first = SSTEP_OK;
  for (int i = 0; i < nrhs; ++i) {
    sstep_status st = sstep_solve(h, b[i], x[i], infos ? infos + i : nullptr);
    if (st != SSTEP_OK && first == SSTEP_OK) first = st;
    if (st != SSTEP_OK && st != SSTEP_NOT_CONVERGED && st != SSTEP_ERR_BREAKDOWN &&
        st != SSTEP_ERR_NONFINITE)
      return st;
  }
  return first;
}

sstep_status sstep_amg_levels(sstep_handle h, int* nlevels) {
  g_err.clear();
  if (!h || !h->amg || !nlevels) return fail(SSTEP_ERR_INVALID, "not an AMG handle");
  *nlevels = amg_nlevels(h->amg);
  return SSTEP_OK;
}

sstep_status sstep_amg_level(sstep_handle h, int l, int64_t* n, int64_t* nnz, int64_t* rowptr,
                             int32_t* colind, double* vals, int32_t* agg) {
  g_err.clear();
  if (!h || !h->amg) return fail(SSTEP_ERR_INVALID, "not an AMG handle");
  sstep_status st = amg_level_copy(h->amg, l, n, nnz, rowptr, colind, vals, agg);
  if (st != SSTEP_OK) return fail(st, "level out of range");
  return SSTEP_OK;
}

sstep_status sstep_amg_apply(sstep_handle h, const double* b, double* x) {
  g_err.clear();
  if (!h || !h->amg || !b || !x || b == x) return fail(SSTEP_ERR_INVALID, "bad AMG apply arguments");
  CK(amg_apply(h->amg, b, x, h->st));
  CK(cudaStreamSynchronize(h->st));
  return SSTEP_OK;
}

sstep_status sstep_get_diagnostics(sstep_handle h, double* eta_a, double* eta_b, int maxlen,
                                   int* count, double* W, int maxw, int* countw) {
  g_err.clear();
  if (!h || h->batch) return fail(SSTEP_ERR_INVALID, "not a single-system handle");
  CK(cudaStreamSynchronize(h->st));
  const int iters = h->o.algo == SSTEP_ALGO_PCG ? 0 : h->hctrl->iters;
  const int na = std::max(0, std::min(maxlen, iters));
  const int nw = std::max(0, std::min({maxw, iters, kDiagW}));
  const int s = h->s, st = red_stride_for(s);
  const int nrec = std::max(na, nw);
  std::vector<double> rec((size_t)nrec * st);
  if (nrec > 0)
    CK(cudaMemcpy(rec.data(), h->red, sizeof(double) * rec.size(), cudaMemcpyDeviceToHost));
  // eta = ||B - W X||_F / ||B||_F of the kept systems (Section 3.3), in FP64 on the host
  auto eta = [s](const double* Wk, const double* B, const double* X, int nrhs) {
    double num = 0.0, den = 0.0;
    for (int c = 0; c < nrhs; ++c)
      for (int i = 0; i < s; ++i) {
        double v = B[i + c * s];
        for (int j = 0; j < s; ++j) v -= Wk[i + j * s] * X[j + c * s];
        num += v * v;
        den += B[i + c * s] * B[i + c * s];
      }
    return den > 0.0 ? std::sqrt(num / den) : 0.0;
  };
  for (int k = 0; k < na; ++k) {
    const double* r = rec.data() + (size_t)k * st;
    if (eta_a) eta_a[k] = eta(r, r + s * s, r + s * s + s, 1);
    if (eta_b && k + 1 < na) eta_b[k] = eta(r, r + s * s + 2 * s, r + 2 * s * s + 2 * s, s);
  }
  if (count) *count = na;
  if (W)
    for (int k = 0; k < nw; ++k)
      std::memcpy(W + (size_t)k * s * s, rec.data() + (size_t)k * st, sizeof(double) * s * s);
  if (countw) *countw = nw;
  return SSTEP_OK;
}

sstep_status sstep_get_batch_config(sstep_handle h, int* s, int* cluster, int* threads,
                                    int* slots, double* tune_ms) {
  g_err.clear();
  if (!h || !h->batch) return fail(SSTEP_ERR_INVALID, "not a batched handle");
  batch_config(h->batch, s, cluster, threads, slots, tune_ms);
  return SSTEP_OK;
}

sstep_status sstep_free(sstep_handle h) {
  destroy(h);
  return SSTEP_OK;
}

const char* sstep_status_string(sstep_status s) {
  switch (s) {
    case SSTEP_OK: return "ok";
    case SSTEP_NOT_CONVERGED: return "not converged (max_outer reached)";
    case SSTEP_ERR_INVALID: return "invalid argument";
    case SSTEP_ERR_BREAKDOWN: return "breakdown (Gram diagonal <= 0 or non-finite)";
    case SSTEP_ERR_NONFINITE: return "non-finite residual";
    case SSTEP_ERR_CUDA: return "CUDA error";
    case SSTEP_ERR_OOM: return "out of device memory";
    case SSTEP_ERR_UNSUPPORTED: return "unsupported";
    case SSTEP_ERR_TIMEOUT: return "a bounded device-side wait ran out";
  }
  return "unknown status";
}

const char* sstep_last_error(void) { return g_err.c_str(); }

sstep_status sstep_mpk(sstep_handle h, const double* r, double* Z, double* AZ, int s_override) {
  g_err.clear();
  if (!h || !r || !Z || !AZ) return fail(SSTEP_ERR_INVALID, "null argument");
  if (h->batch) return fail(SSTEP_ERR_INVALID, "not available on a batched handle");
  const int s = s_override ? s_override : h->s;
  if (s < 1 || s > kMaxS) return fail(SSTEP_ERR_INVALID, "s out of range");
  // Z and AZ given by the caller use leading dimension n.
  const int64_t keep = h->ld;
  h->ld = h->n;
  sstep_status st = run_mpk(h, r, Z, AZ, s, nullptr);
  h->ld = keep;
  return st;
}

sstep_status sstep_block_gram(int64_t n, int nl, const double* const* L, int nr,
                              const double* const* R, int ne, const int* pairs, double* out,
                              void* stream) {
  g_err.clear();
  if (n < 1 || nl < 1 || nr < 1 || nl > kMaxGramVecs || nr > kMaxGramVecs || ne < 1 ||
      ne > kMaxEntries || !L || !R || !pairs || !out)
    return fail(SSTEP_ERR_INVALID, "bad block_gram arguments");
  cudaStream_t st = (cudaStream_t)stream;
  GramArgs g{};
  g.n = n;
  g.nl = nl;
  g.nr = nr;
  g.ne = ne;
  for (int i = 0; i < nl; ++i) g.L[i] = L[i];
  for (int i = 0; i < nr; ++i) g.R[i] = R[i];
  for (int e = 0; e < ne; ++e) {
    if (pairs[2 * e] < 0 || pairs[2 * e] >= nl || pairs[2 * e + 1] < 0 || pairs[2 * e + 1] >= nr)
      return fail(SSTEP_ERR_INVALID, "pair index out of range");
    g.pairs[e] = (unsigned short)((pairs[2 * e] << 8) | pairs[2 * e + 1]);
  }
  g.mode = GM_SUMS;
  g.out = out;
  CK(gram_init());
  // Scratch for the partial sums and the ticket, stream-ordered.
  Ctrl* c = nullptr;
  double* part = nullptr;
  CK(cudaMallocAsync((void**)&c, sizeof(Ctrl), st));
  CK(cudaMallocAsync((void**)&part, sizeof(double) * (size_t)gram_ctas() * ne, st));
  CK(cudaMemsetAsync(c, 0, sizeof(Ctrl), st));
  g.ctrl = c;
  g.partials = part;
  cudaError_t e = launch_gram(g, st);
  cudaFreeAsync(part, st);
  cudaFreeAsync(c, st);
  CK(e);
  return SSTEP_OK;
}

sstep_status sstep_fgs(int s, const double* W, int nrhs, const double* B, int nu, int solver,
                       double* X, int* status_dev, void* stream) {
  g_err.clear();
  if (s < 1 || s > kMaxS || nrhs < 1 || nrhs > kMaxS || nu < 0 || !W || !B || !X ||
      (solver != SSTEP_GRAM_FGS && solver != SSTEP_GRAM_CHOLESKY &&
       solver != SSTEP_GRAM_FGS_OPERATOR))
    return fail(SSTEP_ERR_INVALID, "bad fgs arguments");
  if (solver == SSTEP_GRAM_FGS_OPERATOR && s > 8)
    return fail(SSTEP_ERR_UNSUPPORTED, "the FGS operator form takes s <= 8");
  CK(launch_fgs_standalone(s, W, nrhs, B, nu, solver, X, status_dev, (cudaStream_t)stream));
  return SSTEP_OK;
}

sstep_status sstep_block_update(sstep_handle h, const double* Z, const double* AZ, double* Q,
                                double* AQ, const double* alpha, const double* beta, double* x,
                                double* r, double* rr_out, int s_override) {
  g_err.clear();
  if (h && h->batch) return fail(SSTEP_ERR_INVALID, "not available on a batched handle");
  if (!h || !Z || !AZ || !Q || !AQ || !alpha || !x || !r || !rr_out)
    return fail(SSTEP_ERR_INVALID, "null argument");
  const int s = s_override ? s_override : h->s;
  if (s < 1 || s > kMaxS) return fail(SSTEP_ERR_INVALID, "s out of range");
  UpdArgs u{};
  u.n = h->n;
  u.ld = h->n;
  u.s = s;
  u.mode = beta ? UM_FUSED : UM_FIRST;
  u.Z = Z;
  u.AZ = AZ;
  u.Q = Q;
  u.AQ = AQ;
  u.x = x;
  u.r = r;
  u.alpha = alpha;
  u.beta = beta;
  u.ctrl = nullptr;
  u.rr_out = rr_out;
  u.partials = h->partials;
  u.ticket = &h->ctrl->ticket[TK_UPDATE];
  CK(launch_update(u, h->st));
  CK(cudaStreamSynchronize(h->st));
  return SSTEP_OK;
}

sstep_status sstep_spmv(sstep_handle h, const double* x, double* y) {
  g_err.clear();
  if (!h || !x || !y) return fail(SSTEP_ERR_INVALID, "null argument");
  if (h->batch) return fail(SSTEP_ERR_INVALID, "not available on a batched handle");
  EpiArgs e = epi_base(h, EP_SPMV);
  e.ctrl = nullptr;
  e.u = x;
  e.y = y;
  CK(launch_operator(h->op, e, h->st));
  CK(cudaStreamSynchronize(h->st));
  return SSTEP_OK;
}

sstep_status sstep_get_basis_info(sstep_handle h, double* lambda_min, double* lambda_max,
                                  double* c_alpha, double* c_sigma, double* c_gamma,
                                  int* power_iters_run) {
  if (!h) return fail(SSTEP_ERR_INVALID, "null handle");
  if (h->batch) return fail(SSTEP_ERR_INVALID, "not available on a batched handle");
  if (lambda_min) *lambda_min = h->lmin;
  if (lambda_max) *lambda_max = h->lmax;
  if (c_alpha) *c_alpha = h->c_alpha;
  if (c_sigma) *c_sigma = h->c_sigma;
  if (c_gamma) *c_gamma = h->c_gamma;
  if (power_iters_run) *power_iters_run = h->power_run;
  return SSTEP_OK;
}

sstep_status sstep_profile(sstep_handle h, const double* b, int iters, double* ms) {
  g_err.clear();
  if (!h || !b || !ms || iters < 1) return fail(SSTEP_ERR_INVALID, "bad profile arguments");
  if (h->batch) return fail(SSTEP_ERR_INVALID, "not available on a batched handle");
  const int algo = solve_algo(h);
  CK(cudaMemcpyAsync(h->b, b, sizeof(double) * h->n, cudaMemcpyDefault, h->st));
  CK(cudaMemsetAsync(h->x, 0, sizeof(double) * h->n, h->st));
  if (h->mixed) {
    CK(cudaMemsetAsync(h->xhi, 0, sizeof(float) * h->n, h->st));
    CK(cudaMemsetAsync(h->xlo, 0, sizeof(float) * h->n, h->st));
  }
  CKS(reset_ctrl(h));
  h->hctrl->rtol2 = 0.0;  // never converge while profiling
  h->hctrl->max_iters = 1 << 30;
  CK(cudaMemcpyAsync(h->ctrl, h->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, h->st));
  {
    EpiArgs e = epi_base(h, EP_RESID);
    e.u = h->x;
    e.y = h->mixed ? nullptr : h->r;
    e.b = h->b;
    e.rhi = h->mixed ? h->rhi : nullptr;
    e.rlo = h->mixed ? h->rlo : nullptr;
    CK(launch_operator(h->op, e, h->st));
  }
  if (algo == kAlgoMixed) {
    CKS(mixed_first(h));
  } else if (algo == kAlgoPcgF32) {
    const PcgF32Args a = pcgf_args(h);
    CK(launch_pcgf_rz(a, 1, h->st));
    CK(launch_pcgf_pdir(a, 1, h->st));
  } else if (algo == SSTEP_ALGO_ONESYNC) {
    CKS(run_mpk(h, h->r, h->Z, h->AZ, h->s, h->ctrl));
    CKS(run_gram(h, GM_ONESYNC_FIRST));
    CKS(run_update(h, UM_FIRST));
  } else if (algo == SSTEP_ALGO_LITERAL) {
    CKS(run_mpk(h, h->r, h->Z, h->AZ, h->s, h->ctrl));
    CKS(run_upd_w(h, true));
    CKS(run_update(h, UM_R));
  } else {
    PcgArgs a{h->n, h->x, h->r, h->p, h->Ap, h->M, h->ctrl, h->partials, nullptr};
    CK(launch_pcg_init(a, h->st));
  }
  constexpr int kPh = 4;
  cudaEvent_t ev[kPh + 1];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  double acc[kPh] = {0.0, 0.0, 0.0, 0.0};
  sstep_status st = SSTEP_OK;
  auto ok = [&](sstep_status v) { if (st == SSTEP_OK) st = v; };
  auto okc = [&](cudaError_t v) { if (st == SSTEP_OK && v != cudaSuccess) st = fail(SSTEP_ERR_CUDA, cudaGetErrorString(v)); };
  for (int k = 0; k < iters && st == SSTEP_OK; ++k) {
    cudaEventRecord(ev[0], h->st);
    if (algo == kAlgoMixed) {
      const MixedArgs a = mixed_args(h);
      ok(run_mpk_f32(h));
      cudaEventRecord(ev[1], h->st);
      okc(launch_gram_b2_f32(a, h->s, h->st));
      cudaEventRecord(ev[2], h->st);
      okc(launch_upd_gram_f32(a, h->s, false, h->st));
      cudaEventRecord(ev[3], h->st);
      okc(launch_update_xr_f32(a, h->s, h->st));
    } else if (algo == kAlgoPcgF32) {
      const PcgF32Args a = pcgf_args(h);
      ok(pcgf_product(h));
      cudaEventRecord(ev[1], h->st);
      okc(launch_pcgf_update(a, h->st));
      cudaEventRecord(ev[2], h->st);
      okc(launch_pcgf_pdir(a, 0, h->st));
      cudaEventRecord(ev[3], h->st);
    } else if (algo == SSTEP_ALGO_ONESYNC) {
      ok(run_mpk(h, h->r, h->Z, h->AZ, h->s, h->ctrl));
      cudaEventRecord(ev[1], h->st);
      ok(run_gram(h, GM_ONESYNC));
      cudaEventRecord(ev[2], h->st);
      ok(run_update(h, UM_FUSED));
      cudaEventRecord(ev[3], h->st);
    } else if (algo == SSTEP_ALGO_LITERAL) {
      ok(run_mpk(h, h->r, h->Z, h->AZ, h->s, h->ctrl));
      cudaEventRecord(ev[1], h->st);
      ok(run_gram(h, GM_LITERAL_B2));
      cudaEventRecord(ev[2], h->st);
      ok(run_upd_w(h, false));
      cudaEventRecord(ev[3], h->st);
      ok(run_update(h, UM_R));
    } else {
      EpiArgs e = epi_base(h, EP_PCG_AP);
      e.u = h->p;
      e.y = h->Ap;
      PcgArgs a{h->n, h->x, h->r, h->p, h->Ap, h->M, h->ctrl, h->partials, nullptr};
      okc(launch_operator(h->op, e, h->st));
      cudaEventRecord(ev[1], h->st);
      okc(launch_pcg_update(a, h->st));
      cudaEventRecord(ev[2], h->st);
      okc(launch_pcg_pdir(a, h->st));
      cudaEventRecord(ev[3], h->st);
    }
    cudaEventRecord(ev[4], h->st);
    cudaError_t e = cudaEventSynchronize(ev[4]);
    if (e != cudaSuccess) okc(e);
    for (int p = 0; p < kPh && st == SSTEP_OK; ++p) {
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[p], ev[p + 1]);
      acc[p] += t;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (st != SSTEP_OK) return st;
  CKS(read_ctrl(h));
  if (h->hctrl->done) return fail(SSTEP_ERR_BREAKDOWN, "profile: the iteration stopped early");
  double sum = 0.0;
  for (int p = 0; p < kPh; ++p) {
    ms[p] = acc[p] / iters;
    sum += ms[p];
  }
  ms[kPh] = sum;
  return SSTEP_OK;
}

sstep_status sstep_pattern_grad(int64_t n, const int64_t* rowptr, const int32_t* colind,
                                const double* lam, const double* x, double* grad_vals,
                                double scale, int accumulate, void* stream) {
  g_err.clear();
  if (n < 1 || !rowptr || !colind || !lam || !x || !grad_vals)
    return fail(SSTEP_ERR_INVALID, "bad pattern_grad arguments");
  CsrOp A{n, rowptr, colind, nullptr};
  CK(launch_pattern_grad(A, lam, x, grad_vals, scale, accumulate, (cudaStream_t)stream));
  return SSTEP_OK;
}

sstep_status sstep_q1_exp(int64_t ncell, const double* theta, double* kappa, void* stream) {
  g_err.clear();
  if (ncell < 1 || !theta || !kappa) return fail(SSTEP_ERR_INVALID, "bad q1_exp arguments");
  CK(launch_q1_exp(ncell, theta, kappa, (cudaStream_t)stream));
  return SSTEP_OK;
}

sstep_status sstep_q1_assemble(int nx, int ny, int nz, const double* kappa, const int64_t* rowptr,
                               const int32_t* colind, double* vals, void* stream) {
  g_err.clear();
  if (nx < 1 || ny < 1 || nz < 1 || !kappa || !rowptr || !colind || !vals)
    return fail(SSTEP_ERR_INVALID, "bad q1_assemble arguments");
  const cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = (int64_t)nx * ny * nz;
  int* bad = nullptr;
  CK(cudaMallocAsync((void**)&bad, sizeof(int), st));
  CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
  CK(launch_q1_assemble(nx, ny, nz, kappa, n, rowptr, colind, vals, bad, st));
  int hbad = 0;
  CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaFreeAsync(bad, st));
  CK(cudaStreamSynchronize(st));
  if (hbad) return fail(SSTEP_ERR_INVALID, "q1_assemble: a column is not a neighbour of its row");
  return SSTEP_OK;
}

sstep_status sstep_q1_grad(int nx, int ny, int nz, const double* kappa, const double* lam,
                           const double* x, double* grad, int wrt_log, int accumulate,
                           void* stream) {
  g_err.clear();
  if (nx < 1 || ny < 1 || nz < 1 || !lam || !x || !grad || (wrt_log && !kappa))
    return fail(SSTEP_ERR_INVALID, "bad q1_grad arguments");
  CK(launch_q1_grad(nx, ny, nz, kappa, lam, x, grad, wrt_log, accumulate, (cudaStream_t)stream));
  return SSTEP_OK;
}

sstep_status sstep_stencil7_weight_grad(int nsys, int nrhs, const int* dims, const double* const* lam,
                                        const double* const* x, double* grad, void* stream) {
  g_err.clear();
  if (nsys < 1 || nrhs < 1 || !dims || !lam || !x || !grad)
    return fail(SSTEP_ERR_INVALID, "bad stencil7_weight_grad arguments");
  const int np = nsys * nrhs;
  std::vector<Bil7Prob> tab(np);
  for (int i = 0; i < nsys; ++i) {
    const int nx = dims[3 * i], ny = dims[3 * i + 1], nz = dims[3 * i + 2];
    if (nx < 1 || ny < 1 || nz < 1) return fail(SSTEP_ERR_INVALID, "grid dimensions must be >= 1");
    for (int r = 0; r < nrhs; ++r) {
      const int p = i * nrhs + r;
      if (!lam[p] || !x[p]) return fail(SSTEP_ERR_INVALID, "null vector pointer");
      tab[p] = Bil7Prob{nx, ny, nz, lam[p], x[p]};
    }
  }
  const cudaStream_t st = (cudaStream_t)stream;
  Bil7Prob* dtab = nullptr;
  double* part = nullptr;
  CK(cudaMallocAsync((void**)&dtab, sizeof(Bil7Prob) * np, st));
  CK(cudaMallocAsync((void**)&part, sizeof(double) * 2 * np, st));
  CK(cudaMemcpyAsync(dtab, tab.data(), sizeof(Bil7Prob) * np, cudaMemcpyHostToDevice, st));
  CK(launch_stencil7_bilinear(dtab, np, part, st));
  CK(launch_sum_groups(part, nsys, nrhs, 2, -1.0, grad, st));
  CK(cudaFreeAsync(dtab, st));
  CK(cudaFreeAsync(part, st));
  // the host table must outlive the copy
  CK(cudaStreamSynchronize(st));
  return SSTEP_OK;
}

sstep_status sstep_update_values(sstep_handle h, const double* vals) {
  g_err.clear();
  if (!h || !vals) return fail(SSTEP_ERR_INVALID, "null argument");
  if (h->batch) return fail(SSTEP_ERR_INVALID, "not available on a batched handle");
  if (h->op.kind == SSTEP_MATRIX_Q1) {  // new conductivities
    CK(cudaMemcpyAsync(h->kappa, vals, sizeof(double) * h->ncell, cudaMemcpyDefault, h->st));
    CKS(q1_setup(h));
    if (h->kappaf) CK(launch_q1_kappaf(h->op.q1, h->kappaf, h->st));
    if (h->dinvf) CK(launch_d2f(h->dinv, h->dinvf, h->n, h->st));
    CK(cudaStreamSynchronize(h->st));
    return SSTEP_OK;
  }
  if (h->op.kind != SSTEP_MATRIX_CSR)
    return fail(SSTEP_ERR_INVALID, "the handle's operator is a constant stencil");
  const int64_t nnz = h->nnz;
  CK(cudaMemcpyAsync(h->vals, vals, sizeof(double) * nnz, cudaMemcpyDefault, h->st));
  if (h->dinv) {
    int* bad = nullptr;
    CK(cudaMallocAsync((void**)&bad, sizeof(int), h->st));
    CK(cudaMemsetAsync(bad, 0, sizeof(int), h->st));
    CK(launch_jacobi_csr(h->op.csr, h->dinv, bad, h->st));
    int hbad = 0;
    CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, h->st));
    CK(cudaFreeAsync(bad, h->st));
    CK(cudaStreamSynchronize(h->st));
    if (hbad) return fail(SSTEP_ERR_INVALID, "Jacobi needs a positive diagonal entry in every row");
  }
  if (h->amg) {  // the hierarchy depends on the values: rebuild it, re-capture the graphs
    CK(cudaStreamSynchronize(h->st));
    amg_free(h->amg);
    h->amg = nullptr;
    CKS(amg_build(h->rowptr, h->colind, h->vals, h->n, h->nnz, h->amg_coarse_max,
                  h->amg_max_levels, h->st, &h->amg));
    for (auto& g : h->gexec)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  }
  if (h->valsf) CK(launch_d2f(h->vals, h->valsf, nnz, h->st));
  if (h->dinvf) CK(launch_d2f(h->dinv, h->dinvf, h->n, h->st));
  CK(cudaStreamSynchronize(h->st));
  return SSTEP_OK;
}

sstep_status sstep_get_history(sstep_handle h, double* relres, int maxlen, int* count) {
  if (!h || !relres || maxlen < 1) return fail(SSTEP_ERR_INVALID, "bad arguments");
  if (h->batch) return fail(SSTEP_ERR_INVALID, "not available on a batched handle");
  CK(cudaStreamSynchronize(h->st));
  const int n = std::min(maxlen, h->hctrl->iters + 1);
  CK(cudaMemcpy(relres, h->hist, sizeof(double) * n, cudaMemcpyDeviceToHost));
  relres[0] = h->hctrl->nb2 > 0.0 ? std::sqrt(h->hctrl->rr0 / h->hctrl->nb2) : 0.0;
  if (count) *count = n;
  return SSTEP_OK;
}

}  // extern "C"
