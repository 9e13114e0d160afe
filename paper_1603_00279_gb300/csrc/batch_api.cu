// Host side of the batched C ABI (include/tsfcde.h, "batched instances"): per-instance tables
// and state, per-CTA work arrays sized for the largest instance, the work-queue order, and the
// launches of batch_setup_kernel / batch_level_kernel (level_kernels.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/tsfcde.h"
#include "tsfcde_internal.cuh"

using tsf::Args;

struct tsfcde_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = true;
  int64_t count = 0, M = 0, level = 0;
  tsfcde_options opt;
  std::vector<Args> inst;            // host copies (device pointers inside)
  std::vector<int64_t> n;
  std::vector<size_t> u0_off;
  char *arena = nullptr, *scratch = nullptr;
  Args *d_inst = nullptr;
  tsf::InstanceSetup *d_setup = nullptr;
  tsf::CtaScratch *d_cta = nullptr;
  int *d_order = nullptr;
  unsigned *d_next = nullptr;
  double *d_u0 = nullptr;            // all instances' u^0, concatenated (N_i doubles each)
  std::vector<double> u0_h;          // phi of every instance sampled on its mesh (host, setup only)
  double *d_uout = nullptr;          // staging for tsfcde_batch_get_all (same layout)
  // per-instance status words and per-level histories, contiguous over instances so that one
  // copy reads them all: status K x 4, iters / resid / outer / escalated K x M
  int *d_status = nullptr, *d_iters = nullptr, *d_outer = nullptr, *d_esc = nullptr;
  double *d_resid = nullptr;
  size_t u_total = 0;
  int grid = 0;
  size_t smem = 0;
  int grid_alloc = 0;                // CTAs given per-CTA scratch (the largest launch)
  int budget = 2048;                 // plan: chunk budget and split orientation (autotuner's)
  bool n1_large = false;
  double tune_best_ms = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return TSFCDE_OK;
  if (e == cudaErrorMemoryAllocation) return TSFCDE_E_NOMEM;
  return TSFCDE_E_CUDA;
}
#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

struct Carver {
  size_t off = 0;
  char *base = nullptr;
  template <typename T>
  T *take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// Plan of one instance: FFT sizes, the four-step split of the half-length transform (N1 <= N2,
// or N1 >= N2 when n1_large) and per-pass chunks of at most `budget` complex values.
void plan(Args &A, int64_t n, int budget = 2048, bool n1_large = false) {
  const int lgL = std::max(3, ilog2(2 * n));
  A.cp.lgL = lgL;
  A.cp.L = 1 << lgL;
  A.cp.lgN = lgL - 1;
  A.cp.N = 1 << A.cp.lgN;
  A.cp.lg1 = n1_large ? A.cp.lgN - A.cp.lgN / 2 : A.cp.lgN / 2;
  A.cp.lg2 = A.cp.lgN - A.cp.lg1;
  A.cp.N1 = 1 << A.cp.lg1;
  A.cp.N2 = 1 << A.cp.lg2;
  A.bp.lgNc = lgL;
  A.bp.Nc = 1 << lgL;
  A.bp.lg1 = lgL / 2;
  A.bp.lg2 = lgL - A.bp.lg1;
  A.bp.N1 = 1 << A.bp.lg1;
  A.bp.N2 = 1 << A.bp.lg2;
  // one-CTA team: every item of a pass belongs to the CTA, processed in chunks
  auto cap = [&](int items, int lines_per_item, int lg) {
    return std::max(1, std::min(items, std::max(1, (budget >> lg) / lines_per_item)));
  };
  A.cap_col = cap(A.cp.N2, 1, A.cp.lg1);
  A.cap_row = cap(A.cp.N1 / 2 + 1, 2, A.cp.lg2);
  A.cap_bcol = cap(A.bp.N2, 1, A.bp.lg1);
  A.cap_brow = cap(A.bp.N1, 1, A.bp.lg2);
}

}  // namespace

extern "C" {

void tsfcde_batch_free(tsfcde_batch *b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->arena) cudaFree(b->arena);
  if (b->scratch) cudaFree(b->scratch);
  if (b->d_inst) cudaFree(b->d_inst);
  if (b->d_setup) cudaFree(b->d_setup);
  if (b->d_cta) cudaFree(b->d_cta);
  if (b->d_order) cudaFree(b->d_order);
  if (b->d_next) cudaFree(b->d_next);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->stream && b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

static tsf::BatchArgs batch_args(const tsfcde_batch *b) {
  tsf::BatchArgs B;
  B.count = (int)b->count;
  B.inst = b->d_inst;
  B.setup = b->d_setup;
  B.cta = b->d_cta;
  B.order = b->d_order;
  B.next = b->d_next;
  return B;
}

// Worst per-instance status after a launch (the first non-OK one that is not NOT_CONVERGED, else
// NOT_CONVERGED if any, else OK); a CUDA error code when the copy fails.
static int batch_status(tsfcde_batch *b) {
  std::vector<int> h((size_t)b->count * 4);
  CK(cudaMemcpy(h.data(), b->d_status, h.size() * sizeof(int), cudaMemcpyDeviceToHost));
  int worst = TSFCDE_OK;
  for (int64_t i = 0; i < b->count; ++i) {
    const int hi = h[(size_t)i * 4];
    if (hi && hi != TSFCDE_E_NOT_CONVERGED) return hi;
    if (hi) worst = hi;
  }
  return worst;
}

// Per-instance tables and spectra on the device (they depend on the plan's split).
static int batch_device_setup(tsfcde_batch *b) {
  CK(cudaMemsetAsync(b->d_status, 0, (size_t)b->count * 4 * sizeof(int), b->stream));
  CK(cudaMemsetAsync(b->d_next, 0, 256, b->stream));
  const int st = tsf::launch_batch(batch_args(b), b->grid, b->smem, b->stream, 1, 0, 0);
  if (st) return st;
  CK(cudaStreamSynchronize(b->stream));
  return batch_status(b);
}

// Every instance's plan for a chunk budget and split orientation; the launch shape follows
// (CTAs per SM from the occupancy at that shared memory, never more than were given scratch).
static int batch_apply_plan(tsfcde_batch *b, const tsfcde_instance *in, const cudaDeviceProp &prop,
                            int budget, bool n1_large, bool *usable) {
  size_t smax = 0;
  for (int64_t i = 0; i < b->count; ++i) {
    plan(b->inst[i], in[i].N, budget, n1_large);
    smax = std::max(smax, tsf::level_smem_bytes(b->inst[i]));
  }
  int occ = 0, occ2 = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tsf::batch_level_kernel_ptr(), tsf::kThreads, smax));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, tsf::batch_setup_kernel_ptr(), tsf::kThreads, smax));
  *usable = occ >= 1 && occ2 >= 1;
  if (!*usable) return TSFCDE_OK;
  b->smem = smax;
  b->grid = std::min(b->grid_alloc, std::min(occ, occ2) * prop.multiProcessorCount);
  b->budget = budget;
  b->n1_large = n1_large;
  CK(cudaMemcpyAsync(b->d_inst, b->inst.data(), b->count * sizeof(Args), cudaMemcpyHostToDevice, b->stream));
  return TSFCDE_OK;
}

// Setup-time tuner of the batched launch: chunk budgets of 1024, 2048 and 4096 complex values
// (shared memory per CTA, hence CTAs per SM) times the two split orientations, each timed on
// the first two levels of every instance with its own spectra; the fastest is kept and the
// states go back to level 0.
static int batch_autotune(tsfcde_batch *b, const tsfcde_instance *in, const cudaDeviceProp &prop) {
  bool any_odd = false;
  for (int64_t i = 0; i < b->count; ++i) any_odd = any_odd || (b->inst[i].cp.lgN & 1);
  const int nlev = (int)std::min<int64_t>(b->M, 2);
  float best = 1e30f;
  int best_budget = b->budget;
  bool best_large = b->n1_large;
  for (int budget : {1024, 2048, 4096}) {
    for (bool large : {false, true}) {
      if (large && !any_odd) continue;   // the same split for every instance
      bool usable = false;
      int st = batch_apply_plan(b, in, prop, budget, large, &usable);
      if (st) return st;
      if (!usable) continue;
      st = batch_device_setup(b);
      if (st) return st;
      st = tsfcde_batch_reset(b);
      if (st) return st;
      CK(cudaMemsetAsync(b->d_status, 0, (size_t)b->count * 4 * sizeof(int), b->stream));
      CK(cudaMemsetAsync(b->d_next, 0, 256, b->stream));
      CK(cudaEventRecord(b->ev0, b->stream));
      st = tsf::launch_batch(batch_args(b), b->grid, b->smem, b->stream, 0, 0, nlev);
      if (st) return st;
      CK(cudaEventRecord(b->ev1, b->stream));
      CK(cudaStreamSynchronize(b->stream));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
      st = batch_status(b);
      if (st != TSFCDE_OK && st != TSFCDE_E_NOT_CONVERGED) return st;
      if (ms < best) {
        best = ms;
        best_budget = budget;
        best_large = large;
      }
    }
  }
  bool usable = false;
  int st = batch_apply_plan(b, in, prop, best_budget, best_large, &usable);
  if (st) return st;
  if (!usable) return TSFCDE_E_INVALID_ARG;
  b->tune_best_ms = best;
  return batch_device_setup(b);
}

static int batch_setup_impl(tsfcde_batch *b, const tsfcde_instance *in) {
  const int64_t K = b->count, M = b->M;
  const bool mixed = b->opt.precision == TSFCDE_MIXED;
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, b->device));
  b->grid = 2 * prop.multiProcessorCount;
  // ---- per-instance plans and the largest sizes ----
  b->inst.assign(K, Args());
  b->n.resize(K);
  int lgLmax = 3;
  int64_t nmax = 1;
  size_t smax = 0;
  for (int64_t i = 0; i < K; ++i) {
    Args &A = b->inst[i];
    std::memset(&A, 0, sizeof(A));
    A.n = (int)in[i].N;
    A.M = (int)M;
    plan(A, in[i].N);
    A.precond = b->opt.preconditioner;
    A.sigma = 1.0 - in[i].alpha / 2.0;
    const double tau = in[i].T / (double)M;
    A.hscale = std::pow(tau, -in[i].alpha) / std::tgamma(2.0 - in[i].alpha);
    A.tol = b->opt.tol;
    A.maxit = b->opt.maxit;
    A.precision = b->opt.precision;
    A.inner_tol = b->opt.inner_tol;
    A.inner_maxit = b->opt.inner_maxit;
    A.outer_maxit = b->opt.outer_maxit;
    A.spin_limit = 1ll << b->opt.barrier_spin_log2;
    A.gsf = (b->opt.algorithm == TSFCDE_ALG_IDS_CONST && M >= 2) ? 1 : 0;
    b->n[i] = in[i].N;
    lgLmax = std::max(lgLmax, A.cp.lgL);
    nmax = std::max(nmax, in[i].N);
    smax = std::max(smax, tsf::level_smem_bytes(A));
  }
  b->smem = smax;
  for (const void *fn : {tsf::batch_level_kernel_ptr(), tsf::batch_setup_kernel_ptr()}) {
    if (tsf::raise_smem_limit(fn, prop) < b->smem) return TSFCDE_E_INVALID_ARG;
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, tsf::kThreads, b->smem));
    if (occ < 1) return TSFCDE_E_INVALID_ARG;
    b->grid = std::min(b->grid, occ * prop.multiProcessorCount);
  }
  const size_t Lmax = size_t(1) << lgLmax, Nmax = Lmax / 2;

  // ---- per-instance arena ----
  std::vector<tsf::InstanceSetup> setup(K);
  Carver cv;
  size_t u0_total = 0;
  for (int pass = 0; pass < 2; ++pass) {
    cv.off = 0;
    cv.base = pass ? b->arena : nullptr;
    b->d_status = cv.take<int>((size_t)K * 4);
    b->d_iters = cv.take<int>((size_t)K * M);
    b->d_resid = cv.take<double>((size_t)K * M);
    b->d_outer = cv.take<int>((size_t)K * M);
    b->d_esc = cv.take<int>((size_t)K * M);
    for (int64_t i = 0; i < K; ++i) {
      Args &A = b->inst[i];
      const size_t L = A.cp.L, N = A.cp.N, n = A.n;
      A.u = cv.take<double>(L);
      A.ring_stride = (long long)((n + 31) / 32 * 32);
      A.ring = cv.take<double>((size_t)M * A.ring_stride);
      A.twL = cv.take<double2>(L);
      A.What = cv.take<double2>(N + 1);
      A.LamW = cv.take<double2>(n);
      A.LamQ = cv.take<double2>(n);
      A.chirpI = cv.take<double2>(n);
      A.BhI = cv.take<double2>(L);
      setup[i].BhF = cv.take<double2>(L);
      setup[i].omega = cv.take<double>(n + 2);
      setup[i].gtmp = cv.take<double>(n + 2);
      A.lv_eta = cv.take<double>(M);
      A.lv_q = cv.take<double>(M);
      A.lv_kp = cv.take<double>(M);
      A.lv_km = cv.take<double>(M);
      A.lv_newsym = cv.take<int>(M);
      A.hc = cv.take<double>(M + 2);
      A.hl = cv.take<double>(M + 2);
      A.iters = b->d_iters + (size_t)i * M;
      A.resid = b->d_resid + (size_t)i * M;
      A.outer_iters = b->d_outer + (size_t)i * M;
      A.escalated = b->d_esc + (size_t)i * M;
      A.status = b->d_status + (size_t)i * 4;
      A.lv_inner = cv.take<int>(M);
      A.lv_floor = cv.take<double>(M);
      if (A.gsf) {   // Gohberg-Semencul generators and factor spectra persist across launches
        A.gx = cv.take<double>(L);
        A.gy = cv.take<double>(L);
        A.SL = cv.take<double2>(N + 1);
        A.SR = cv.take<double2>(N + 1);
        A.SL0 = cv.take<double2>(N + 1);
        A.SR0 = cv.take<double2>(N + 1);
      }
      if (mixed) {
        A.twL32 = cv.take<float2>(L);
        A.twLff = cv.take<tsf::ffc>(L);
      }
    }
    b->u0_off.assign(K, 0);
    double *u0base = cv.take<double>(1);
    (void)u0base;
    u0_total = 0;
    for (int64_t i = 0; i < K; ++i) {
      b->u0_off[i] = u0_total;
      u0_total += (size_t)b->n[i];
    }
    b->d_u0 = cv.take<double>(u0_total);
    b->d_uout = cv.take<double>(u0_total);
    b->u_total = u0_total;
    if (!pass) {
      if (b->opt.test_inject == TSFCDE_INJECT_NOMEM) return TSFCDE_E_NOMEM;   // testing hook
      CK(cudaMalloc(&b->arena, cv.off + 256));
      CK(cudaMemsetAsync(b->arena, 0, cv.off + 256, b->stream));
    }
  }
  // ---- per-CTA scratch ----
  std::vector<tsf::CtaScratch> cta(b->grid);
  Carver cs;
  for (int pass = 0; pass < 2; ++pass) {
    cs.off = 0;
    cs.base = pass ? b->scratch : nullptr;
    for (int c = 0; c < b->grid; ++c) {
      tsf::CtaScratch &C = cta[c];
      C.x = cs.take<double>(Lmax);
      C.r = cs.take<double>(Lmax);
      C.rt = cs.take<double>(Lmax);
      C.p = cs.take<double>(Lmax);
      C.q = cs.take<double>(Lmax);
      C.uu = cs.take<double>(Lmax);
      C.vh = cs.take<double>(Lmax);
      C.H = cs.take<double>(Lmax);
      C.xb = cs.take<double>(Lmax);
      C.cprime = cs.take<double>(nmax);
      C.partials = cs.take<double>(8);
      C.bar = cs.take<unsigned>(tsf::kBarWords);
      C.SA = cs.take<double2>(Nmax + 1);
      C.SB = cs.take<double2>(Nmax + 1);
      C.SP = cs.take<double2>(Nmax + 1);
      C.Y1 = cs.take<double2>(Lmax);
      C.Y2 = cs.take<double2>(Lmax);
      if (b->opt.algorithm == TSFCDE_ALG_IDS_CONST) C.Y3 = cs.take<double2>(Nmax);
      if (mixed) {
        C.g = cs.take<double>(Lmax);
        C.x32 = cs.take<float>(Lmax);
        C.r32 = cs.take<float>(Lmax);
        C.rt32 = cs.take<float>(Lmax);
        C.p32 = cs.take<float>(Lmax);
        C.q32 = cs.take<float>(Lmax);
        C.uu32 = cs.take<float>(Lmax);
        C.vh32 = cs.take<float>(Lmax);
        C.SA32 = cs.take<float2>(Nmax + 1);
        C.SP32 = cs.take<float2>(Nmax + 1);
        C.Y1f = cs.take<float2>(Nmax);
        C.Y2f = cs.take<float2>(Nmax);
        C.x32b = cs.take<float>(Lmax);
        C.xffb = cs.take<tsf::ff>(Lmax);
        C.xff = cs.take<tsf::ff>(Lmax);
        C.rff = cs.take<tsf::ff>(Lmax);
        C.rtff = cs.take<tsf::ff>(Lmax);
        C.pff = cs.take<tsf::ff>(Lmax);
        C.qff = cs.take<tsf::ff>(Lmax);
        C.uuff = cs.take<tsf::ff>(Lmax);
        C.vhff = cs.take<tsf::ff>(Lmax);
        C.SAff = cs.take<tsf::ffc>(Nmax + 1);
        C.SPff = cs.take<tsf::ffc>(Nmax + 1);
        C.Y1ff = cs.take<tsf::ffc>(Nmax);
        C.Y2ff = cs.take<tsf::ffc>(Nmax);
      }
    }
    if (!pass) {
      CK(cudaMalloc(&b->scratch, cs.off + 256));
      CK(cudaMemsetAsync(b->scratch, 0, cs.off + 256, b->stream));
    }
  }
  // ---- setup inputs, order (largest first), uploads ----
  const std::vector<double> &u0all = b->u0_h;
  for (int64_t i = 0; i < K; ++i) {
    const tsfcde_instance &I = in[i];
    tsf::InstanceSetup &S = setup[i];
    S.alpha = I.alpha;
    S.beta = I.beta;
    S.tau = I.T / (double)M;
    S.h = (I.b - I.a) / (double)(I.N + 1);
    S.gamma = I.gamma;
    S.d_plus = I.d_plus;
    S.d_minus = I.d_minus;
  }
  std::vector<int> order(K);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->n[x] > b->n[y]; });
  CK(cudaMalloc(&b->d_inst, K * sizeof(Args)));
  CK(cudaMalloc(&b->d_setup, K * sizeof(tsf::InstanceSetup)));
  CK(cudaMalloc(&b->d_cta, b->grid * sizeof(tsf::CtaScratch)));
  CK(cudaMalloc(&b->d_order, K * sizeof(int)));
  CK(cudaMalloc(&b->d_next, 256));
  CK(cudaMemcpyAsync(b->d_inst, b->inst.data(), K * sizeof(Args), cudaMemcpyHostToDevice, b->stream));
  CK(cudaMemcpyAsync(b->d_setup, setup.data(), K * sizeof(tsf::InstanceSetup), cudaMemcpyHostToDevice, b->stream));
  CK(cudaMemcpyAsync(b->d_cta, cta.data(), b->grid * sizeof(tsf::CtaScratch), cudaMemcpyHostToDevice, b->stream));
  CK(cudaMemcpyAsync(b->d_order, order.data(), K * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  CK(cudaMemcpyAsync(b->d_u0, u0all.data(), u0_total * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  // precision controller per instance and level (constant coefficients: j = 0 and j >= 1)
  std::vector<int> inner_all((size_t)K * M);
  std::vector<double> floor_all((size_t)K * M);
  for (int64_t i = 0; i < K; ++i) {
    const tsfcde_instance &I = in[i];
    const double sigma = 1.0 - I.alpha / 2.0, tau = I.T / (double)M, h = (I.b - I.a) / (double)(I.N + 1);
    const double a0 = std::pow(sigma, 1.0 - I.alpha);
    const double b1 = (std::pow(1.0 + sigma, 2.0 - I.alpha) - std::pow(sigma, 2.0 - I.alpha)) / (2.0 - I.alpha) -
                      0.5 * (std::pow(1.0 + sigma, 1.0 - I.alpha) + std::pow(sigma, 1.0 - I.alpha));
    const double den = std::pow(tau, I.alpha) * std::tgamma(2.0 - I.alpha), hb = std::pow(h, I.beta);
    for (int64_t j = 0; j < M; ++j) {
      const double eta = (j == 0 ? a0 : a0 + b1) / den;
      tsf::precision_control(sigma, I.beta, eta, I.gamma / (2.0 * h), I.d_plus / hb, I.d_minus / hb,
                             b->opt.inner_precision, b->opt.tol, &inner_all[(size_t)i * M + j],
                             &floor_all[(size_t)i * M + j]);
    }
    CK(cudaMemcpyAsync((void *)b->inst[i].lv_inner, inner_all.data() + (size_t)i * M, M * sizeof(int),
                       cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync((void *)b->inst[i].lv_floor, floor_all.data() + (size_t)i * M, M * sizeof(double),
                       cudaMemcpyHostToDevice, b->stream));
  }
  CK(cudaStreamSynchronize(b->stream));
  // ---- device setup: weights, tables, spectra of every instance; then the plan tuner ----
  b->grid_alloc = b->grid;
  int st = batch_device_setup(b);
  if (st) return st;
  if (b->opt.autotune) {
    st = batch_autotune(b, in, prop);
    if (st) return st;
  }
  return tsfcde_batch_reset(b);
}

int tsfcde_batch_setup(tsfcde_batch **out, int64_t count, const tsfcde_instance *inst, int64_t M,
                       const tsfcde_options *opt) {
  if (!out) return TSFCDE_E_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || !inst || M < 1 || M > (int64_t(1) << 30)) return TSFCDE_E_INVALID_ARG;
  tsfcde_options o;
  tsfcde_default_options(&o);
  if (opt) o = *opt;
  if (o.preconditioner < 0 || o.preconditioner > 2 ||
      (o.precision != TSFCDE_FP64 && o.precision != TSFCDE_MIXED) || !(o.tol > 0) || o.maxit < 1 ||
      (o.algorithm != TSFCDE_ALG_IDS && o.algorithm != TSFCDE_ALG_IDS_CONST))
    return TSFCDE_E_INVALID_ARG;
  if (o.test_inject != TSFCDE_INJECT_NONE && o.test_inject != TSFCDE_INJECT_NOMEM) return TSFCDE_E_INVALID_ARG;
  if (o.fast_history != 0) return TSFCDE_E_INVALID_ARG;   // single contexts only
  size_t total = 0;
  for (int64_t i = 0; i < count; ++i) {
    const tsfcde_instance &I = inst[i];
    if (!(I.a < I.b) || !(I.T > 0) || I.N < 1 || I.N > 16383 || !(I.alpha > 0 && I.alpha <= 1) ||
        !(I.beta > 1 && I.beta <= 2) || !(I.d_plus >= 0) || !(I.d_minus >= 0) || !I.phi ||
        !std::isfinite(I.gamma))
      return TSFCDE_E_INVALID_ARG;
    total += (size_t)I.N;
  }
  // u^0_i = phi(x_i) on each instance's mesh x_i = a + i h (Section 2.1), before any device work
  std::vector<double> u0h(total), xg;
  size_t off = 0;
  for (int64_t i = 0; i < count; ++i) {
    const tsfcde_instance &I = inst[i];
    const double h = (I.b - I.a) / (double)(I.N + 1);
    xg.resize(I.N);
    for (int64_t k = 0; k < I.N; ++k) xg[k] = I.a + (double)(k + 1) * h;
    I.phi(0.0, xg.data(), u0h.data() + off, I.N, I.user);
    for (int64_t k = 0; k < I.N; ++k)
      if (!std::isfinite(u0h[off + k])) return TSFCDE_E_NONFINITE;
    off += (size_t)I.N;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= o.device || o.device < 0) return TSFCDE_E_NO_DEVICE;
  tsfcde_batch *b = new tsfcde_batch();
  b->u0_h.swap(u0h);
  b->device = o.device;
  b->opt = o;
  b->count = count;
  b->M = M;
  if (cudaSetDevice(b->device) != cudaSuccess) {
    delete b;
    return TSFCDE_E_CUDA;
  }
  if (o.stream) {
    b->stream = (cudaStream_t)o.stream;
    b->own_stream = false;
  } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return TSFCDE_E_CUDA;
  }
  if (cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess) {
    tsfcde_batch_free(b);
    return TSFCDE_E_CUDA;
  }
  const int st = batch_setup_impl(b, inst);
  cudaStreamSynchronize(b->stream);   // the host samples are on the device (or no longer needed)
  std::vector<double>().swap(b->u0_h);
  if (st != TSFCDE_OK) {
    tsfcde_batch_free(b);
    return st;
  }
  *out = b;
  return TSFCDE_OK;
}

int tsfcde_batch_reset(tsfcde_batch *b) {
  if (!b) return TSFCDE_E_INVALID_ARG;
  CK(cudaSetDevice(b->device));
  for (int64_t i = 0; i < b->count; ++i)
    CK(cudaMemcpyAsync(b->inst[i].u, b->d_u0 + b->u0_off[i], b->n[i] * sizeof(double),
                       cudaMemcpyDeviceToDevice, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  b->level = 0;
  return TSFCDE_OK;
}

int tsfcde_batch_set_initial(tsfcde_batch *b, const double *u0_all) {
  if (!b || !u0_all) return TSFCDE_E_INVALID_ARG;
  CK(cudaSetDevice(b->device));
  CK(cudaMemcpyAsync(b->d_u0, u0_all, b->u_total * sizeof(double), cudaMemcpyHostToDevice, b->stream));
  return tsfcde_batch_reset(b);
}

int tsfcde_batch_solve(tsfcde_batch *b, double *u_all, tsfcde_stats *stats) {
  if (!b) return TSFCDE_E_INVALID_ARG;
  const int st = tsfcde_batch_step(b, b->M - b->level, stats);
  if (st != TSFCDE_OK && st != TSFCDE_E_NOT_CONVERGED) return st;
  if (u_all) {
    const int st2 = tsfcde_batch_get_all(b, u_all);
    if (st2) return st2;
  }
  return st;
}

int tsfcde_batch_get_plan(tsfcde_batch *b, int32_t *budget, int32_t *n1_ge_n2, int32_t *ctas,
                          double *best_ms) {
  if (!b) return TSFCDE_E_INVALID_ARG;
  if (budget) *budget = b->budget;
  if (n1_ge_n2) *n1_ge_n2 = b->n1_large ? 1 : 0;
  if (ctas) *ctas = b->grid;
  if (best_ms) *best_ms = b->tune_best_ms;
  return TSFCDE_OK;
}

int tsfcde_batch_get_all(tsfcde_batch *b, double *u_all) {
  if (!b || !u_all) return TSFCDE_E_INVALID_ARG;
  CK(cudaSetDevice(b->device));
  for (int64_t i = 0; i < b->count; ++i)
    CK(cudaMemcpyAsync(b->d_uout + b->u0_off[i], b->inst[i].u, b->n[i] * sizeof(double),
                       cudaMemcpyDeviceToDevice, b->stream));
  CK(cudaMemcpyAsync(u_all, b->d_uout, b->u_total * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  CK(cudaStreamSynchronize(b->stream));
  return TSFCDE_OK;
}

int tsfcde_batch_step(tsfcde_batch *b, int64_t nsteps, tsfcde_stats *stats) {
  if (!b || nsteps < 0) return TSFCDE_E_INVALID_ARG;
  if (b->level + nsteps > b->M) return TSFCDE_E_STATE;
  CK(cudaSetDevice(b->device));
  const int64_t j0 = b->level, j1 = b->level + nsteps;
  float ms = 0.f;
  int launches = 0;
  if (nsteps > 0) {
    CK(cudaMemsetAsync(b->d_status, 0, (size_t)b->count * 4 * sizeof(int), b->stream));
    CK(cudaMemsetAsync(b->d_next, 0, 256, b->stream));
    tsf::BatchArgs B;
    B.count = (int)b->count;
    B.inst = b->d_inst;
    B.setup = b->d_setup;
    B.cta = b->d_cta;
    B.order = b->d_order;
    B.next = b->d_next;
    CK(cudaEventRecord(b->ev0, b->stream));
    const int st = tsf::launch_batch(B, b->grid, b->smem, b->stream, 0, (int)j0, (int)j1);
    if (st) return st;
    CK(cudaEventRecord(b->ev1, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    CK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
    launches = 1;
  }
  int worst = TSFCDE_OK;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->min_iterations = 1 << 30;
  }
  if (nsteps > 0) {
    const int64_t K = b->count, M = b->M;
    std::vector<int> h((size_t)K * 4);
    CK(cudaMemcpy(h.data(), b->d_status, h.size() * sizeof(int), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < K; ++i) {
      const int hi = h[(size_t)i * 4];
      if (hi && hi != TSFCDE_E_NOT_CONVERGED) return hi;
      if (hi) worst = hi;
    }
    if (stats) {
      // the [j0, j1) window of every instance's per-level history, one strided copy each
      const bool mixed = b->opt.precision == TSFCDE_MIXED;
      const bool gsf = b->opt.algorithm == TSFCDE_ALG_IDS_CONST && M >= 2;
      std::vector<int> it((size_t)K * nsteps), oi, es;
      std::vector<double> rs((size_t)K * nsteps);
      CK(cudaMemcpy2D(it.data(), nsteps * sizeof(int), b->d_iters + j0, M * sizeof(int),
                      nsteps * sizeof(int), K, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy2D(rs.data(), nsteps * sizeof(double), b->d_resid + j0, M * sizeof(double),
                      nsteps * sizeof(double), K, cudaMemcpyDeviceToHost));
      if (mixed || gsf) {
        oi.resize((size_t)K * nsteps);
        es.resize((size_t)K * nsteps);
        CK(cudaMemcpy2D(oi.data(), nsteps * sizeof(int), b->d_outer + j0, M * sizeof(int),
                        nsteps * sizeof(int), K, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy2D(es.data(), nsteps * sizeof(int), b->d_esc + j0, M * sizeof(int),
                        nsteps * sizeof(int), K, cudaMemcpyDeviceToHost));
      }
      for (int64_t i = 0; i < K; ++i) {
        for (int64_t k = 0; k < nsteps; ++k) {
          const size_t x = (size_t)i * nsteps + k;
          stats->total_iterations += it[x];
          stats->max_iterations = std::max(stats->max_iterations, it[x]);
          stats->min_iterations = std::min(stats->min_iterations, it[x]);
          stats->max_residual = std::max(stats->max_residual, rs[x]);
          if (mixed || gsf) {
            stats->outer_iterations += oi[x];
            stats->escalated_levels += es[x] & 1;
            stats->floor_levels += (es[x] >> 1) & 1;
          }
          if (gsf && j0 + k >= 1) ++stats->gsf_levels;
        }
      }
    }
  }
  b->level = j1;
  if (stats) {
    stats->level = b->level;
    stats->levels_advanced = nsteps;
    stats->status = worst;
    stats->device_launches = launches;
    stats->device_ms = ms;
    if (stats->min_iterations == (1 << 30)) stats->min_iterations = 0;
  }
  return worst;
}

int tsfcde_batch_get_level(tsfcde_batch *b, int64_t i, int64_t j, double *u_out) {
  if (!b || !u_out || i < 0 || i >= b->count || j < 0 || j > b->level) return TSFCDE_E_INVALID_ARG;
  CK(cudaSetDevice(b->device));
  const Args &A = b->inst[i];
  if (j == b->level) {
    CK(cudaMemcpyAsync(u_out, A.u, b->n[i] * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  } else {
    // the get_all staging area of this instance holds the rebuilt level
    double *tmp = b->d_uout + b->u0_off[i];
    const int st = tsf::launch_level_rebuild(b->d_u0 + b->u0_off[i], A.u, A.ring, A.ring_stride, A.n, (int)j,
                                             (int)b->level, tmp, b->stream);
    if (st) return st;
    CK(cudaMemcpyAsync(u_out, tmp, b->n[i] * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  }
  CK(cudaStreamSynchronize(b->stream));
  return TSFCDE_OK;
}

int tsfcde_batch_level(tsfcde_batch *b, int64_t *level) {
  if (!b || !level) return TSFCDE_E_INVALID_ARG;
  *level = b->level;
  return TSFCDE_OK;
}

int tsfcde_batch_get_history(tsfcde_batch *b, int64_t i, int32_t *iters, double *resid, int64_t count) {
  if (!b || i < 0 || i >= b->count || count < 0 || count > b->level) return TSFCDE_E_INVALID_ARG;
  CK(cudaSetDevice(b->device));
  if (count == 0) return TSFCDE_OK;
  if (iters) CK(cudaMemcpy(iters, b->inst[i].iters, count * sizeof(int), cudaMemcpyDeviceToHost));
  if (resid) CK(cudaMemcpy(resid, b->inst[i].resid, count * sizeof(double), cudaMemcpyDeviceToHost));
  return TSFCDE_OK;
}

}  // extern "C"
