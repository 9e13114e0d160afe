// Device side of the level solve (Algorithm "Practical implementation of IDS", arXiv:1603.00279
// Section 3.2) as persistent cooperative kernels.  One launch advances a range of levels; every
// phase below is separated from the next by a bounded grid barrier, so each level costs a fixed
// sequence of phases and no host round trip:
//
//   symbols  (when the level operators change):  Lambda_P -> 1/Lambda_P -> inverse n-point DFT
//            by Bluestein (3 phases) -> Toeplitz embedding of P^{-1}'s circulant column ->
//            forward FFT and the spectra of A, B, P^{-1} (2 phases)               [Eq. (3.7)]
//   RHS      commit of the previous level + history sum of Lemma 1 + column FFT of u^j; row
//            pass with B's spectrum; column pass giving g = B u^j - hscale*H + f  [Eq. (3.1)]
//   solve    FP64: preconditioned CGS from x0 = 0 (Section 4), the elementwise updates and dot
//            products fused into the column passes of the FFT convolutions; each iteration is
//            10 phases (P^{-1} p, A p^, dot, q/w update, P^{-1} w, A u^, dots).
//            Mixed: iterative refinement whose residual r = g - A x, solution update and history
//            stay in FP64, with the same CGS run in FP32 (FP32 FFTs, spectra rounded from FP64)
//            on A d = r; a level whose FP64 residual stops falling is finished by the FP64 CGS.
#include "level_device.cuh"

#include <algorithm>
#include <cstring>

namespace tsf {
// ------------------------------------------------------------------------------------------------
// diagnostic: the history sum of level j alone (the march's phase, no commit)
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1) history_kernel(Args Ap, int j) {
  __shared__ Args A;
  if (threadIdx.x == 0) A = Ap;
  __syncthreads();
  const Smem S = smem_view(lp_max_of(A), tw_max_of(A));
  grid_sync_init();
  if (A.fh_B && j >= A.fh_B) {   // fast history: the far part of j's block from the stored spectra
    ph_far_update(A, S, j >> A.fh_lgB, false);
    if (!grid_sync(A)) return;
  }
  ph_history(A, j, false);
}

// ------------------------------------------------------------------------------------------------
// Spectra of the fast-history kernel windows: window m = 1..nblk holds w_m[t] = hc[(m-1)B + t] for
// t < 2B, with hc[0] taken as 0 and lags l >= M as 0 (no level uses them), and
// K[(m-1)(B+1) + k] = DFT_2B(w_m)[k] / (2B) for k = 0..B, each by a direct sum of 2B terms.
// ------------------------------------------------------------------------------------------------
__global__ void fh_kernel_spectra_kernel(const double *hc, int M, int B, int nblk, double2 *K) {
  const int T2 = 2 * B;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nblk * (B + 1); idx += gridDim.x * blockDim.x) {
    const int m = idx / (B + 1) + 1, k = idx % (B + 1);
    double re = 0.0, im = 0.0;
    for (int t = 0; t < T2; ++t) {
      const long long l = (long long)(m - 1) * B + t;
      const double w = (l >= 1 && l < M) ? hc[l] : 0.0;
      double sn, cs;
      sincospi(-2.0 * (double)((k * t) % T2) / (double)T2, &sn, &cs);
      re += w * cs;
      im += w * sn;
    }
    K[idx] = make_double2(re / (double)T2, im / (double)T2);
  }
}

// ------------------------------------------------------------------------------------------------
// FP64 fused multiply-add throughput of the device (the denominator of the level kernels' ALU
// roofline): 16 independent FMA chains per thread, enough warps per SM to keep every SM
// sub-partition's FP64 unit busy; each FMA counts 2 flops.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) fp64_fma_kernel(double *out, int iters, double b, double c) {
  double v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = 1e-3 * (double)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __fma_rn(v[k], b, c);
  }
  double sacc = 0.0;
#pragma unroll
  for (int k = 0; k < 16; ++k) sacc += v[k];
  if (sacc == 12345.678) out[0] = sacc;   // keeps the chains live; never true for these inputs
}

int launch_fp64_fma(double *out, int blocks, int iters, cudaStream_t st) {
  fp64_fma_kernel<<<blocks, 256, 0, st>>>(out, iters, 0.999999, 1e-7);
  return cudaGetLastError() == cudaSuccess ? kOK : kECuda;
}

int launch_fh_kernel_spectra(const double *hc, int M, int B, int nblk, double2 *K, cudaStream_t st) {
  const int total = nblk * (B + 1);
  fh_kernel_spectra_kernel<<<(total + kThreads - 1) / kThreads, kThreads, 0, st>>>(hc, M, B, nblk, K);
  return cudaGetLastError() == cudaSuccess ? kOK : kECuda;
}

// ------------------------------------------------------------------------------------------------
// level u^j of a march from its u^0, current level u^c and ring of increments d^s = u^{s+1} - u^s
// (s < c): the shorter of u^0 + sum_{s<j} d^s and u^c - sum_{j<=s<c} d^s, summed in order of s
// (coalesced over i; one ring row per term)
// ------------------------------------------------------------------------------------------------
__global__ void level_rebuild_kernel(const double *u0, const double *uc, const double *ring,
                                     long long stride, int n, int j, int c, double *out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double v;
    if (j <= c - j) {
      v = u0[i];
      for (int s = 0; s < j; ++s) v += ring[(long long)s * stride + i];
    } else {
      v = uc[i];
      for (int s = c - 1; s >= j; --s) v -= ring[(long long)s * stride + i];
    }
    out[i] = v;
  }
}

int launch_level_rebuild(const double *u0, const double *uc, const double *ring, long long stride, int n,
                         int j, int c, double *out, cudaStream_t st) {
  const int blocks = std::min((n + kThreads - 1) / kThreads, 4 * kMaxGrid);
  level_rebuild_kernel<<<blocks, kThreads, 0, st>>>(u0, uc, ring, stride, n, j, c, out);
  return cudaGetLastError() == cudaSuccess ? kOK : kECuda;
}

// ------------------------------------------------------------------------------------------------
// diagnostic products y = op_j x (op 0: A, 1: B, 2: P^{-1}, 3: A^{-1} by the Gohberg-Semencul
// formula); x and y are padded device vectors.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1) apply_kernel(Args Ap, int op, int j, const double *xin, double *yout) {
  __shared__ Args A;
  if (threadIdx.x == 0) A = Ap;
  __syncthreads();
  const Smem S = smem_view(lp_max_of(A), tw_max_of(A));
  grid_sync_init();
  const int n = A.n;
  if (op == 3) {   // y = A^{-1} x by the Gohberg-Semencul formula (generators already built)
    col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y1,
                                   [&](int m, double2) -> double2 { return ld2(xin, m); });
    if (!grid_sync(A)) return;
    gsf_apply<false>(A, S, [&](int m, double2 z) -> double2 {
      st2(yout, m, z);
      return z;
    });
    return;
  }
  if (!level_symbols(A, S, j)) return;
  col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y1,
                                 [&](int m, double2) -> double2 { return ld2(xin, m); });
  if (!grid_sync(A)) return;
  row_pass<0, double2>(A, S, A.twL, A.Y1, A.Y2, op == 0 ? A.SA : (op == 1 ? A.SB : A.SP), nullptr, 0.0, -1);
  if (!grid_sync(A)) return;
  col_pass<true, false, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, A.Y2, nullptr,
                                 [&](int m, double2 z) -> double2 {
                                   if (2 * m >= n) z.x = 0.0;
                                   if (2 * m + 1 >= n) z.y = 0.0;
                                   st2(yout, m, z);
                                   return z;
                                 });
}

__global__ void __launch_bounds__(kThreads, 1) setup_kernel(Args Ap, SetupArgs T) {
  __shared__ Args A;
  if (threadIdx.x == 0) A = Ap;
  __syncthreads();
  const Smem S = smem_view(lp_max_of(A), tw_max_of(A));
  grid_sync_init();
  setup_body(A, T, S);
}

// ------------------------------------------------------------------------------------------------
// weights and per-level tables (Lemma 1, Lemma 2)
// ------------------------------------------------------------------------------------------------
// omega_k for k = 0..n+1: the Grunwald recurrence g_k = (1 - (beta+1)/k) g_{k-1} (Lemma 3) with
// explicit rounding (no contraction): factors in parallel, the running product by one thread;
// then the WSGD combination (Lemma 2).
__global__ void grunwald_factors_kernel(double *f, int K, double beta) {
  for (int k = 1 + blockIdx.x * blockDim.x + threadIdx.x; k <= K; k += gridDim.x * blockDim.x)
    f[k] = __dadd_rn(1.0, -__ddiv_rn(beta + 1.0, (double)k));
}

__global__ void grunwald_kernel(double *g, const double *f, int K) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double gk = 1.0;
    g[0] = gk;
    for (int k = 1; k <= K; ++k) {
      gk = __dmul_rn(f[k], gk);
      g[k] = gk;
    }
  }
}

__global__ void wsgd_kernel(const double *g, double *omega, int K, double beta) {
  double lam1, lam0, lamm1;
  wsgd_lambdas(beta, lam1, lam0, lamm1);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= K; k += gridDim.x * blockDim.x) {
    double w = __dmul_rn(lam1, g[k]);
    if (k >= 1) w = __dadd_rn(w, __dmul_rn(lam0, g[k - 1]));
    if (k >= 2) w = __dadd_rn(w, __dmul_rn(lamm1, g[k - 2]));
    omega[k] = w;
  }
}

__global__ void time_tables_kernel(int M, double alpha, double tau, double h, double beta,
                                   const double *gam, const double *dp, const double *dm,
                                   double *hc, double *hl, double *eta, double *q, double *kp,
                                   double *km) {
  const double sigma = 1.0 - alpha / 2.0;
  const double denom = pow(tau, alpha) * tgamma(2.0 - alpha);
  const double hb = pow(h, beta);
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l <= M; l += gridDim.x * blockDim.x) {
    const double al = l21_a(alpha, sigma, l), bl = l21_b(alpha, sigma, l);
    hl[l] = al - bl;
    hc[l] = l >= 1 ? al + l21_b(alpha, sigma, l + 1) - bl : 0.0;
    if (l < M) {
      const double c0 = l == 0 ? l21_a(alpha, sigma, 0) : l21_a(alpha, sigma, 0) + l21_b(alpha, sigma, 1);
      eta[l] = c0 / denom;
      q[l] = gam[l] / (2.0 * h);
      kp[l] = dp[l] / hb;
      km[l] = dm[l] / hb;
    }
  }
}

// ------------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------------
static int coop_launch(const void *fn, int grid, size_t smem, cudaStream_t st, void **args) {
  return coop_launch_n(fn, grid, kThreads, smem, st, args);
}

size_t level_smem_bytes(const Args &A) { return smem_lines_bytes(A); }

const void *level_kernel_ptr() { return (const void *)level_kernel<kThreads>; }
const void *history_kernel_ptr() { return (const void *)history_kernel; }

int launch_history(const Args &A, int grid, size_t smem, cudaStream_t st, int j) {
  Args a = A;
  void *args[] = {&a, &j};
  return coop_launch((const void *)history_kernel, grid, smem, st, args);
}
const void *apply_kernel_ptr() { return (const void *)apply_kernel; }
const void *setup_kernel_ptr() { return (const void *)setup_kernel; }

int launch_levels(const Args &A, int grid, size_t smem, cudaStream_t st, int j0, int j1, int threads) {
  if (grid == 1) return launch_levels_cta(A, smem, st, j0, j1);   // one-CTA team (level_wide.cu)
  if (threads == kWideThreads) return launch_levels_wide(A, grid, smem, st, j0, j1);
  Args a = A;
  void *args[] = {&a, &j0, &j1};
  return coop_launch_n((const void *)level_kernel<kThreads>, grid, kThreads, smem, st, args);
}

int launch_apply(const Args &A, int grid, size_t smem, cudaStream_t st, int op, int j,
                 const double *xin, double *yout) {
  Args a = A;
  void *args[] = {&a, &op, &j, &xin, &yout};
  return coop_launch((const void *)apply_kernel, grid, smem, st, args);
}

int launch_setup(const Args &A, int grid, size_t smem, cudaStream_t st, const double *omega,
                 double2 *What, double2 *LamW, double2 *LamQ, double2 *BhI, double2 *BhF,
                 double2 *chirpI, double2 *twL, double beta, int precond) {
  (void)beta;
  SetupArgs T;
  T.omega = omega;
  T.What = What;
  T.LamW = LamW;
  T.LamQ = LamQ;
  T.BhI = BhI;
  T.BhF = BhF;
  T.chirpI = chirpI;
  T.twL = twL;
  T.precond = precond;
  Args a = A;
  void *args[] = {&a, &T};
  return coop_launch((const void *)setup_kernel, grid, smem, st, args);
}

int launch_weights(double *omega, double *g_tmp, int n, double beta, cudaStream_t st) {
  // factors in omega's storage first, then the sequential product into g_tmp, then omega
  grunwald_factors_kernel<<<(n + 1 + kThreads - 1) / kThreads, kThreads, 0, st>>>(omega, n + 1, beta);
  grunwald_kernel<<<1, 32, 0, st>>>(g_tmp, omega, n + 1);
  wsgd_kernel<<<(n + 2 + kThreads - 1) / kThreads, kThreads, 0, st>>>(g_tmp, omega, n + 1, beta);
  return cudaGetLastError() == cudaSuccess ? kOK : kECuda;
}

int launch_time_tables(int M, double alpha, double tau, double h, double beta, const double *gam,
                       const double *dp, const double *dm, double *hc, double *hl, double *eta,
                       double *q, double *kp, double *km, cudaStream_t st) {
  time_tables_kernel<<<(M + 1 + kThreads - 1) / kThreads, kThreads, 0, st>>>(
      M, alpha, tau, h, beta, gam, dp, dm, hc, hl, eta, q, kp, km);
  return cudaGetLastError() == cudaSuccess ? kOK : kECuda;
}

// ================================================================================================
// Operator product without any device allocation.
//
// Some callers cannot call cudaMalloc: code running inside another runtime's memory pool or
// allocator hooks, processes whose device memory is fully reserved up front, or callers that
// must not make an allocating call on a latency-critical path.  tsfcde_apply_operator_static()
// serves them: it computes y = A x or y = B x for one level (the operators of Eq. (3.3)) from
// the level's scalars alone, with every intermediate (WSGD weights, twiddles, the spectrum of
// W's circulant embedding, the operator spectrum, FFT work arrays, barrier words) kept in the
// file-scope device array below.  The caller passes x and y in device memory.
//
// The array is a fixed 3 MiB per device, allocated by the CUDA runtime when the library is
// loaded and held until the process exits; it bounds N (interior points) to 16383.  Every call
// reuses it and the array keeps the previous call's contents; each call clears what must start
// at zero (barrier words, status) and rewrites everything else before reading it.  Calls that
// overlap on the GPU (different streams, or host threads) race on the array and must be
// serialised by the caller.
// ================================================================================================
}  // namespace tsf

#include <mutex>
#include "../../include/tsfcde.h"

namespace {

constexpr int64_t kStaticMaxN = 16383;                       // L = 32768, N = 16384
constexpr size_t kStaticScratchBytes = size_t(3) << 20;      // 3 MiB
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

struct StaticDevice {
  bool ready = false;
  int status = 0;
  unsigned char *base = nullptr;   // device address of g_static_scratch on this device
  int sms = 0;
  size_t smem = 0;
};
constexpr int kMaxDevices = 64;
StaticDevice g_static_dev[kMaxDevices];
std::mutex g_static_mu;

__global__ void __launch_bounds__(tsf::kThreads, 1)
static_operator_kernel(tsf::Args A, double *omega, double *gtmp, double beta, double eta, double q,
                       double kp, double km, int op, const double *x, double *y, double *xin) {
  using namespace tsf;
  const Smem S = smem_view(lp_max_of(A), tw_max_of(A));
  grid_sync_init();
  const int n = A.n, L = A.cp.L;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
  // Grunwald recurrence (Lemma 3), one thread, explicit rounding as in the setup path
  if (gt == 0) {
    double gk = 1.0;
    gtmp[0] = gk;
    for (int k = 1; k <= n + 1; ++k) {
      const double f = __dadd_rn(1.0, -__ddiv_rn(beta + 1.0, (double)k));
      gk = __dmul_rn(f, gk);
      gtmp[k] = gk;
    }
  }
  for (int k = gt; k < L; k += gs) {
    double s, c;
    sincospi(-2.0 * (double)k / (double)L, &s, &c);
    const_cast<double2 *>(A.twL)[k] = make_double2(c, s);
    xin[k] = k < n ? x[k] : 0.0;
  }
  if (!grid_sync(A)) return;
  {
    double lam1, lam0, lamm1;
    wsgd_lambdas(beta, lam1, lam0, lamm1);
    for (int k = gt; k <= n + 1; k += gs) {
      double w = __dmul_rn(lam1, gtmp[k]);
      if (k >= 1) w = __dadd_rn(w, __dmul_rn(lam0, gtmp[k - 1]));
      if (k >= 2) w = __dadd_rn(w, __dmul_rn(lamm1, gtmp[k - 2]));
      omega[k] = w;
    }
  }
  if (!grid_sync(A)) return;
  // spectrum of W's circulant embedding (t_0 = omega_1, ..., t_{n-1} = omega_n, t_{-1} = omega_0)
  col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y1,
                        [&](int m, double2) -> double2 {
                          double v[2];
#pragma unroll
                          for (int h = 0; h < 2; ++h) {
                            const int i = 2 * m + h;
                            v[h] = i < n ? omega[i + 1] : (i == L - 1 ? omega[0] : 0.0);
                          }
                          return make_double2(v[0], v[1]);
                        });
  if (!grid_sync(A)) return;
  row_pass<1, double2>(A, S, A.twL, A.Y1, nullptr, nullptr, const_cast<double2 *>(A.What), 1.0, -1);
  if (!grid_sync(A)) return;
  // operator spectrum: A = eta I - sigma L or B = eta I + (1-sigma) L, scaled 1/(4N)
  {
    LevelScalars s;
    s.eta = eta;
    s.q = q;
    s.kp = kp;
    s.km = km;
    const ConvPlan &P = A.cp;
    for (int sl = gt; sl <= P.N; sl += gs) {
      const int k = sl == P.N ? P.N : ((sl & (P.N2 - 1)) * P.N1 + (sl >> P.lg2));
      double2 sa, sb;
      // twL was written earlier in this launch: a plain (coherent) load, not the read-only path
      ab_symbols(A, s, A.twL[k], sl == P.N, A.What[sl], sa, sb);
      A.SA[sl] = op == 0 ? sa : sb;
    }
  }
  if (!grid_sync(A)) return;
  col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y1,
                        [&](int m, double2) -> double2 { return ld2(xin, m); });
  if (!grid_sync(A)) return;
  row_pass<0, double2>(A, S, A.twL, A.Y1, A.Y2, A.SA, nullptr, 0.0, -1);
  if (!grid_sync(A)) return;
  col_pass<true, false, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, A.Y2, nullptr,
                        [&](int m, double2 z) -> double2 {
                          if (2 * m < n) y[2 * m] = z.x;
                          if (2 * m + 1 < n) y[2 * m + 1] = z.y;
                          return z;
                        });
}

// Scratch layout inside g_static_scratch for a problem of n interior points.
struct StaticLayout {
  size_t off = 0;
  unsigned char *base;
  template <typename T>
  T *take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T *p = reinterpret_cast<T *>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

// One-time set-up per device (run by the first call on that device, with it current): the
// device address of the scratch array, the SM count, and the kernel's shared-memory limit.
int static_setup(int dev, StaticDevice **out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  StaticDevice &d = g_static_dev[dev];
  if (!d.ready) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess) return TSFCDE_E_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return TSFCDE_E_CUDA;
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return TSFCDE_E_CUDA;
    // largest plan (N = 16384 = 128 x 128): lines of 128 points, 4096 complex per buffer at most
    const size_t smem = (size_t)(2 * 4096 + 4096) * sizeof(double2) + 4 * 32 * sizeof(double);
    if (smem > (size_t)optin) return TSFCDE_E_INVALID_ARG;
    if (cudaFuncSetAttribute((const void *)static_operator_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return TSFCDE_E_CUDA;
    d.base = static_cast<unsigned char *>(ptr);
    d.sms = sms;
    d.smem = smem;
    d.ready = true;
  }
  *out = &d;
  return TSFCDE_OK;
}

}  // namespace

extern "C" int tsfcde_apply_operator_static(int64_t N, double beta, double sigma, double eta,
                                            double q, double kappa_plus, double kappa_minus,
                                            int32_t op, const double *x, double *y, void *stream) {
  using namespace tsf;
  if (N < 1 || N > kStaticMaxN) return TSFCDE_E_INVALID_ARG;
  if (op != TSFCDE_OP_A && op != TSFCDE_OP_B) return TSFCDE_E_INVALID_ARG;
  if (!x || !y || !(beta > 1.0 && beta <= 2.0) || !(sigma > 0.0 && sigma <= 1.0)) return TSFCDE_E_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TSFCDE_E_NO_DEVICE;
  StaticDevice *d = nullptr;
  int st = static_setup(dev, &d);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;

  Args A;
  memset(&A, 0, sizeof(A));
  const int n = (int)N;
  A.n = n;
  A.M = 1;
  int lgL = 3;
  while ((1 << lgL) < 2 * n) ++lgL;
  A.cp.lgL = lgL;
  A.cp.L = 1 << lgL;
  A.cp.lgN = lgL - 1;
  A.cp.N = 1 << A.cp.lgN;
  A.cp.lg1 = A.cp.lgN / 2;
  A.cp.lg2 = A.cp.lgN - A.cp.lg1;
  A.cp.N1 = 1 << A.cp.lg1;
  A.cp.N2 = 1 << A.cp.lg2;
  A.bp.lg1 = 1;   // no complex-plan phases run here
  A.bp.lg2 = 1;
  A.sigma = sigma;
  A.spin_limit = kSpinLimit;
  const int G = std::min(d->sms, kMaxGrid);
  auto cap = [&](int items, int lines_per_item, int lg) {
    const int per = (items + G - 1) / G;
    const int fit = std::max(1, (4096 >> lg) / lines_per_item);
    return std::max(1, std::min(per, fit));
  };
  A.cap_col = cap(A.cp.N2, 1, A.cp.lg1);
  A.cap_row = cap(A.cp.N1 / 2 + 1, 2, A.cp.lg2);
  A.cap_bcol = 1;
  A.cap_brow = 1;
  const size_t smem = level_smem_bytes(A);
  if (smem > d->smem) return TSFCDE_E_INVALID_ARG;

  const size_t L = (size_t)A.cp.L, Nc = (size_t)A.cp.N;
  StaticLayout lay;
  lay.base = d->base;
  A.bar = lay.take<unsigned>(kBarWords);
  A.status = lay.take<int>(4);
  A.twL = lay.take<double2>(L);
  A.What = lay.take<double2>(Nc + 1);
  A.SA = lay.take<double2>(Nc + 1);
  A.Y1 = lay.take<double2>(Nc);
  A.Y2 = lay.take<double2>(Nc);
  double *xin = lay.take<double>(L);
  double *omega = lay.take<double>(N + 2);
  double *gtmp = lay.take<double>(N + 2);
  if (lay.off > kStaticScratchBytes) return TSFCDE_E_INVALID_ARG;

  // barrier words and status must start at zero on every call
  if (cudaMemsetAsync(A.bar, 0, kBarWords * sizeof(unsigned), s) != cudaSuccess) return TSFCDE_E_CUDA;
  if (cudaMemsetAsync(A.status, 0, 4 * sizeof(int), s) != cudaSuccess) return TSFCDE_E_CUDA;
  void *args[] = {&A, &omega, &gtmp, &beta, &eta, &q, &kappa_plus, &kappa_minus, &op, &x, &y, &xin};
  if (cudaLaunchCooperativeKernel((const void *)static_operator_kernel, G, kThreads, args, smem, s) !=
      cudaSuccess)
    return TSFCDE_E_CUDA;
  int hst[2] = {0, 0};
  if (cudaMemcpyAsync(hst, A.status, sizeof(hst), cudaMemcpyDeviceToHost, s) != cudaSuccess) return TSFCDE_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return TSFCDE_E_CUDA;
  return hst[0];
}
