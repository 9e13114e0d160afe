// Internal declarations shared by the translation units of libtsfcde (not part of the C ABI).
//
// Data layout in device memory (one context = one TSFCDE instance):
//   * real vectors of the level solve (u, x, r, r~, p, q, u_cgs, v^, H) hold n values followed by
//     zeros up to L = max(8, 2^ceil(log2 2n)), the length of the circulant embedding of an n x n
//     Toeplitz matrix, through which Section 3.2 evaluates the products with A and B by FFT;
//     viewed as L/2 complex numbers z_m = (v_{2m}, v_{2m+1}) they feed a half-length complex
//     FFT (real-input trick);
//   * FFTs of length N = L/2 are split N = N1 x N2 (four-step): "column" items are the N2
//     strided lines of N1 points, "row" items are the N1 contiguous lines of N2 points.  Spectra
//     of Toeplitz kernels are stored in the permuted order slot(k) = (k mod N1) N2 + k / N1
//     produced by the row pass, plus the Nyquist value at slot N;
//   * the Bluestein transforms (n-point DFTs of the circulant columns, Eq. (3.7) and the
//     diagonalisation below it) use complex FFTs of length L split L = Nb1 x Nb2 the same way;
//   * the history ring holds d^s = u^{s+1} - u^s for every committed level s, level-major with a
//     256-byte aligned stride, FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tsf {

constexpr int kThreads = 256;                 // threads per CTA of every kernel but one:
constexpr int kWideThreads = 512;             // the whole-grid level march for FFT half-lengths
constexpr int kWideMinLgN = 19;               // N >= 2^19 (more warps to cover memory latency)
constexpr long long kSpinLimit = 1ll << 23;   // default bound on a barrier wait (a few seconds)

// status codes (mirror include/tsfcde.h)
constexpr int kOK = 0, kEInvalid = 1, kENoMem = 2, kECuda = 3, kENonFinite = 4,
              kENotConverged = 5, kEBreakdown = 6, kESingular = 7, kETimeout = 8, kEState = 9,
              kEBounds = 11;
constexpr int kFP64 = 0, kMixed = 1;

struct ConvPlan {  // real length L, complex length N = L/2 = N1 * N2
  int L, lgL, N, lgN, N1, lg1, N2, lg2;
};
struct CplxPlan {  // complex length Nc = L = N1 * N2
  int Nc, lgNc, N1, lg1, N2, lg2;
};

struct ff;    // float-float real (defined below)
struct ffc;   // float-float complex

// Everything a device kernel needs, passed by value.
struct Args {
  int n, M;
  ConvPlan cp;
  CplxPlan bp;
  int precond;          // 0 Strang, 1 T. Chan, 2 none
  double sigma, hscale; // sigma = 1 - alpha/2, hscale = tau^-alpha / Gamma(2-alpha)
  double tol;
  int maxit;
  int cap_col, cap_row, cap_bcol, cap_brow;   // lines per CTA chunk in each phase kind
  // tables
  const double2 *twL;     // e^{-2 pi i k / L}, k < L
  const double2 *What;    // spectrum of the L-embedding of W_beta, permuted, N+1
  const double2 *LamW;    // n-point DFT of the circulant column s(W_beta), n
  const double2 *LamQ;    // n-point DFT of the circulant column s(Q), n
  const double2 *BhI;     // Bluestein kernel spectrum for the inverse n-DFT, permuted, L
  const double2 *chirpI;  // e^{+i pi k^2 / n}, k < n
  const double *lv_eta, *lv_q, *lv_kp, *lv_km;  // per level: eta_j, gamma/(2h), d+/h^b, d-/h^b
  const int *lv_newsym;   // per level: 1 if the level operators differ from the previous level
  const double *hc;       // hc[m] = a_m + b_{m+1} - b_m, m >= 1 (Lemma 1)
  const double *hl;       // hl[j] = a_j - b_j (Lemma 1, m = j)
  int src_rank;
  const double *src_x;    // src_rank x n
  const double *src_t;    // src_rank x M
  const double *f_dense;  // M x n or null
  // state
  double *u, *x, *r, *rt, *p, *q, *uu, *vh, *H;
  double *xb;             // minimum-residual iterate of the FP64 CGS
  double *ring;
  long long ring_stride;
  double2 *SA, *SB, *SP;  // per-level spectra (permuted, N+1), scaled by 1/(4N)
  double2 *Y1, *Y2;       // FFT work, L complex each
  double *cprime;         // first column of P^{-1}, n
  double *partials;       // 2 x gridDim x 4
  unsigned *bar;          // kBarWords barrier words: [0, 2) 64-bit arrival counter
  int *status;            // [0] status, [1] abort flag
  int *iters;             // M
  double *resid;          // M
  // mixed precision (FP32 inner CGS inside FP64 iterative refinement)
  int precision;          // 0 FP64, 1 mixed
  double inner_tol;       // relative residual target of each FP32 inner solve
  int inner_maxit, outer_maxit;
  double *g;              // FP64 right-hand side of the level
  float *x32, *r32, *rt32, *p32, *q32, *uu32, *vh32;   // FP32 inner Krylov vectors (L each)
  float *x32b;            // minimum-residual iterate of the FP32 inner solve
  float2 *SA32, *SP32;    // FP32 copies of the level spectra (rounded from FP64)
  float2 *Y1f, *Y2f;      // FP32 FFT work, L/2 complex each
  float2 *twL32;          // FP32 twiddles (rounded from the FP64 table)
  int *outer_iters;       // M: refinement steps per level
  int *escalated;         // M: 1 if the level fell back to FP64 CGS
  long long spin_limit;   // polls before a barrier wait gives up
  int test_skip;          // testing hook: CTA 0 skips its first barrier arrival
  int inject;             // testing hook (tsfcde_options.test_inject): 2 breakdown, 3 singular P
  int resident;           // one-CTA march: the per-level working arrays live in shared memory
  // fast history (blocked convolution in time by 2B-point FFTs; fh_B = 0: the direct sum)
  int fh_B, fh_lgB;       // block length B = 2^fh_lgB in levels
  int fh_lines;           // complex FFT lines of length 2B per shared-memory tile (2 points each)
  int fh_nblk;            // increment blocks whose spectra are kept
  double2 *fh_E;          // spectra of the increment blocks: block p, frequency k <= B, point i at
                          // (p (B+1) + k) ring_stride + i
  const double2 *fh_K;    // spectra of the kernel windows, scaled 1/(2B): window m >= 1 at
                          // (m-1)(B+1) + k
  double *fh_far;         // far part of the history of the current block's levels: B x ring_stride
  // float-float inner solve (mixed mode, levels where FP32 cannot resolve the operator)
  const int *lv_inner;    // per level: 0 FP32 inner solve, 1 float-float inner solve
  const double *lv_floor; // per level: FP64 residual accepted once refinement stagnates below it
  ff *xff, *rff, *rtff, *pff, *qff, *uuff, *vhff;   // float-float Krylov vectors (L each)
  ff *xffb;               // minimum-residual iterate of the float-float inner solve
  ffc *SAff, *SPff;       // float-float spectra (rounded from FP64), N+1
  ffc *Y1ff, *Y2ff;       // float-float FFT work, L/2 each
  ffc *twLff;             // float-float twiddles, L
  // constant coefficients: A^{(j+sigma)} = A for j >= 1, solved by the Gohberg-Semencul formula
  int gsf;                // 1: levels j >= 1 compute u^{j+1} = A^{-1} g (no Krylov iterations)
  double *gx, *gy;        // generators x = A^{-1} e_1, y = A^{-1} e_n (Eq. (3.5)); L each, zero tail
  double2 *SL, *SR, *SL0, *SR0;   // spectra of L_p / xi_0, R_p, L0_p / xi_0, R0_p (permuted, N+1)
  double2 *Y3;            // third FFT work buffer, N complex
};

// ---------------------------------------------------------------------------------------------
// complex helpers (double2 for the FP64 path, float2 for the FP32 inner solve)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a * conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 mul_i(double2 a) { return make_double2(-a.y, a.x); }     // * i
__device__ __forceinline__ double2 mul_mi(double2 a) { return make_double2(a.y, -a.x); }    // * -i

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 mul_i(float2 a) { return make_float2(-a.y, a.x); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

// ---------------------------------------------------------------------------------------------
// float-float numbers (an unevaluated sum hi + lo of two floats, |lo| <= ulp(hi)/2): about 48-bit
// significands computed on the FP32 pipe.  Error-free transformations after Dekker and Knuth
// (TwoSum, FastTwoSum) and the FMA-based product; additions use the "sloppy" form
// (s, e) = TwoSum(a.hi, b.hi); e += a.lo + b.lo; renormalise -- relative error about 2^-46 of
// |a| + |b|, which is what FFT butterflies and axpy updates need.
// ---------------------------------------------------------------------------------------------
struct __align__(8) ff {
  float hi, lo;
  __device__ __forceinline__ ff() {}
  __device__ __forceinline__ ff(double d) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
  }
  __device__ __forceinline__ ff(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ ff ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return ff(s, e);
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_fast_two_sum(s, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return ff(-a.hi, -a.lo); }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ ff operator+(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ ff operator-(ff a, ff b) { return ff_sub(a, b); }
__device__ __forceinline__ ff operator*(ff a, ff b) { return ff_mul(a, b); }
__device__ __forceinline__ ff operator-(ff a) { return ff_neg(a); }
__device__ __forceinline__ ff &operator+=(ff &a, ff b) { a = ff_add(a, b); return a; }

struct __align__(16) ffc {   // complex float-float
  ff x, y;
};
__device__ __forceinline__ ffc cadd(ffc a, ffc b) { ffc r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
__device__ __forceinline__ ffc csub(ffc a, ffc b) { ffc r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
__device__ __forceinline__ ffc cmul(ffc a, ffc b) {
  ffc r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
__device__ __forceinline__ ffc cmulc(ffc a, ffc b) {
  ffc r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.y * b.x - a.x * b.y;
  return r;
}
__device__ __forceinline__ ffc cconj(ffc a) { ffc r; r.x = a.x; r.y = -a.y; return r; }
__device__ __forceinline__ ffc mul_i(ffc a) { ffc r; r.x = -a.y; r.y = a.x; return r; }
__device__ __forceinline__ ffc mul_mi(ffc a) { ffc r; r.x = a.y; r.y = -a.x; return r; }
__device__ __forceinline__ void mkc(ffc &z, ff x, ff y) { z.x = x; z.y = y; }
__device__ __forceinline__ ffc to_ffc(double2 v) { ffc r; r.x = ff(v.x); r.y = ff(v.y); return r; }

template <typename T> struct RealOf;
template <> struct RealOf<double2> { using R = double; };
template <> struct RealOf<float2> { using R = float; };
template <> struct RealOf<ffc> { using R = ff; };
__device__ __forceinline__ void mkc(double2 &z, double x, double y) { z = make_double2(x, y); }
__device__ __forceinline__ void mkc(float2 &z, float x, float y) { z = make_float2(x, y); }

// ---------------------------------------------------------------------------------------------
// Butterflies.  FP64 and FP32 use the fused multiply-add form of the radix-2 butterfly
// (Goedecker's): y0 = a + w b takes two FMAs per component, y1 = a - w b = 2a - y0 one, so a
// twiddled radix-2 butterfly is 6 FMAs for its 10 flops (against 4 multiplies/FMAs and 4 adds
// plainly).  A twiddled radix-4 butterfly is built from four of them: with stage twiddles
// w1 = W^k, w2 = W^2k (W^3k = w1 w2),
//   c0,1 = a0 +- w2 a2,  d0,1 = a1 +- w2 a3,  y0,2 = c0 +- w1 d0,  y1,3 = c1 +- (-+i w1) d1,
// 24 FMAs and two twiddle loads per four points.  The untwiddled first stage uses plain adds.
// Float-float keeps the textbook form (its products are not single FMAs).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void bfly_fma(double2 a, double2 b, double2 w, double2 &y0, double2 &y1) {
  double tx = __fma_rn(w.x, b.x, a.x);
  tx = __fma_rn(-w.y, b.y, tx);
  double ty = __fma_rn(w.x, b.y, a.y);
  ty = __fma_rn(w.y, b.x, ty);
  y0 = make_double2(tx, ty);
  y1 = make_double2(__fma_rn(2.0, a.x, -tx), __fma_rn(2.0, a.y, -ty));
}
__device__ __forceinline__ void bfly_fma(float2 a, float2 b, float2 w, float2 &y0, float2 &y1) {
  float tx = __fmaf_rn(w.x, b.x, a.x);
  tx = __fmaf_rn(-w.y, b.y, tx);
  float ty = __fmaf_rn(w.x, b.y, a.y);
  ty = __fmaf_rn(w.y, b.x, ty);
  y0 = make_float2(tx, ty);
  y1 = make_float2(__fmaf_rn(2.f, a.x, -tx), __fmaf_rn(2.f, a.y, -ty));
}

template <typename T> struct FmaButterfly { static constexpr bool value = false; };
template <> struct FmaButterfly<double2> { static constexpr bool value = true; };
template <> struct FmaButterfly<float2> { static constexpr bool value = true; };

// Radix-4 DIT butterfly of Stockham sub-length Ls at position k (stage twiddles from tw[m << sh],
// tw[m] = e^{-2 pi i m / 2^lgT}; conjugated for SIGN > 0).
template <int SIGN, typename T>
__device__ __forceinline__ void radix4(T &a0, T &a1, T &a2, T &a3, const T *tw, int k, int sh, bool first) {
  if (first) {   // k = 0 throughout the first stage: no twiddles
    const T b0 = cadd(a0, a2), b1 = csub(a0, a2), b2 = cadd(a1, a3);
    const T b3 = SIGN < 0 ? mul_mi(csub(a1, a3)) : mul_i(csub(a1, a3));
    a0 = cadd(b0, b2);
    a1 = cadd(b1, b3);
    a2 = csub(b0, b2);
    a3 = csub(b1, b3);
    return;
  }
  if constexpr (FmaButterfly<T>::value) {
    T w1 = tw[k << sh], w2 = tw[(2 * k) << sh];
    if (SIGN > 0) { w1 = cconj(w1); w2 = cconj(w2); }
    T c0, c1, d0, d1;
    bfly_fma(a0, a2, w2, c0, c1);
    bfly_fma(a1, a3, w2, d0, d1);
    T v;
    if (SIGN < 0) mkc(v, w1.y, -w1.x);   // -i w1
    else mkc(v, -w1.y, w1.x);            // +i w1
    bfly_fma(c0, d0, w1, a0, a2);
    bfly_fma(c1, d1, v, a1, a3);
  } else {
    if (k) {
      T w1 = tw[k << sh];
      T w2 = tw[(2 * k) << sh];
      T w3 = tw[(3 * k) << sh];
      if (SIGN > 0) { w1 = cconj(w1); w2 = cconj(w2); w3 = cconj(w3); }
      a1 = cmul(a1, w1);
      a2 = cmul(a2, w2);
      a3 = cmul(a3, w3);
    }
    const T b0 = cadd(a0, a2), b1 = csub(a0, a2), b2 = cadd(a1, a3);
    const T b3 = SIGN < 0 ? mul_mi(csub(a1, a3)) : mul_i(csub(a1, a3));
    a0 = cadd(b0, b2);
    a1 = cadd(b1, b3);
    a2 = csub(b0, b2);
    a3 = csub(b1, b3);
  }
}

// Radix-2 DIT butterfly (the odd last stage of a power-of-two length).
template <int SIGN, typename T>
__device__ __forceinline__ void radix2(T &a0, T &a1, const T *tw, int k, int sh, bool first) {
  if (first) {
    const T y0 = cadd(a0, a1), y1 = csub(a0, a1);
    a0 = y0;
    a1 = y1;
    return;
  }
  if constexpr (FmaButterfly<T>::value) {
    T w1 = tw[k << sh];
    if (SIGN > 0) w1 = cconj(w1);
    T y0, y1;
    bfly_fma(a0, a1, w1, y0, y1);
    a0 = y0;
    a1 = y1;
  } else {
    if (k) {
      T w1 = tw[k << sh];
      if (SIGN > 0) w1 = cconj(w1);
      a1 = cmul(a1, w1);
    }
    const T y0 = cadd(a0, a1), y1 = csub(a0, a1);
    a0 = y0;
    a1 = y1;
  }
}

// ---------------------------------------------------------------------------------------------
// Stockham radix-4/2 FFT of `nl` lines of length P = 2^lgP in shared memory.
// Line l occupies a[l*P .. l*P+P); b is a scratch area of the same size.  SIGN = -1 forward,
// +1 inverse (unnormalised).  Twiddles come from tw[k] = e^{-2 pi i k / 2^lgT}, 2^lgT >= P
// (a shared-memory table of the line length in every caller).
// All threads of the CTA take part; returns the buffer holding the result.
// Stage with current sub-length Ls and radix r: for j < P/r, k = j mod Ls, a_q = x[j + q P/r]
// is twiddled by e^{SIGN 2 pi i q k/(r Ls)}, an r-point DFT is taken, and output q goes to
// y[(j - k) r + k + q Ls].
// ---------------------------------------------------------------------------------------------
template <int SIGN, typename T>
__device__ __forceinline__ T *smem_fft(T *a, T *b, int lgP, int nl, const T *tw, int lgT) {
  const int P = 1 << lgP;
  int lgLs = 0;
  while (lgLs < lgP) {
    const int Ls = 1 << lgLs;
    if (lgP - lgLs >= 2) {
      const int Q = P >> 2;
      const int nb = nl * Q;
      const int sh = lgT - lgLs - 2;
      for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        const int l = t >> (lgP - 2);
        const int j = t & (Q - 1);
        const int k = j & (Ls - 1);
        const T *x = a + l * P;
        T *y = b + l * P;
        T a0 = x[j], a1 = x[j + Q], a2 = x[j + 2 * Q], a3 = x[j + 3 * Q];
        radix4<SIGN>(a0, a1, a2, a3, tw, k, sh, lgLs == 0);
        const int base = ((j - k) << 2) + k;
        y[base] = a0;
        y[base + Ls] = a1;
        y[base + 2 * Ls] = a2;
        y[base + 3 * Ls] = a3;
      }
      lgLs += 2;
    } else {
      const int Q = P >> 1;
      const int nb = nl * Q;
      const int sh = lgT - lgLs - 1;
      for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        const int l = t >> (lgP - 1);
        const int j = t & (Q - 1);
        const int k = j & (Ls - 1);
        const T *x = a + l * P;
        T *y = b + l * P;
        T a0 = x[j], a1 = x[j + Q];
        radix2<SIGN>(a0, a1, tw, k, sh, lgLs == 0);
        const int base = ((j - k) << 1) + k;
        y[base] = a0;
        y[base + Ls] = a1;
      }
      lgLs += 1;
    }
    __syncthreads();
    T *t = a;
    a = b;
    b = t;
  }
  return a;
}

// ---------------------------------------------------------------------------------------------
// memory-order helpers and the bounded device-wide barrier
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int *p) { return *(const volatile int *)p; }

// The team of CTAs that works on one instance: the whole grid (one instance per launch) or a
// single CTA (batched instances, one per CTA at a time; small single instances).  Kept in shared
// memory, set at kernel start; every work split, reduction and barrier of the level solve goes
// through it.  `abort` mirrors the instance's abort flag for a one-CTA team, so that its barriers
// need no global-memory read.
struct TeamInfo {
  int idx, cnt, grid, abort;
};
__device__ __forceinline__ TeamInfo &team() {
  __shared__ TeamInfo t;
  return t;
}

// Index checks of the TSFCDE_CHECKED build: an index outside [0, n) is recorded (status word 0
// = TSFCDE_E_BOUNDS unless an error was already set, word 2 = the first failing site, word 3 =
// its index) and replaced by 0, so the access stays inside the array and nothing traps.  In
// the normal build TSF_CHK(i, n, site) is just i.
#ifdef TSFCDE_CHECKED
static __device__ __noinline__ long long chk_fail(const Args &A, long long i, int site) {
  if (atomicCAS(A.status + 2, 0, site) == 0) atomicExch(A.status + 3, (int)i);
  atomicCAS(A.status, 0, kEBounds);
  return 0;
}
#define TSF_CHK(i, n, site) \
  (((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n)) ? (long long)(i) : ::tsf::chk_fail(A, (long long)(i), (site)))
#else
#define TSF_CHK(i, n, site) (i)
#endif

// Sets a fatal status (first one wins) and raises the abort flag.
__device__ __forceinline__ void raise_fatal(const Args &A, int code) {
  atomicCAS(A.status, 0, code);
  atomicExch(A.status + 1, 1);
  __threadfence();
  *(volatile int *)&team().abort = 1;
}

// Barrier words: [0, 2) the 64-bit arrival counter; the rest is reserved.
constexpr int kMaxGrid = 1024;
constexpr int kBarWords = 32 + kMaxGrid;


// What the shared-memory line-twiddle table holds (source table, destination, line length), so
// that a pass whose line twiddles are already there does not reload them.  Reset at kernel start.
struct TwTag {
  const void *tab;
  const void *dst;
  int lg;
};
__device__ __forceinline__ TwTag &tw_tag() {
  __shared__ TwTag t;
  return t;
}

// Per-CTA count of grid barriers passed in this launch.
__device__ __forceinline__ unsigned long long &bar_count() {
  __shared__ unsigned long long k;
  return k;
}
// Run once at the start of every kernel that calls grid_sync (the team is the whole grid).
__device__ __forceinline__ void grid_sync_init() {
  if (threadIdx.x == 0) {
    bar_count() = 0ull;
    team().idx = blockIdx.x;
    team().cnt = gridDim.x;
    team().grid = 1;
    team().abort = 0;
    tw_tag().tab = nullptr;
  }
  __syncthreads();
}
// Team of one CTA (batched instances).
__device__ __forceinline__ void cta_team_init() {
  if (threadIdx.x == 0) {
    bar_count() = 0ull;
    team().idx = 0;
    team().cnt = 1;
    team().grid = 0;
    team().abort = 0;
    tw_tag().tab = nullptr;
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_add_release_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch: a 64-bit arrival counter that only grows during
// a launch (zeroed by the host before it).  At its k-th barrier a CTA adds 1 with release
// semantics and waits until the counter reaches k * gridDim.x.  Every wait is bounded: after
// kSpinLimit polls the CTA records E_TIMEOUT, raises the abort flag and leaves.  Returns false
// when the kernel must stop (abort raised anywhere); all CTAs then return without touching the
// barrier again.
__device__ __forceinline__ bool grid_sync(const Args &A) {
  __shared__ int s_go;
  __syncthreads();
  if (!team().grid) {   // one-CTA team: a block barrier orders the CTA's global writes
    if (threadIdx.x == 0) s_go = *(volatile int *)&team().abort == 0;
    __syncthreads();
    return s_go != 0;
  }
  if (threadIdx.x == 0) {
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(A.bar);
    const unsigned long long k = ++bar_count();
    const unsigned long long target = k * (unsigned long long)gridDim.x;
    __threadfence();
    if (!(A.test_skip && blockIdx.x == 0 && k == 1)) red_add_release_u64(cnt, 1ull);
    long long spins = 0;
    while (ld_acquire_u64(cnt) < target) {
      if (++spins > A.spin_limit) {
        raise_fatal(A, kETimeout);
        break;
      }
      if ((spins & 255) == 0 && ld_volatile_i32(A.status + 1)) break;
    }
    __threadfence();
    s_go = ld_volatile_i32(A.status + 1) == 0;
  }
  __syncthreads();
  return s_go != 0;
}

// Deterministic block reduction of K values (fixed shuffle tree, fixed warp order).
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double *sm /* K*32 doubles */) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    v[k] = x;
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sm[k * 32 + w] = v[k];
  }
  __syncthreads();
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += sm[k * 32 + i];
    v[k] = s;
  }
  __syncthreads();
}

// Host-side precision controller of the mixed mode: for level j with eta_j, q, kappa_pm
// returns the inner type (0 FP32, 1 float-float) and the FP64 residual floor.
inline void precision_control(double sigma, double beta, double eta, double q, double kp, double km,
                              int inner_opt, double tol, int *inner, double *floor_out) {
  const double lam1 = (beta * beta + 3.0 * beta + 2.0) / 12.0;
  const double lam0 = (4.0 - beta * beta) / 6.0;
  const double w1 = lam0 - beta * lam1;   // omega_1 = lambda_1 g_1 + lambda_0 g_0
  const double ab = (w1 < 0 ? -w1 : w1);
  const double qa = (q < 0 ? -q : q);
  const double kappa = 1.0 + sigma * ((kp + km) * 2.0 * ab + 2.0 * qa) / eta;
  const double u32 = 5.9604644775390625e-08, u64 = 1.1102230246251565e-16;
  int t = (u32 * kappa < 1e-3) ? 0 : 1;
  if (inner_opt == 1) t = 0;
  if (inner_opt == 2) t = 1;
  *inner = t;
  const double fl = 64.0 * u64 * kappa;
  *floor_out = fl > tol ? fl : tol;
}

// Per-CTA work arrays of the batched solver (sized for the largest instance).
struct CtaScratch {
  double *x, *r, *rt, *p, *q, *uu, *vh, *H, *cprime, *partials, *g, *xb;
  unsigned *bar;
  double2 *SA, *SB, *SP, *Y1, *Y2, *Y3;
  float *x32, *r32, *rt32, *p32, *q32, *uu32, *vh32;
  float2 *SA32, *SP32, *Y1f, *Y2f;
  ff *xff, *rff, *rtff, *pff, *qff, *uuff, *vhff;
  ffc *SAff, *SPff, *Y1ff, *Y2ff;
  float *x32b;
  ff *xffb;
};
// Per-instance inputs of the batched setup (constant coefficients).
struct InstanceSetup {
  double alpha, beta, tau, h, gamma, d_plus, d_minus;
  double *omega, *gtmp;
  double2 *BhF;
};
struct BatchArgs {
  int count;
  const Args *inst;            // per-instance Args (per-CTA pointers patched in-kernel)
  const InstanceSetup *setup;  // per-instance setup inputs
  const CtaScratch *cta;       // per-CTA work arrays
  const int *order;            // work-queue order (largest instances first)
  unsigned *next;              // work-queue counter (zeroed before each launch)
};

// Raise a kernel's dynamic shared-memory limit to the device maximum (minus its static shared
// memory).  The limit is a per-function, process-wide attribute: setting it to one context's
// need would break another context that needs more; occupancy depends only on what each launch
// requests.  Returns the usable dynamic bytes, or 0 on a CUDA error.
inline size_t raise_smem_limit(const void *fn, const cudaDeviceProp &prop) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return 0;
  const size_t dyn = prop.sharedMemPerBlockOptin > fa.sharedSizeBytes
                         ? prop.sharedMemPerBlockOptin - fa.sharedSizeBytes : 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) return 0;
  return dyn;
}

// Bytes of the per-CTA shared-memory line buffers, line twiddles and reduction scratch of a plan
// (the layout smem_view uses): two buffers of the largest chunk, the longest line's twiddles and
// 4 x 32 doubles.
__host__ __device__ inline size_t smem_lines_bytes(const Args &A) {
  int m = A.cap_col << A.cp.lg1;
  m = m > ((2 * A.cap_row) << A.cp.lg2) ? m : ((2 * A.cap_row) << A.cp.lg2);
  m = m > (A.cap_bcol << A.bp.lg1) ? m : (A.cap_bcol << A.bp.lg1);
  m = m > (A.cap_brow << A.bp.lg2) ? m : (A.cap_brow << A.bp.lg2);
  int lt = A.cp.lg1 > A.cp.lg2 ? A.cp.lg1 : A.cp.lg2;
  lt = lt > A.bp.lg1 ? lt : A.bp.lg1;
  lt = lt > A.bp.lg2 ? lt : A.bp.lg2;
  if (A.fh_B) {   // fast-history tiles: fh_lines lines of 2B points
    m = m > (A.fh_lines << (A.fh_lgB + 1)) ? m : (A.fh_lines << (A.fh_lgB + 1));
    lt = lt > A.fh_lgB + 1 ? lt : A.fh_lgB + 1;
  }
  return (size_t)(2 * m + (1 << lt)) * 16 + 4 * 32 * sizeof(double);
}

// The working arrays of one level solve that a one-CTA march keeps in shared memory after the
// line buffers: Krylov vectors and FFT work arrays of every precision in use, the level spectra,
// P^{-1}'s circulant column and the reduction partials.  Tables, the level state u, the history
// ring, the Gohberg-Semencul generators and per-level outputs stay in global memory (they outlive
// a launch).  Returns the bytes; with `base` non-null, points A's fields into [base, base+bytes).
struct ResCarve {
  size_t off;
  char *base;
  template <typename T>
  __host__ __device__ T *take(size_t count) {
    off = (off + 15) & ~size_t(15);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};
__host__ __device__ inline size_t resident_patch(Args &A, char *base) {
  ResCarve c{0, base};
  const size_t L = (size_t)A.cp.L, N = (size_t)A.cp.N, n = (size_t)A.n;
  A.x = c.take<double>(L);
  A.r = c.take<double>(L);
  A.rt = c.take<double>(L);
  A.p = c.take<double>(L);
  A.q = c.take<double>(L);
  A.uu = c.take<double>(L);
  A.vh = c.take<double>(L);
  A.H = c.take<double>(L);
  A.xb = c.take<double>(L);
  A.Y1 = c.take<double2>(L);
  A.Y2 = c.take<double2>(L);
  A.SA = c.take<double2>(N + 1);
  A.SB = c.take<double2>(N + 1);
  A.SP = c.take<double2>(N + 1);
  A.cprime = c.take<double>(n);
  A.partials = c.take<double>(8);
  if (A.gsf) A.Y3 = c.take<double2>(N);
  if (A.precision == kMixed) {
    A.g = c.take<double>(L);
    A.x32 = c.take<float>(L);
    A.r32 = c.take<float>(L);
    A.rt32 = c.take<float>(L);
    A.p32 = c.take<float>(L);
    A.q32 = c.take<float>(L);
    A.uu32 = c.take<float>(L);
    A.vh32 = c.take<float>(L);
    A.x32b = c.take<float>(L);
    A.SA32 = c.take<float2>(N + 1);
    A.SP32 = c.take<float2>(N + 1);
    A.Y1f = c.take<float2>(N);
    A.Y2f = c.take<float2>(N);
    A.xff = c.take<ff>(L);
    A.rff = c.take<ff>(L);
    A.rtff = c.take<ff>(L);
    A.pff = c.take<ff>(L);
    A.qff = c.take<ff>(L);
    A.uuff = c.take<ff>(L);
    A.vhff = c.take<ff>(L);
    A.xffb = c.take<ff>(L);
    A.SAff = c.take<ffc>(N + 1);
    A.SPff = c.take<ffc>(N + 1);
    A.Y1ff = c.take<ffc>(N);
    A.Y2ff = c.take<ffc>(N);
  }
  return (c.off + 15) & ~size_t(15);
}

// Host-side entry points implemented in level_kernels.cu.
int launch_levels(const Args &A, int grid, size_t smem, cudaStream_t st, int j0, int j1,
                  int threads = kThreads);
int launch_levels_wide(const Args &A, int grid, size_t smem, cudaStream_t st, int j0, int j1);
int launch_levels_cta(const Args &A, size_t smem, cudaStream_t st, int j0, int j1);
int launch_apply(const Args &A, int grid, size_t smem, cudaStream_t st, int op, int j,
                 const double *xin, double *yout);
int launch_setup(const Args &A, int grid, size_t smem, cudaStream_t st, const double *omega,
                 double2 *What, double2 *LamW, double2 *LamQ, double2 *BhI, double2 *BhF,
                 double2 *chirpI, double2 *twL, double beta, int precond);
int launch_weights(double *omega, double *g_tmp, int n, double beta, cudaStream_t st);
int launch_time_tables(int M, double alpha, double tau, double h, double beta, const double *gam,
                       const double *dp, const double *dm, double *hc, double *hl, double *eta,
                       double *q, double *kp, double *km, cudaStream_t st);
size_t level_smem_bytes(const Args &A);
const void *level_kernel_ptr();
const void *level_kernel_cta_ptr();
const void *level_kernel_wide_ptr();
const void *history_kernel_ptr();
int launch_history(const Args &A, int grid, size_t smem, cudaStream_t st, int j);
int launch_fh_kernel_spectra(const double *hc, int M, int B, int nblk, double2 *K, cudaStream_t st);
int launch_fp64_fma(double *out, int blocks, int iters, cudaStream_t st);
int launch_level_rebuild(const double *u0, const double *uc, const double *ring, long long stride, int n,
                         int j, int c, double *out, cudaStream_t st);
const void *batch_level_kernel_ptr();
const void *batch_setup_kernel_ptr();
int launch_batch(const BatchArgs &B, int grid, size_t smem, cudaStream_t st, int setup, int j0, int j1);
const void *apply_kernel_ptr();
const void *setup_kernel_ptr();

}  // namespace tsf
