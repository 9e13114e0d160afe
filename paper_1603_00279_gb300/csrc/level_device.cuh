// Device code of the level solve shared by the kernels of level_kernels.cu (whole-grid march,
// operator products, setup), level_wide.cu (512-thread and one-CTA marches) and
// batch_kernels.cu (batched instances).  Included by those translation units only; the build
// compiles them in parallel.  The phase structure is described in level_kernels.cu.
#pragma once
#include "tsfcde_internal.cuh"

namespace tsf {


// ------------------------------------------------------------------------------------------------
// per-CTA shared memory view (sized for FP64 lines; FP32 passes use the same regions)
// ------------------------------------------------------------------------------------------------
struct Smem {
  void *a, *b;   // ping-pong line buffers
  void *tw;      // twiddles of the current pass's line length, e^{-2 pi i m / P}
  double *red;   // reduction scratch (4 * 32 doubles)
};

__device__ __forceinline__ int tw_max_of(const Args &A) {
  int lt = max(max(A.cp.lg1, A.cp.lg2), max(A.bp.lg1, A.bp.lg2));
  if (A.fh_B) lt = max(lt, A.fh_lgB + 1);
  return 1 << lt;
}

__device__ __forceinline__ Smem smem_view(int lp_max, int tw_max) {
  extern __shared__ double2 dsm[];
  Smem s;
  s.a = dsm;
  s.b = dsm + lp_max;
  s.tw = dsm + 2 * lp_max;
  s.red = reinterpret_cast<double *>(dsm + 2 * lp_max + tw_max);
  return s;
}

__device__ __forceinline__ int lp_max_of(const Args &A) {
  int m = A.cap_col << A.cp.lg1;
  m = max(m, (2 * A.cap_row) << A.cp.lg2);
  m = max(m, A.cap_bcol << A.bp.lg1);
  m = max(m, A.cap_brow << A.bp.lg2);
  if (A.fh_B) m = max(m, A.fh_lines << (A.fh_lgB + 1));
  return m;
}

// Fill S.tw with the line twiddles e^{-2 pi i m / 2^lgP}, m < 2^lgP (a subset of the L table).
// Skipped when the table already holds them (the tag is CTA-uniform: read after a barrier).
template <typename T>
__device__ __forceinline__ void load_line_twiddles(const Args &A, const Smem &S, const T *twG, int lgP) {
  __syncthreads();
  TwTag &tg = tw_tag();
  if (tg.tab == static_cast<const void *>(twG) && tg.dst == S.tw && tg.lg == lgP) return;
  const int P = 1 << lgP, sh = A.cp.lgL - lgP;
  T *tw = static_cast<T *>(S.tw);
  for (int m = threadIdx.x; m < P; m += blockDim.x) tw[m] = twG[TSF_CHK(m << sh, A.cp.L, 1)];
  __syncthreads();
  if (threadIdx.x == 0) {
    tg.tab = twG;
    tg.dst = S.tw;
    tg.lg = lgP;
  }
}

// Contiguous item range of this CTA: [lo, hi).
__device__ __forceinline__ void my_items(int nitems, int &lo, int &hi) {
  const TeamInfo t = team();
  const int per = (nitems + t.cnt - 1) / t.cnt;
  lo = min(nitems, t.idx * per);
  hi = min(nitems, lo + per);
}
// Grid-stride loop bounds over the team: first index and stride.
__device__ __forceinline__ int team_tid() { return team().idx * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int team_threads() { return team().cnt * blockDim.x; }

// ------------------------------------------------------------------------------------------------
// Column pass of a four-step FFT: lines of P1 = 2^lg1 points, 2^lg2 of them, element m = m1*P2+m2.
// INV: line m2 loads Yin[k1*P2 + m2] * conj(W^{m2 k1}) and is inverse-transformed (with Yin2
//      given, the difference Yin - Yin2 is loaded).
// body(m, z) -> next forward input (z: inverse result when INV, otherwise undefined).
// FWD: forward transform of body's outputs, twiddle W^{m2 k1}, store Yout[k1*P2 + m2].
// W^{e} = twG[e << tws] (tws = 1 for the half-length conv plan, 0 for the length-L plan).
// ------------------------------------------------------------------------------------------------
template <bool INV, bool FWD, typename T, class Body>
__device__ __forceinline__ void col_pass(const Args &A, const Smem &S, const T *twG, int lg1, int lg2,
                                         int tws, int cap, const T *Yin, T *Yout, Body body,
                                         const T *Yin2 = nullptr) {
  const int P1 = 1 << lg1, P2 = 1 << lg2;
  T *tw = static_cast<T *>(S.tw);
  int lo, hi;
  my_items(P2, lo, hi);
  if (lo < hi) load_line_twiddles<T>(A, S, twG, lg1);
  for (int c0 = lo; c0 < hi; c0 += cap) {
    const int cnt = min(cap, hi - c0);
    T *a = static_cast<T *>(S.a), *b = static_cast<T *>(S.b);
    if (INV) {
      for (int e = threadIdx.x; e < cnt * P1; e += blockDim.x) {
        const int l = e % cnt, k1 = e / cnt, m2 = c0 + l;
        T v = Yin[TSF_CHK((k1 << lg2) + m2, P1 * P2, 2)];
        if (Yin2) v = csub(v, Yin2[TSF_CHK((k1 << lg2) + m2, P1 * P2, 3)]);
        a[(l << lg1) + k1] = cmulc(v, twG[TSF_CHK((m2 * k1) << tws, A.cp.L, 4)]);
      }
      __syncthreads();
      a = smem_fft<+1>(a, b, lg1, cnt, tw, lg1);
      b = (a == static_cast<T *>(S.a)) ? static_cast<T *>(S.b) : static_cast<T *>(S.a);
    }
    for (int e = threadIdx.x; e < cnt * P1; e += blockDim.x) {
      const int l = e % cnt, m1 = e / cnt, m2 = c0 + l;
      const int idx = (l << lg1) + m1;
      a[idx] = body(TSF_CHK((m1 << lg2) + m2, P1 * P2, 5), a[idx]);
    }
    __syncthreads();
    if (FWD) {
      a = smem_fft<-1>(a, b, lg1, cnt, tw, lg1);
      for (int e = threadIdx.x; e < cnt * P1; e += blockDim.x) {
        const int l = e % cnt, k1 = e / cnt, m2 = c0 + l;
        Yout[TSF_CHK((k1 << lg2) + m2, P1 * P2, 6)] = cmul(a[(l << lg1) + k1], twG[TSF_CHK((m2 * k1) << tws, A.cp.L, 7)]);
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Row pass of the half-length (real-input) convolution plan.  Item it < N1/2+1 holds rows
// (ka, kb) = (it, N1-it) (rows 0 and N1/2 pair with themselves).  After the forward row FFTs,
// Z_k and Z_{N-k} sit in the same item, which is what the real-FFT split needs:
//   X_k = (E2 + w O2)/2, X_{k+N} = (E2 - w O2)/2, E2 = Z_k + conj Z_{N-k},
//   O2 = -i (Z_k - conj Z_{N-k}), w = e^{-2 pi i k / L}.
// MODE 0 (convolve): Y = S X at k and k+N (S_{k+N} = conj S_{N-k}, S_N stored at slot N), then
//   the inverse split and the inverse row FFTs; result to Yout.  Spectra are pre-scaled 1/(4N).
// MODE 1 (spectrum, FP64 only): store X_k (times `scale`) into Sout at slot(k) and X_N at slot
//   N, and, when sym_level >= 0, also the spectra of A and B of that level at the same slots
//   (plus their FP32 copies in the mixed mode).
// ------------------------------------------------------------------------------------------------
struct LevelScalars {
  double eta, q, kp, km;
};
__device__ __forceinline__ double l21_a(double alpha, double sigma, int l);
__device__ __forceinline__ double l21_b(double alpha, double sigma, int l);

// lambda_1, lambda_0, lambda_{-1} of Lemma 2, each operation rounded on its own (no contraction
// into fused multiply-adds), in the order the formulas are written: the weights then round
// exactly as a plain binary64 evaluation of Lemma 2 does on any conforming host.
__device__ __forceinline__ void wsgd_lambdas(double beta, double &lam1, double &lam0, double &lamm1) {
  const double bb = __dmul_rn(beta, beta), b3 = __dmul_rn(3.0, beta);
  lam1 = __ddiv_rn(__dadd_rn(__dadd_rn(bb, b3), 2.0), 12.0);
  lam0 = __ddiv_rn(__dsub_rn(4.0, bb), 6.0);
  lamm1 = __ddiv_rn(__dadd_rn(__dsub_rn(bb, b3), 2.0), 12.0);
}

__device__ __forceinline__ LevelScalars level_scalars(const Args &A, int j) {
  LevelScalars s;
  s.eta = A.lv_eta[j];
  s.q = A.lv_q[j];
  s.kp = A.lv_kp[j];
  s.km = A.lv_km[j];
  return s;
}

// Spectra of A = eta I - sigma L and B = eta I + (1-sigma) L at frequency k of the L-embedding,
// L = q Q + kp W + km W^T; Q's symbol is 2 i sin(2 pi k / L), W^T's is conj(W's).  Scaled 1/(4N).
__device__ __forceinline__ void ab_symbols(const Args &A, const LevelScalars &s, double2 w_k,
                                           bool nyq, double2 Wk, double2 &sa, double2 &sb) {
  const double qs = nyq ? 0.0 : -2.0 * w_k.y;   // Im of Q's symbol (real part 0)
  const double lre = (s.kp + s.km) * Wk.x;
  const double lim = s.q * qs + (s.kp - s.km) * Wk.y;
  const double sc = 1.0 / (4.0 * (double)A.cp.N);
  sa = make_double2((s.eta - A.sigma * lre) * sc, (-A.sigma * lim) * sc);
  sb = make_double2((s.eta + (1.0 - A.sigma) * lre) * sc, ((1.0 - A.sigma) * lim) * sc);
}

__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }

__device__ __forceinline__ void store_ab(const Args &A, const LevelScalars &s, int slot, int k, bool nyq) {
  double2 sa, sb;
  ab_symbols(A, s, __ldg(A.twL + k), nyq, A.What[slot], sa, sb);
  A.SA[slot] = sa;
  A.SB[slot] = sb;
  if (A.precision == kMixed) {
    A.SA32[slot] = to_f2(sa);
    A.SAff[slot] = to_ffc(sa);
  }
}

template <int MODE, typename T>
__device__ __forceinline__ void row_pass(const Args &A, const Smem &S, const T *twG, const T *Yin, T *Yout,
                                         const T *Sym, double2 *Sout, double scale, int sym_level) {
  const ConvPlan &P = A.cp;
  const int N1 = P.N1, N2 = P.N2, lg2 = P.lg2, N = P.N;
  T *tw = static_cast<T *>(S.tw);
  const int nitems = N1 / 2 + 1;
  int lo, hi;
  my_items(nitems, lo, hi);
  if (lo < hi) load_line_twiddles<T>(A, S, twG, lg2);
  LevelScalars ls;
  if (MODE == 1 && sym_level >= 0) ls = level_scalars(A, sym_level);
  for (int i0 = lo; i0 < hi; i0 += A.cap_row) {
    const int cnt = min(A.cap_row, hi - i0);
    const int nl = 2 * cnt;
    T *a = static_cast<T *>(S.a), *b = static_cast<T *>(S.b);
    // load: line 2t = row ka, line 2t+1 = row kb
    for (int e = threadIdx.x; e < nl * N2; e += blockDim.x) {
      const int line = e >> lg2, k2 = e & (N2 - 1);
      const int it = i0 + (line >> 1);
      const int row = (line & 1) ? ((N1 - it) & (N1 - 1)) : it;
      a[e] = Yin[TSF_CHK((row << lg2) + k2, N, 8)];
    }
    __syncthreads();
    a = smem_fft<-1>(a, b, lg2, nl, tw, lg2);
    b = (a == static_cast<T *>(S.a)) ? static_cast<T *>(S.b) : static_cast<T *>(S.a);
    // split / multiply / merge, pairwise in k and N-k
    for (int e = threadIdx.x; e < cnt * N2; e += blockDim.x) {
      const int t = e >> lg2, k2 = e & (N2 - 1);
      const int it = i0 + t;
      const int ka = it, kb = (N1 - it) & (N1 - 1);
      T *ra = a + ((2 * t) << lg2);
      T *rb = (ka == kb) ? ra : a + ((2 * t + 1) << lg2);
      int k2p;
      if (ka == 0) {
        if (k2 > N2 / 2) continue;
        k2p = (N2 - k2) & (N2 - 1);
      } else if (ka == kb) {   // row N1/2
        if (k2 >= N2 / 2) continue;
        k2p = N2 - 1 - k2;
      } else {
        k2p = N2 - 1 - k2;
      }
      const int k = ka + N1 * k2;
      const T Zk = ra[k2], Zp = rb[k2p];
      const T w = twG[TSF_CHK(k, A.cp.L, 9)];
      const T Zc = cconj(Zp);
      const T E2 = cadd(Zk, Zc);
      const T O2 = mul_mi(csub(Zk, Zc));
      const T t2 = cmul(w, O2);
      const T X0 = cadd(E2, t2), X1 = csub(E2, t2);
      const int sk = (ka << lg2) + k2, sp = (kb << lg2) + k2p;
      const bool self = (rb == ra) && (k2p == k2);
      if (MODE == 0) {
        const T S0 = Sym[TSF_CHK(sk, N + 1, 10)];
        const T S1 = (k == 0) ? Sym[N] : cconj(Sym[TSF_CHK(sp, N + 1, 11)]);
        const T Y0 = cmul(S0, X0), Y1 = cmul(S1, X1);
        const T Ep = cadd(Y0, Y1);
        const T Op = cmulc(csub(Y0, Y1), w);
        const T iOp = mul_i(Op);
        ra[k2] = cadd(Ep, iOp);
        if (!self) rb[k2p] = cconj(csub(Ep, iOp));
      } else {
        const double sc = 0.5 * scale;
        const double2 v0 = make_double2((double)X0.x * sc, (double)X0.y * sc);
        const double2 v1 = make_double2((double)X1.x * sc, -(double)X1.y * sc);
        const double2 vn = make_double2((double)X1.x * sc, (double)X1.y * sc);
        Sout[TSF_CHK(sk, N + 1, 12)] = v0;
        if (!self) Sout[TSF_CHK(sp, N + 1, 13)] = v1;
        if (k == 0) Sout[N] = vn;
        if (A.precision == kMixed && sym_level >= 0 && Sout == A.SP) {
          A.SP32[sk] = to_f2(v0);
          A.SPff[sk] = to_ffc(v0);
          if (!self) {
            A.SP32[sp] = to_f2(v1);
            A.SPff[sp] = to_ffc(v1);
          }
          if (k == 0) {
            A.SP32[N] = to_f2(vn);
            A.SPff[N] = to_ffc(vn);
          }
        }
        if (sym_level >= 0) {
          store_ab(A, ls, sk, k, false);
          if (!self) store_ab(A, ls, sp, (N - k) & (N - 1), false);
          if (k == 0) store_ab(A, ls, N, N, true);
        }
      }
    }
    __syncthreads();
    if (MODE == 0) {
      a = smem_fft<+1>(a, b, lg2, nl, tw, lg2);
      for (int e = threadIdx.x; e < nl * N2; e += blockDim.x) {
        const int line = e >> lg2, k2 = e & (N2 - 1);
        const int it = i0 + (line >> 1);
        const int row = (line & 1) ? ((N1 - it) & (N1 - 1)) : it;
        if ((line & 1) && row == it) continue;   // self-paired row stored once
        Yout[TSF_CHK((row << lg2) + k2, N, 14)] = a[e];
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Row pass of the length-L complex plan (Bluestein), FP64: forward row FFT, then either multiply
// by Tab (permuted) and inverse row FFT into Y2 (MODE 0) or store the spectrum * scale (MODE 1).
// ------------------------------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void crow_pass(const Args &A, const Smem &S, const double2 *Tab,
                                          double2 *Out, double scale) {
  const CplxPlan &P = A.bp;
  const int lg2 = P.lg2, N2 = P.N2;
  double2 *tw = static_cast<double2 *>(S.tw);
  int lo, hi;
  my_items(P.N1, lo, hi);
  if (lo < hi) load_line_twiddles<double2>(A, S, A.twL, lg2);
  for (int r0 = lo; r0 < hi; r0 += A.cap_brow) {
    const int cnt = min(A.cap_brow, hi - r0);
    double2 *a = static_cast<double2 *>(S.a), *b = static_cast<double2 *>(S.b);
    for (int e = threadIdx.x; e < cnt * N2; e += blockDim.x) a[e] = A.Y1[TSF_CHK((r0 << lg2) + e, P.Nc, 15)];
    __syncthreads();
    a = smem_fft<-1>(a, b, lg2, cnt, tw, lg2);
    b = (a == static_cast<double2 *>(S.a)) ? static_cast<double2 *>(S.b) : static_cast<double2 *>(S.a);
    if (MODE == 0) {
      for (int e = threadIdx.x; e < cnt * N2; e += blockDim.x) a[e] = cmul(a[e], Tab[TSF_CHK((r0 << lg2) + e, P.Nc, 16)]);
      __syncthreads();
      a = smem_fft<+1>(a, b, lg2, cnt, tw, lg2);
      for (int e = threadIdx.x; e < cnt * N2; e += blockDim.x) A.Y2[TSF_CHK((r0 << lg2) + e, P.Nc, 17)] = a[e];
    } else {
      for (int e = threadIdx.x; e < cnt * N2; e += blockDim.x) Out[TSF_CHK((r0 << lg2) + e, P.Nc, 18)] = cscale(a[e], scale);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------------
// helpers on the level state
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ double source_at(const Args &A, int j, int i) {
  if (A.f_dense) return A.f_dense[TSF_CHK((long long)j * A.n + i, (long long)A.M * A.n, 19)];
  double s = 0.0;
  for (int r = 0; r < A.src_rank; ++r)
    s += A.src_t[TSF_CHK((long long)r * A.M + j, (long long)A.src_rank * A.M, 20)] *
         A.src_x[TSF_CHK((long long)r * A.n + i, (long long)A.src_rank * A.n, 21)];
  return s;
}

// eigenvalue of the level-j circulant preconditioner at n-frequency m (Eq. (3.7), diagonalised)
__device__ __forceinline__ double2 lambda_p(const Args &A, const LevelScalars &s, int m) {
  const double2 lw = A.LamW[TSF_CHK(m, A.n, 22)], lq = A.LamQ[TSF_CHK(m, A.n, 23)];
  // q*lq + kp*lw + km*conj(lw)
  const double re = s.q * lq.x + (s.kp + s.km) * lw.x;
  const double im = s.q * lq.y + (s.kp - s.km) * lw.y;
  return make_double2(s.eta - A.sigma * re, -A.sigma * im);
}

__device__ __forceinline__ void write_partials(const Args &A, const Smem &S, int rb, double (&acc)[3]) {
  block_sum<3>(acc, S.red);
  if (threadIdx.x == 0) {
    double *p = A.partials + ((size_t)rb * team().cnt + team().idx) * 4;
    p[0] = acc[0];
    p[1] = acc[1];
    p[2] = acc[2];
  }
}

// Sum of all CTAs' partials of buffer rb, identical in every CTA (fixed order).
__device__ __forceinline__ void read_partials(const Args &A, const Smem &S, int rb, double (&tot)[3]) {
  double v[3] = {0.0, 0.0, 0.0};
  const int cnt = team().cnt;
  for (int b = threadIdx.x; b < cnt; b += blockDim.x) {
    const double *p = A.partials + ((size_t)rb * cnt + b) * 4;
    v[0] += p[0];
    v[1] += p[1];
    v[2] += p[2];
  }
  block_sum<3>(v, S.red);
  tot[0] = v[0];
  tot[1] = v[1];
  tot[2] = v[2];
}

template <typename T>
__device__ __forceinline__ T ldp(const typename RealOf<T>::R *v, int m) { return reinterpret_cast<const T *>(v)[m]; }
template <typename T>
__device__ __forceinline__ void stp(typename RealOf<T>::R *v, int m, T z) { reinterpret_cast<T *>(v)[m] = z; }
__device__ __forceinline__ double2 ld2(const double *v, int m) { return reinterpret_cast<const double2 *>(v)[m]; }
__device__ __forceinline__ void st2(double *v, int m, double2 z) { reinterpret_cast<double2 *>(v)[m] = z; }

// ------------------------------------------------------------------------------------------------
// phases of the level symbols
// ------------------------------------------------------------------------------------------------

// Deterministic block min and max (fixed shuffle tree, fixed warp order); every thread gets both.
__device__ __forceinline__ void block_minmax(double &mn, double &mx, double *sm /* 64 doubles */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    sm[w] = mn;
    sm[32 + w] = mx;
  }
  __syncthreads();
  mn = sm[0];
  mx = sm[32];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
    mn = fmin(mn, sm[i]);
    mx = fmax(mx, sm[32 + i]);
  }
  __syncthreads();
}

// Bluestein, inverse n-point DFT of 1/Lambda_P (first column of P^{-1}), phase 1 of 3.  Also the
// smallest and largest |Lambda_P|^2 of this CTA's frequencies, into slot 3 of its partials records
// (buffer 0: min, buffer 1: max; the CGS reductions use slots 0-2 only).
static __device__ void ph_pinv_b1(const Args &A, const Smem &S, int j) {
  const LevelScalars s = level_scalars(A, j);
  const int n = A.n;
  double dmin = INFINITY, dmax = 0.0;
  col_pass<false, true, double2>(A, S, A.twL, A.bp.lg1, A.bp.lg2, 0, A.cap_bcol, nullptr, A.Y1,
                                 [&](int m, double2) -> double2 {
                                   if (m >= n) return make_double2(0.0, 0.0);
                                   const double2 lp = lambda_p(A, s, m);
                                   double d = lp.x * lp.x + lp.y * lp.y;
                                   if (A.inject == 3 && m == 0) d = 0.0;   // testing hook
                                   if (!(d > 0.0) || !isfinite(d)) {
                                     raise_fatal(A, kESingular);
                                     return make_double2(0.0, 0.0);
                                   }
                                   dmin = fmin(dmin, d);
                                   dmax = fmax(dmax, d);
                                   const double2 inv = make_double2(lp.x / d, -lp.y / d);
                                   return cmul(inv, A.chirpI[TSF_CHK(m, n, 24)]);
                                 });
  block_minmax(dmin, dmax, S.red);
  if (threadIdx.x == 0) {
    const int cnt = team().cnt, idx = team().idx;
    A.partials[((size_t)0 * cnt + idx) * 4 + 3] = dmin;
    A.partials[((size_t)1 * cnt + idx) * 4 + 3] = dmax;
  }
}
// Bluestein phase 2 of 3, after the check that P is numerically nonsingular: its eigenvalues
// must satisfy min |Lambda_P| > 1e3 u64 max |Lambda_P| (Theorem 4 proves nonsingularity only for
// beta above about 1.6168; below that the check stands in for it).
constexpr double kSingRel2 = (1e3 * 1.1102230246251565e-16) * (1e3 * 1.1102230246251565e-16);
static __device__ void ph_pinv_b2(const Args &A, const Smem &S) {
  if (team().idx == 0 && threadIdx.x == 0) {
    const int cnt = team().cnt;
    double mn = INFINITY, mx = 0.0;
    for (int b = 0; b < cnt; ++b) {
      mn = fmin(mn, A.partials[(size_t)b * 4 + 3]);
      mx = fmax(mx, A.partials[((size_t)cnt + b) * 4 + 3]);
    }
    if (!(mn > kSingRel2 * mx)) raise_fatal(A, kESingular);
  }
  crow_pass<0>(A, S, A.BhI, nullptr, 1.0);
}
static __device__ void ph_pinv_b3(const Args &A, const Smem &S) {
  const int n = A.n;
  col_pass<true, false, double2>(A, S, A.twL, A.bp.lg1, A.bp.lg2, 0, A.cap_bcol, A.Y2, nullptr,
                                 [&](int m, double2 z) -> double2 {
                                   if (m < n) A.cprime[TSF_CHK(m, n, 25)] = cmul(z, A.chirpI[TSF_CHK(m, n, 26)]).x;
                                   return z;
                                 });
}
// Toeplitz embedding of the circulant P^{-1} (entries t_d = c'_{d mod n}) and its column FFT.
static __device__ void ph_pinv_c1(const Args &A, const Smem &S) {
  const int n = A.n, L = A.cp.L;
  col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y1,
                                 [&](int m, double2) -> double2 {
                                   double v[2];
#pragma unroll
                                   for (int h = 0; h < 2; ++h) {
                                     const int i = 2 * m + h;
                                     // t_{-d} = c'_{n-d}
                                     v[h] = i < n ? A.cprime[TSF_CHK(i, n, 27)] : (i > L - n ? A.cprime[TSF_CHK(i + n - L, n, 28)] : 0.0);
                                   }
                                   return make_double2(v[0], v[1]);
                                 });
}
// Spectrum of P^{-1}'s embedding, plus A and B of level j.
static __device__ void ph_pinv_c2(const Args &A, const Smem &S, int j) {
  row_pass<1, double2>(A, S, A.twL, A.Y1, nullptr, nullptr, A.SP, 1.0 / (4.0 * (double)A.cp.N), j);
}
// A and B spectra only (no preconditioner).
static __device__ void ph_ab_only(const Args &A, const Smem &S, int j) {
  const LevelScalars s = level_scalars(A, j);
  const ConvPlan &P = A.cp;
  for (int sl = team_tid(); sl <= P.N; sl += team_threads()) {
    const int k = sl == P.N ? P.N : ((sl & (P.N2 - 1)) * P.N1 + (sl >> P.lg2));
    store_ab(A, s, sl, k, sl == P.N);
  }
}

// Symbols for level j (preconditioned or not).  Returns false if aborted.
static __device__ bool level_symbols(const Args &A, const Smem &S, int j) {
  if (A.precond != 2) {
    ph_pinv_b1(A, S, j);
    if (!grid_sync(A)) return false;
    ph_pinv_b2(A, S);
    if (!grid_sync(A)) return false;
    ph_pinv_b3(A, S);
    if (!grid_sync(A)) return false;
    ph_pinv_c1(A, S);
    if (!grid_sync(A)) return false;
    ph_pinv_c2(A, S, j);
  } else {
    ph_ab_only(A, S, j);
  }
  return grid_sync(A);
}

// Commit of level j-1 (when commit), history sum of Lemma 1 for level j into H, contiguous.
#ifndef TSFCDE_HIST_UNROLL
#define TSFCDE_HIST_UNROLL 16
#endif
constexpr int kHistUnroll = TSFCDE_HIST_UNROLL;

static __device__ void ph_history(const Args &A, int j, bool commit) {
  const int npair = (A.n + 1) >> 1;
  const long long st = A.ring_stride;
  const double2 *ring2 = reinterpret_cast<const double2 *>(A.ring);
  // fast history from the second block on: the far part (blocks before j's own) was formed by
  // ph_far_update; here the endpoint term s = 0 and the direct terms s in [qB, j)
  const bool fast = A.fh_B && j >= A.fh_B;
  const int s0 = fast ? (j >> A.fh_lgB) << A.fh_lgB : 0;
  const double2 *far2 = fast ? reinterpret_cast<const double2 *>(A.fh_far + (long long)(j - s0) * st) : nullptr;
  for (int t = team_tid(); t < npair; t += team_threads()) {
    double2 dlast = make_double2(0.0, 0.0);
    if (commit) {
      const double2 xv = reinterpret_cast<const double2 *>(A.x)[t];
      const double2 uv = reinterpret_cast<const double2 *>(A.u)[t];
      dlast = make_double2(xv.x - uv.x, xv.y - uv.y);
      reinterpret_cast<double2 *>(A.ring + (long long)(j - 1) * st)[t] = dlast;
      reinterpret_cast<double2 *>(A.u)[t] = xv;
    }
    double hx = 0.0, hy = 0.0;
    if (fast) {
      const double2 fv = far2[t];
      const double2 d0 = ring2[t];
      const double cl = A.hl[j];
      hx = fv.x + cl * d0.x;
      hy = fv.y + cl * d0.y;
      const int smax = commit ? j - 1 : j;
      for (int s = s0; s < smax; ++s) {
        const double2 d = ring2[TSF_CHK(s * (st >> 1) + t, (long long)A.M * (st >> 1), 29)];
        const double c = A.hc[j - s];
        hx += c * d.x;
        hy += c * d.y;
      }
      if (commit) {   // s = j-1 >= s0 >= B from registers
        const double c = A.hc[1];
        hx += c * dlast.x;
        hy += c * dlast.y;
      }
    } else if (j >= 1) {
      // s = 0 term: c^{(j)}_j = a_j - b_j; 1 <= s <= j-1: c^{(j)}_{j-s} = a + b - b (Lemma 1)
      const int smax = commit ? j - 1 : j;   // levels read from the ring
      int s = 0;
      // kHistUnroll ring rows in flight per thread (16-byte loads), summed in order of s
      for (; s + kHistUnroll <= smax; s += kHistUnroll) {
        double2 d[kHistUnroll];
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) d[u] = ring2[TSF_CHK((s + u) * (st >> 1) + t, (long long)A.M * (st >> 1), 30)];
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) {
          const double c = (s + u) == 0 ? A.hl[j] : A.hc[j - s - u];
          hx += c * d[u].x;
          hy += c * d[u].y;
        }
      }
      for (; s < smax; ++s) {
        const double2 d = ring2[TSF_CHK(s * (st >> 1) + t, (long long)A.M * (st >> 1), 31)];
        const double c = s == 0 ? A.hl[j] : A.hc[j - s];
        hx += c * d.x; hy += c * d.y;
      }
      if (commit) {   // s = j-1 from registers
        const double c = (j - 1) == 0 ? A.hl[j] : A.hc[1];
        hx += c * dlast.x; hy += c * dlast.y;
      }
    }
    reinterpret_cast<double2 *>(A.H)[t] = make_double2(hx, hy);
  }
}

// Final commit (end of a launch): d^j = x - u into the ring, u = x.
static __device__ void ph_commit(const Args &A, int j) {
  const int npair = (A.n + 1) >> 1;
  for (int t = team_tid(); t < npair; t += team_threads()) {
    const double2 xv = reinterpret_cast<const double2 *>(A.x)[t];
    const double2 uv = reinterpret_cast<const double2 *>(A.u)[t];
    reinterpret_cast<double2 *>(A.ring + (long long)j * A.ring_stride)[t] = make_double2(xv.x - uv.x, xv.y - uv.y);
    reinterpret_cast<double2 *>(A.u)[t] = xv;
  }
}

// ------------------------------------------------------------------------------------------------
// Fast history: the sum of Lemma 1 as a blocked convolution in time.
//   H^j = c^{(j)}_j d^0 + sum_{s=1}^{j-1} hc[j-s] d^s,   hc[m] = a_m + b_{m+1} - b_m  (Lemma 1)
// is, for s >= 1, a causal convolution of the increments with the kernel hc.  With blocks of B
// levels, level j = qB + r takes from the blocks p < q (increments s = pB + v, v < B, s >= 1)
//   Far_q[r] = sum_{p<q} sum_v hc[(q-p)B + r - v] d^{pB+v}.
// Per point and block p this is the 2B-point circular convolution of [d^{pB..pB+B-1}, 0] with the
// kernel window w_{q-p}[t] = hc[(q-p-1)B + t] (t < 2B; hc[0] taken as 0), read at output B + r:
// the window's other taps meet the zero half, so no wrap-around enters.  By the convolution
// theorem
//   Far_q[r] = IDFT_2B( sum_{p<q} DFT(w_{q-p}) . DFT([d_p, 0]) )[B + r],
// so each block's spectrum is computed once, when the block is complete, and each later block of
// levels costs one frequency-domain accumulation and one inverse transform per point instead of
// q B products.  ph_history adds the endpoint term and the direct terms s in [qB, j).
// Two points share one complex transform (real and imaginary parts), separated by the conjugate
// symmetry of the spectra of real sequences.  Tiles of 2 fh_lines consecutive points go to the
// team's CTAs; `transform` also computes and stores the spectrum of block q - 1.
// ------------------------------------------------------------------------------------------------
static __device__ void ph_far_update(const Args &A, const Smem &S, int q, bool transform) {
  const int B = A.fh_B, lgT = A.fh_lgB + 1, T2 = 2 * B;
  const int lines = A.fh_lines, P = 2 * lines;
  const long long st = A.ring_stride;
  const int ntiles = (A.n + P - 1) / P;
  const double2 *ring2 = reinterpret_cast<const double2 *>(A.ring);
  double2 *tw = static_cast<double2 *>(S.tw);
  int lo, hi;
  my_items(ntiles, lo, hi);
  if (lo < hi) load_line_twiddles<double2>(A, S, A.twL, lgT);
  for (int tile = lo; tile < hi; ++tile) {
    const int i0 = tile * P;   // even; i0 + P <= ring_stride (P divides 32, the stride's unit)
    double2 *a = static_cast<double2 *>(S.a), *b = static_cast<double2 *>(S.b);
    if (transform) {
      const int p = q - 1;
      // line l: z_t = d^{pB+t}_{i0+2l} + i d^{pB+t}_{i0+2l+1} for t < B (d^0 enters as 0), 0 after
      for (int e = threadIdx.x; e < lines * T2; e += blockDim.x) {
        const int l = e % lines, t = e / lines;
        const int s = p * B + t;
        double2 z = make_double2(0.0, 0.0);
        if (t < B && s >= 1) z = ring2[TSF_CHK((long long)s * (st >> 1) + (i0 >> 1) + l, (long long)A.M * (st >> 1), 32)];
        a[l * T2 + t] = z;
      }
      __syncthreads();
      double2 *y = smem_fft<-1>(a, b, lgT, lines, tw, lgT);
      for (int e = threadIdx.x; e < lines * (B + 1); e += blockDim.x) {
        const int l = e % lines, k = e / lines;
        const double2 zk = y[l * T2 + k], zm = cconj(y[l * T2 + ((T2 - k) & (T2 - 1))]);
        const double2 ea = cscale(cadd(zk, zm), 0.5);            // (Z_k + conj Z_{-k}) / 2
        const double2 eb = cscale(mul_mi(csub(zk, zm)), 0.5);    // (Z_k - conj Z_{-k}) / 2i
        double2 *E = A.fh_E + TSF_CHK((long long)(p * (B + 1) + k) * st + i0 + 2 * l,
                                      (long long)A.fh_nblk * (B + 1) * st - 1, 33);
        E[0] = ea;
        E[1] = eb;
      }
      __syncthreads();   // the block's spectrum (global) is read below by the same CTA
    }
    // Y_k = sum_{p<q} K_{q-p,k} (E_p,k(a) + i E_p,k(b)), then the Hermitian extension of both
    for (int e = threadIdx.x; e < lines * (B + 1); e += blockDim.x) {
      const int l = e % lines, k = e / lines;
      double2 sa = make_double2(0.0, 0.0), sb = make_double2(0.0, 0.0);
      for (int p = 0; p < q; ++p) {
        const double2 K = A.fh_K[TSF_CHK((long long)(q - p - 1) * (B + 1) + k, (long long)A.fh_nblk * (B + 1), 34)];
        const double2 *E = A.fh_E + TSF_CHK((long long)(p * (B + 1) + k) * st + i0 + 2 * l,
                                            (long long)A.fh_nblk * (B + 1) * st - 1, 35);
        const double2 ea = E[0], eb = E[1];
        sa = cadd(sa, cmul(K, ea));
        sb = cadd(sb, cmul(K, eb));
      }
      a[l * T2 + k] = make_double2(sa.x - sb.y, sa.y + sb.x);
      if (k > 0 && k < B) a[l * T2 + T2 - k] = make_double2(sa.x + sb.y, sb.x - sa.y);
    }
    __syncthreads();
    double2 *y = smem_fft<+1>(a, b, lgT, lines, tw, lgT);   // window spectra carry 1/(2B)
    for (int e = threadIdx.x; e < lines * B; e += blockDim.x) {
      const int l = e % lines, r = e / lines;
      reinterpret_cast<double2 *>(A.fh_far)[TSF_CHK(((long long)r * st + i0) / 2 + l, (long long)B * st / 2, 36)] = y[l * T2 + B + r];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------------
// Preconditioned CGS (Section 4; Barrett et al. "Templates" form) on A d = b in element type T,
// from the current iterate x with r = b - A x, r~ = u = p = r already stored, rho = (r~, r).
// The forward column transform of p is already in Y1 when fwd_done.  Stops when
// ||r_k|| < tol * nref (nref = ||r_0|| for a plain solve) or after maxit iterations.
// Returns the status; `its` and `rel` (= ||r_k|| / nref) are set; `alive` is false if the
// kernel must stop.  Every CTA takes the same decisions (identical reduced scalars).  Dot
// products accumulate per thread in T's precision and are reduced across the grid in FP64.
// ------------------------------------------------------------------------------------------------
template <typename T>
struct Krylov {
  typename RealOf<T>::R *x, *r, *rt, *p, *q, *uu, *vh;
  typename RealOf<T>::R *xb;   // minimum-residual iterate (kept when non-null)
  const T *SA, *SP;
  T *Y1, *Y2;
  const T *twG;
};

template <typename T>
__device__ int cgs_solve(const Args &A, const Smem &S, const Krylov<T> &V, double rho, double nref,
                         double tol, int maxit, bool fwd_done, int &rb, int &its, double &rel,
                         bool &alive) {
  using R = typename RealOf<T>::R;
  const int n = A.n;
  const bool pc = A.precond != 2;
  its = 0;
  rel = 0.0;
  alive = true;
  if (!(nref > 0.0)) return kOK;
  // the start x0 (zero when fwd_done) is the first candidate for the minimum-residual iterate
  bool have = false;       // xb holds a saved iterate (else the best is x0 = 0)
  if (!fwd_done) {
    const bool keep0 = V.xb != nullptr;
    col_pass<false, true, T>(A, S, V.twG, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, V.Y1,
                             [&](int m, T) -> T {
                               if (keep0) stp<T>(V.xb, m, ldp<T>(V.x, m));
                               return ldp<T>(V.p, m);
                             });
    have = keep0;
    if (!(alive = grid_sync(A))) return kOK;
  }
  double tot[3];
  bool first = true;
  double beta = 0.0;
  double best = sqrt(rho) / nref;   // ||r_0|| / nref (r~ = r at the start, so rho = ||r_0||^2)
  bool save = false;       // the iterate after the last iteration is the best so far
  while (true) {
    ++its;
    if (!first) {
      const R bt = (R)beta;
      const bool keep = save && V.xb != nullptr;
      have = have || keep;
      // u = r + beta q; p = u + beta (q + beta p); forward transform of p; keep the best x
      col_pass<false, true, T>(A, S, V.twG, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, V.Y1,
                               [&](int m, T) -> T {
                                 if (keep) stp<T>(V.xb, m, ldp<T>(V.x, m));
                                 const T rv = ldp<T>(V.r, m), qv = ldp<T>(V.q, m), pv = ldp<T>(V.p, m);
                                 T uv, pn;
                                 mkc(uv, rv.x + bt * qv.x, rv.y + bt * qv.y);
                                 mkc(pn, uv.x + bt * (qv.x + bt * pv.x), uv.y + bt * (qv.y + bt * pv.y));
                                 stp<T>(V.uu, m, uv);
                                 stp<T>(V.p, m, pn);
                                 return pn;
                               });
      if (!(alive = grid_sync(A))) return kOK;
    }
    first = false;
    if (pc) {   // p^ = P^{-1} p
      row_pass<0, T>(A, S, V.twG, V.Y1, V.Y2, V.SP, nullptr, 0.0, -1);
      if (!(alive = grid_sync(A))) return kOK;
      col_pass<true, true, T>(A, S, V.twG, A.cp.lg1, A.cp.lg2, 1, A.cap_col, V.Y2, V.Y1,
                              [&](int m, T z) -> T {
                                if (2 * m >= n) z.x = (R)0;
                                if (2 * m + 1 >= n) z.y = (R)0;
                                return z;
                              });
      if (!(alive = grid_sync(A))) return kOK;
    }
    // v^ = A p^, sigma = (r~, v^)
    row_pass<0, T>(A, S, V.twG, V.Y1, V.Y2, V.SA, nullptr, 0.0, -1);
    if (!(alive = grid_sync(A))) return kOK;
    {
      R a0 = (R)0;
      col_pass<true, false, T>(A, S, V.twG, A.cp.lg1, A.cp.lg2, 1, A.cap_col, V.Y2, nullptr,
                               [&](int m, T z) -> T {
                                 if (2 * m >= n) z.x = (R)0;
                                 if (2 * m + 1 >= n) z.y = (R)0;
                                 stp<T>(V.vh, m, z);
                                 const T rtv = ldp<T>(V.rt, m);
                                 a0 += rtv.x * z.x + rtv.y * z.y;
                                 return z;
                               });
      double acc[3] = {(double)a0, 0.0, 0.0};
      write_partials(A, S, rb, acc);
    }
    if (!(alive = grid_sync(A))) return kOK;
    read_partials(A, S, rb, tot);
    rb ^= 1;
    const double sig = A.inject == 2 ? 0.0 : tot[0];   // testing hook: (r~, v^) = 0
    if (sig == 0.0) return kEBreakdown;
    if (!(sig == sig) || isinf(sig)) return kENonFinite;
    const R alpha = (R)(rho / sig);
    // q = u - alpha v^; w = u + q; forward transform of w (x += alpha w when unpreconditioned)
    col_pass<false, true, T>(A, S, V.twG, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, V.Y1,
                             [&](int m, T) -> T {
                               const T uv = ldp<T>(V.uu, m), vv = ldp<T>(V.vh, m);
                               T qv, wv;
                               mkc(qv, uv.x - alpha * vv.x, uv.y - alpha * vv.y);
                               mkc(wv, uv.x + qv.x, uv.y + qv.y);
                               stp<T>(V.q, m, qv);
                               if (!pc) {
                                 const T xv = ldp<T>(V.x, m);
                                 T xn;
                                 mkc(xn, xv.x + alpha * wv.x, xv.y + alpha * wv.y);
                                 stp<T>(V.x, m, xn);
                               }
                               return wv;
                             });
    if (!(alive = grid_sync(A))) return kOK;
    if (pc) {   // u^ = P^{-1} w; x += alpha u^
      row_pass<0, T>(A, S, V.twG, V.Y1, V.Y2, V.SP, nullptr, 0.0, -1);
      if (!(alive = grid_sync(A))) return kOK;
      col_pass<true, true, T>(A, S, V.twG, A.cp.lg1, A.cp.lg2, 1, A.cap_col, V.Y2, V.Y1,
                              [&](int m, T z) -> T {
                                if (2 * m >= n) z.x = (R)0;
                                if (2 * m + 1 >= n) z.y = (R)0;
                                const T xv = ldp<T>(V.x, m);
                                T xn;
                                mkc(xn, xv.x + alpha * z.x, xv.y + alpha * z.y);
                                stp<T>(V.x, m, xn);
                                return z;
                              });
      if (!(alive = grid_sync(A))) return kOK;
    }
    // r -= alpha A u^; rho' = (r~, r), ||r||^2
    row_pass<0, T>(A, S, V.twG, V.Y1, V.Y2, V.SA, nullptr, 0.0, -1);
    if (!(alive = grid_sync(A))) return kOK;
    {
      R a0 = (R)0, a1 = (R)0;
      col_pass<true, false, T>(A, S, V.twG, A.cp.lg1, A.cp.lg2, 1, A.cap_col, V.Y2, nullptr,
                               [&](int m, T z) -> T {
                                 if (2 * m >= n) z.x = (R)0;
                                 if (2 * m + 1 >= n) z.y = (R)0;
                                 const T rv = ldp<T>(V.r, m), rtv = ldp<T>(V.rt, m);
                                 T rn;
                                 mkc(rn, rv.x - alpha * z.x, rv.y - alpha * z.y);
                                 stp<T>(V.r, m, rn);
                                 a0 += rtv.x * rn.x + rtv.y * rn.y;
                                 a1 += rn.x * rn.x + rn.y * rn.y;
                                 return z;
                               });
      double acc[3] = {(double)a0, (double)a1, 0.0};
      write_partials(A, S, rb, acc);
    }
    if (!(alive = grid_sync(A))) return kOK;
    read_partials(A, S, rb, tot);
    rb ^= 1;
    rel = sqrt(tot[1]) / nref;
    if (!(rel == rel) || isinf(rel)) return kENonFinite;
    if (rel < tol) return kOK;
    save = rel < best;
    if (save) best = rel;
    if (its >= maxit) {
      // like MATLAB's cgs: a solve that does not converge returns its minimum-residual iterate
      // (the saved one, or the zero start when nothing improved on it)
      if (V.xb != nullptr && !save) {
        const bool from_xb = have;
        col_pass<false, false, T>(A, S, V.twG, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, nullptr,
                                  [&](int m, T z) -> T {
                                    T v;
                                    if (from_xb) {
                                      v = ldp<T>(V.xb, m);
                                    } else {
                                      mkc(v, (R)0, (R)0);
                                    }
                                    stp<T>(V.x, m, v);
                                    return z;
                                  });
        if (!(alive = grid_sync(A))) return kOK;
        rel = best;
      }
      return kENotConverged;
    }
    if (tot[0] == 0.0) return kEBreakdown;
    beta = tot[0] / rho;
    rho = tot[0];
  }
}

// ------------------------------------------------------------------------------------------------
// Constant coefficients: the Gohberg-Semencul formula (Section 3.1, Eq. (3.6))
//   A^{-1} = (L_p R_p - L0_p R0_p) / xi_0,  x = A^{-1} e_1 = (xi_k), y = A^{-1} e_n = (eta_k),
//   L_p  lower triangular Toeplitz, first column x;   R_p  upper, first row (eta_{n-1}, ..., eta_0);
//   L0_p strictly lower, first column (0, eta_0, ..., eta_{n-2});
//   R0_p strictly upper, first row (0, xi_{n-1}, ..., xi_1).
// Each factor is a Toeplitz product through the same L-point circulant embedding as A and B.
// ------------------------------------------------------------------------------------------------

// Spectra of the four factors from gx, gy (4 phases).  1/xi_0 is folded into L_p and L0_p.
// Returns false when the kernel must stop; sets `st` to E_BREAKDOWN when xi_0 is 0 or not finite.
static __device__ bool gsf_spectra(const Args &A, const Smem &S, int &st) {
  const int n = A.n, L = A.cp.L;
  const double *gx = A.gx, *gy = A.gy;
  const double sc = 1.0 / (4.0 * (double)A.cp.N);
  // L_p: t_d = xi_d (0 <= d < n); R_p: t_0 = eta_{n-1}, t_{-d} = eta_{n-1-d} at index L - d
  col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y1,
                                 [&](int m, double2) -> double2 {
                                   double v[2];
#pragma unroll
                                   for (int h = 0; h < 2; ++h) {
                                     const int i = 2 * m + h;
                                     v[h] = i < n ? gx[i] : 0.0;
                                   }
                                   return make_double2(v[0], v[1]);
                                 });
  col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y2,
                                 [&](int m, double2) -> double2 {
                                   double v[2];
#pragma unroll
                                   for (int h = 0; h < 2; ++h) {
                                     const int i = 2 * m + h;
                                     v[h] = i == 0 ? gy[n - 1] : (i > L - n ? gy[i + n - 1 - L] : 0.0);
                                   }
                                   return make_double2(v[0], v[1]);
                                 });
  if (!grid_sync(A)) return false;
  const double xi0 = gx[0];
  if (xi0 == 0.0 || !(xi0 == xi0) || isinf(xi0)) {
    st = kEBreakdown;
    return true;
  }
  row_pass<1, double2>(A, S, A.twL, A.Y1, nullptr, nullptr, A.SL, sc / xi0, -1);
  row_pass<1, double2>(A, S, A.twL, A.Y2, nullptr, nullptr, A.SR, sc, -1);
  if (!grid_sync(A)) return false;
  // L0_p: t_d = eta_{d-1} (1 <= d < n); R0_p: t_{-d} = xi_{n-d} at index L - d (1 <= d < n)
  col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y1,
                                 [&](int m, double2) -> double2 {
                                   double v[2];
#pragma unroll
                                   for (int h = 0; h < 2; ++h) {
                                     const int i = 2 * m + h;
                                     v[h] = (i >= 1 && i < n) ? gy[i - 1] : 0.0;
                                   }
                                   return make_double2(v[0], v[1]);
                                 });
  col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y2,
                                 [&](int m, double2) -> double2 {
                                   double v[2];
#pragma unroll
                                   for (int h = 0; h < 2; ++h) {
                                     const int i = 2 * m + h;
                                     v[h] = i > L - n ? gx[i + n - L] : 0.0;
                                   }
                                   return make_double2(v[0], v[1]);
                                 });
  if (!grid_sync(A)) return false;
  row_pass<1, double2>(A, S, A.twL, A.Y1, nullptr, nullptr, A.SL0, sc / xi0, -1);
  row_pass<1, double2>(A, S, A.twL, A.Y2, nullptr, nullptr, A.SR0, sc, -1);
  return grid_sync(A);
}

// z = A^{-1} v by Algorithm "Compute z = A^{-1} v", from the forward column transform of v in Y1
// (4 phases): z2 = R_p v and z1 = R0_p v share that transform; z4 = L_p z2 and z3 = L0_p z1;
// z = z4 - z3 is formed in the last inverse column pass, whose body(m, z) sees z (zero beyond n)
// and returns the next forward input (stored to Y1 when FWD).
template <bool FWD, class Body>
__device__ bool gsf_apply(const Args &A, const Smem &S, Body body) {
  const int n = A.n;
  auto trunc = [n](int m, double2 z) -> double2 {
    if (2 * m >= n) z.x = 0.0;
    if (2 * m + 1 >= n) z.y = 0.0;
    return z;
  };
  row_pass<0, double2>(A, S, A.twL, A.Y1, A.Y2, A.SR, nullptr, 0.0, -1);
  row_pass<0, double2>(A, S, A.twL, A.Y1, A.Y3, A.SR0, nullptr, 0.0, -1);
  if (!grid_sync(A)) return false;
  col_pass<true, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, A.Y2, A.Y2, trunc);
  col_pass<true, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, A.Y3, A.Y3, trunc);
  if (!grid_sync(A)) return false;
  row_pass<0, double2>(A, S, A.twL, A.Y2, A.Y2, A.SL, nullptr, 0.0, -1);
  row_pass<0, double2>(A, S, A.twL, A.Y3, A.Y3, A.SL0, nullptr, 0.0, -1);
  if (!grid_sync(A)) return false;
  col_pass<true, FWD, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, A.Y2, A.Y1,
                               [&](int m, double2 z) -> double2 { return body(m, trunc(m, z)); },
                               A.Y3);
  return grid_sync(A);
}

// Residual r = b - A v with the level spectrum S_A, from the forward column transform of v in Y1
// (2 phases); b(m) gives the right-hand side pair; the forward column transform of r goes to Y1
// and ||r||^2 is returned in tot[0].
template <class RHS>
__device__ bool residual_pass(const Args &A, const Smem &S, int &rb, RHS b, double (&tot)[3]) {
  const int n = A.n;
  row_pass<0, double2>(A, S, A.twL, A.Y1, A.Y2, A.SA, nullptr, 0.0, -1);
  if (!grid_sync(A)) return false;
  double acc[3] = {0.0, 0.0, 0.0};
  col_pass<true, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, A.Y2, A.Y1,
                                [&](int m, double2 z) -> double2 {
                                  const double2 bv = b(m);
                                  double2 rv = make_double2(bv.x - z.x, bv.y - z.y);
                                  if (2 * m >= n) rv.x = 0.0;
                                  if (2 * m + 1 >= n) rv.y = 0.0;
                                  acc[0] += rv.x * rv.x + rv.y * rv.y;
                                  return rv;
                                });
  write_partials(A, S, rb, acc);
  if (!grid_sync(A)) return false;
  read_partials(A, S, rb, tot);
  rb ^= 1;
  return true;
}

// Generators of the constant level matrix A (level symbols of j >= 1 in S_A, S_P): the systems
// A x = e_1 and A y = e_n of Eq. (3.5) by the preconditioned CGS, the factor spectra, one
// refinement of each generator with the inverse they define (x += A^{-1}(e_1 - A x)), and the
// spectra again.  Returns the status; `its` counts the CGS iterations.
static __device__ int gsf_build(const Args &A, const Smem &S, const Krylov<double2> &V64, int &rb, int &its,
                         bool &alive) {
  const int n = A.n, L = A.cp.L;
  its = 0;
  alive = true;
  for (int g = 0; g < 2; ++g) {
    const int hot = g == 0 ? 0 : n - 1;
    for (int i = team_tid(); i < L; i += team_threads()) {
      const double e = i == hot ? 1.0 : 0.0;
      A.x[i] = 0.0;
      A.r[i] = e;
      A.rt[i] = e;
      A.uu[i] = e;
      A.p[i] = e;
    }
    if (!(alive = grid_sync(A))) return kOK;
    int it = 0;
    double rel = 0.0;
    const int st = cgs_solve<double2>(A, S, V64, 1.0, 1.0, A.tol, A.maxit, false, rb, it, rel, alive);
    if (!alive) return kOK;
    its += it;
    if (st != kOK && st != kENotConverged) return st;
    double *dst = g == 0 ? A.gx : A.gy;
    for (int i = team_tid(); i < L; i += team_threads()) dst[i] = i < n ? A.x[i] : 0.0;
    if (!(alive = grid_sync(A))) return kOK;
  }
  int st = kOK;
  if (!(alive = gsf_spectra(A, S, st))) return kOK;
  if (st != kOK) return st;
  for (int g = 0; g < 2; ++g) {
    double *gv = g == 0 ? A.gx : A.gy;
    const int hot = g == 0 ? 0 : n - 1;
    col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y1,
                                   [&](int m, double2) -> double2 { return ld2(gv, m); });
    if (!(alive = grid_sync(A))) return kOK;
    double tot[3];
    if (!(alive = residual_pass(A, S, rb,
                                [&](int m) -> double2 {
                                  return make_double2(2 * m == hot ? 1.0 : 0.0, 2 * m + 1 == hot ? 1.0 : 0.0);
                                },
                                tot)))
      return kOK;
    if (!(alive = gsf_apply<false>(A, S, [&](int m, double2 z) -> double2 {
          const double2 v = ld2(gv, m);
          st2(gv, m, make_double2(v.x + z.x, v.y + z.y));
          return z;
        })))
      return kOK;
  }
  if (!(alive = gsf_spectra(A, S, st))) return kOK;
  return st;
}

// ------------------------------------------------------------------------------------------------
// the level kernel
// ------------------------------------------------------------------------------------------------
// Start of an inner solve on A d = r: d = 0, r = r~ = u = p = r rounded to the inner type;
// returns this element pair's contribution to (r, r) in the inner type.
__device__ __forceinline__ double inner_start(const Args &A, bool useff, int m, double2 rv) {
  if (useff) {
    const ffc r = to_ffc(rv);
    ffc z;
    z.x = ff(0.0);
    z.y = ff(0.0);
    stp<ffc>(A.xff, m, z);
    stp<ffc>(A.rff, m, r);
    stp<ffc>(A.rtff, m, r);
    stp<ffc>(A.uuff, m, r);
    stp<ffc>(A.pff, m, r);
    return (double)(r.x * r.x + r.y * r.y);
  }
  const float2 r32 = to_f2(rv);
  stp<float2>(A.x32, m, make_float2(0.f, 0.f));
  stp<float2>(A.r32, m, r32);
  stp<float2>(A.rt32, m, r32);
  stp<float2>(A.uu32, m, r32);
  stp<float2>(A.p32, m, r32);
  return (double)(r32.x * r32.x + r32.y * r32.y);
}
__device__ __forceinline__ double2 inner_solution(const Args &A, bool useff, int m) {
  if (useff) {
    const ffc d = ldp<ffc>(A.xff, m);
    return make_double2((double)d.x, (double)d.y);
  }
  const float2 d = ldp<float2>(A.x32, m);
  return make_double2((double)d.x, (double)d.y);
}

// March levels [j0, j1) of one instance with the current team (whole grid or one CTA).
static __device__ void march_body(const Args &A, const Smem &S, int j0, int j1) {
  const int n = A.n;
  const bool mixed = A.precision == kMixed;
  int rb = 0;
  // the vector sets of the three CGS precisions, CTA-uniform, kept in shared memory (passed by
  // reference, they would otherwise be per-thread local copies)
  __shared__ Krylov<double2> V64;
  __shared__ Krylov<float2> V32;
  __shared__ Krylov<ffc> VF;
  __syncthreads();
  if (threadIdx.x == 0) {
    V64.x = A.x; V64.r = A.r; V64.rt = A.rt; V64.p = A.p; V64.q = A.q; V64.uu = A.uu; V64.vh = A.vh;
    V64.xb = A.xb;
    V64.SA = A.SA; V64.SP = A.SP; V64.Y1 = A.Y1; V64.Y2 = A.Y2; V64.twG = A.twL;
    V32.x = A.x32; V32.r = A.r32; V32.rt = A.rt32; V32.p = A.p32; V32.q = A.q32; V32.uu = A.uu32;
    V32.xb = A.x32b;
    V32.vh = A.vh32; V32.SA = A.SA32; V32.SP = A.SP32; V32.Y1 = A.Y1f; V32.Y2 = A.Y2f; V32.twG = A.twL32;
    VF.x = A.xff; VF.r = A.rff; VF.rt = A.rtff; VF.p = A.pff; VF.q = A.qff; VF.uu = A.uuff;
    VF.xb = A.xffb;
    VF.vh = A.vhff; VF.SA = A.SAff; VF.SP = A.SPff; VF.Y1 = A.Y1ff; VF.Y2 = A.Y2ff; VF.twG = A.twLff;
  }
  __syncthreads();

  for (int j = j0; j < j1; ++j) {
    if (j == j0 || A.lv_newsym[j]) {
      if (!level_symbols(A, S, j)) return;
    }
    const bool useff = mixed && A.lv_inner[j] != 0;
    // constant coefficients: levels j >= 1 share A, applied as A^{-1} by the Gohberg-Semencul formula
    const bool gsf = A.gsf && j >= 1;
    bool commit = j > j0;
    int gen_its = 0;
    if (gsf && j == 1) {
      // the generator solves reuse the Krylov vectors: commit u^1 first
      if (commit) {
        ph_commit(A, 0);
        if (!grid_sync(A)) return;
        commit = false;
      }
      bool alive = true;
      const int gst = gsf_build(A, S, V64, rb, gen_its, alive);
      if (!alive) return;
      if (gst != kOK) {
        if (team().idx == 0 && threadIdx.x == 0) {
          A.iters[j] = gen_its;
          atomicCAS(A.status, 0, gst);
          atomicExch(A.status + 1, 1);
        }
        return;   // consistent in every CTA
      }
    }
    // ---- fast history: at a block start the new block's spectrum and the block's far part; at
    //      the first level of a launch the far part of its block ----
    if (A.fh_B && j >= A.fh_B) {
      const bool start = (j & (A.fh_B - 1)) == 0;
      if (start || j == j0) {
        if (commit) {   // the block's last increment must be in the ring before its transform
          ph_commit(A, j - 1);
          if (!grid_sync(A)) return;
          commit = false;
        }
        ph_far_update(A, S, j >> A.fh_lgB, start);
        if (!grid_sync(A)) return;
      }
    }
    // ---- RHS: g = B u^j - hscale * H^j + f^{j+sigma} (Eq. (3.1)) ----
    ph_history(A, j, commit);
    {
      const double *src = commit ? A.x : A.u;
      col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y1,
                                     [&](int m, double2) -> double2 { return ld2(src, m); });
    }
    if (!grid_sync(A)) return;
    row_pass<0, double2>(A, S, A.twL, A.Y1, A.Y2, A.SB, nullptr, 0.0, -1);
    if (!grid_sync(A)) return;
    double acc[3] = {0.0, 0.0, 0.0};
    // plain: x = 0, r = r~ = u = p = g and the forward transform of p fused here;
    // mixed: g kept in FP64, x = 0, r = g, and the FP32 inner start r32 = r~32 = u32 = p32 = g
    col_pass<true, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, A.Y2, A.Y1,
                                  [&](int m, double2 y) -> double2 {
                                    double gv[2] = {y.x, y.y};
                                    const double2 hv = ld2(A.H, m);
                                    const double hh[2] = {hv.x, hv.y};
#pragma unroll
                                    for (int h = 0; h < 2; ++h) {
                                      const int i = 2 * m + h;
                                      if (i < n) {
                                        gv[h] = gv[h] - A.hscale * hh[h] + source_at(A, j, i);
                                        acc[0] += gv[h] * gv[h];
                                      } else {
                                        gv[h] = 0.0;
                                      }
                                    }
                                    const double2 g = make_double2(gv[0], gv[1]);
                                    if (gsf) {   // g kept for the residual; its transform goes on to A^{-1}
                                      st2(A.rt, m, g);
                                      return g;
                                    }
                                    st2(A.x, m, make_double2(0.0, 0.0));
                                    st2(A.r, m, g);
                                    if (mixed) {
                                      st2(A.g, m, g);
                                      acc[1] += inner_start(A, useff, m, g);
                                    } else {
                                      st2(A.rt, m, g);
                                      st2(A.uu, m, g);
                                      st2(A.p, m, g);
                                    }
                                    return g;
                                  });
    write_partials(A, S, rb, acc);
    if (!grid_sync(A)) return;
    double tot[3];
    read_partials(A, S, rb, tot);
    rb ^= 1;
    const double gnorm = sqrt(tot[0]);
    int lstat = kOK, its = 0, outer = 0, esc = 0;
    double rel = 0.0;
    bool alive = true;
    if (!(gnorm == gnorm) || isinf(gnorm)) {
      lstat = kENonFinite;
    } else if (gsf) {
      // u^{j+1} = A^{-1} g (Algorithm "Compute z = A^{-1} v"), the FP64 residual, and at most two
      // refinements u += A^{-1}(g - A u) while it is above both tol and the FP64 floor
      its = gen_its;
      if (!gsf_apply<true>(A, S, [&](int m, double2 z) -> double2 {
            st2(A.x, m, z);
            return z;
          }))
        return;
      outer = 1;
      double prev = 0.0;
      while (true) {
        if (!residual_pass(A, S, rb, [&](int m) -> double2 { return ld2(A.rt, m); }, tot)) return;
        rel = gnorm > 0.0 ? sqrt(tot[0]) / gnorm : 0.0;
        if (!(rel == rel) || isinf(rel)) { lstat = kENonFinite; break; }
        if (rel < A.tol) break;
        if (rel < A.lv_floor[j]) {   // accepted at the FP64 residual floor, above tol
          esc = 2;
          break;
        }
        if (outer >= 3 || (outer > 1 && rel > 0.5 * prev)) { lstat = kENotConverged; break; }
        prev = rel;
        if (!gsf_apply<true>(A, S, [&](int m, double2 z) -> double2 {
              const double2 xv = ld2(A.x, m);
              const double2 xn = make_double2(xv.x + z.x, xv.y + z.y);
              st2(A.x, m, xn);
              return xn;
            }))
          return;
        ++outer;
      }
    } else if (!mixed) {
      lstat = cgs_solve<double2>(A, S, V64, tot[0], gnorm, A.tol, A.maxit, true, rb, its, rel, alive);
      if (!alive) return;
    } else if (gnorm > 0.0) {
      // iterative refinement: FP32 CGS on A d = r, x += d and r = g - A x in FP64
      double rho32 = tot[1];
      double prev = 1.0;
      while (true) {
        int ii = 0;
        double irel = 0.0;
        const int ist = useff ? cgs_solve<ffc>(A, S, VF, rho32, sqrt(rho32), A.inner_tol, A.inner_maxit,
                                                false, rb, ii, irel, alive)
                              : cgs_solve<float2>(A, S, V32, rho32, sqrt(rho32), A.inner_tol,
                                                  A.inner_maxit, false, rb, ii, irel, alive);
        if (!alive) return;
        its += ii;
        ++outer;
        const bool inner_ok = ist == kOK || ist == kENotConverged;
        // x += d (FP64); forward transform of x
        col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y1,
                                       [&](int m, double2) -> double2 {
                                         double2 xv = ld2(A.x, m);
                                         if (inner_ok) {
                                           const double2 dv = inner_solution(A, useff, m);
                                           xv = make_double2(xv.x + dv.x, xv.y + dv.y);
                                           st2(A.x, m, xv);
                                         }
                                         return xv;
                                       });
        if (!grid_sync(A)) return;
        row_pass<0, double2>(A, S, A.twL, A.Y1, A.Y2, A.SA, nullptr, 0.0, -1);
        if (!grid_sync(A)) return;
        // r = g - A x (FP64); restart values for the next inner solve (FP32) or the FP64 CGS
        acc[0] = acc[1] = acc[2] = 0.0;
        col_pass<true, false, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, A.Y2, nullptr,
                                       [&](int m, double2 z) -> double2 {
                                         const double2 gv = ld2(A.g, m);
                                         double2 rv = make_double2(gv.x - z.x, gv.y - z.y);
                                         if (2 * m >= n) rv.x = 0.0;
                                         if (2 * m + 1 >= n) rv.y = 0.0;
                                         acc[0] += rv.x * rv.x + rv.y * rv.y;
                                         st2(A.r, m, rv);
                                         st2(A.rt, m, rv);
                                         st2(A.uu, m, rv);
                                         st2(A.p, m, rv);
                                         acc[1] += inner_start(A, useff, m, rv);
                                         return z;
                                       });
        write_partials(A, S, rb, acc);
        if (!grid_sync(A)) return;
        read_partials(A, S, rb, tot);
        rb ^= 1;
        rel = sqrt(tot[0]) / gnorm;
        rho32 = tot[1];
        if (!(rel == rel) || isinf(rel)) { lstat = kENonFinite; break; }
        if (rel < A.tol) break;
        // stagnation at the FP64 residual floor (about u64 * kappa_eff) is convergence
        if (inner_ok && rel > 0.5 * prev && rel < A.lv_floor[j]) {
          esc = 2;
          break;
        }
        // no progress (or diverging) in the inner precision -> finish with the FP64 CGS from x
        if (!inner_ok || rel > 0.5 * prev || outer >= A.outer_maxit) {
          esc = 1;
          int i64 = 0;
          lstat = cgs_solve<double2>(A, S, V64, tot[0], gnorm, A.tol, A.maxit, false, rb, i64, rel, alive);
          if (!alive) return;
          its += i64;
          break;
        }
        prev = rel;
      }
    }
    if (team().idx == 0 && threadIdx.x == 0) {
      A.iters[j] = its;
      A.resid[j] = rel;
      // escalated[j] holds flags: bit 0 finished by the FP64 CGS, bit 1 accepted at the floor
      if (gsf) {
        A.outer_iters[j] = outer;
        A.escalated[j] = esc;
      } else if (mixed) {
        A.outer_iters[j] = outer;
        A.escalated[j] = esc;
      }
      if (lstat != kOK) {
        atomicCAS(A.status, 0, lstat);
        if (lstat != kENotConverged) atomicExch(A.status + 1, 1);
      }
    }
    if (lstat != kOK && lstat != kENotConverged) return;   // consistent in every CTA
  }
  if (!grid_sync(A)) return;
  ph_commit(A, j1 - 1);
}

// Every kernel of the library copies its Args parameter once into shared memory: the device
// functions take it by reference, and a reference to the parameter itself would give every thread
// a private local-memory copy (~0.9 KB per thread, more than L1 holds for a CTA).  The whole-grid
// march, instantiated for 256 threads (level_kernels.cu) and 512 threads (level_wide.cu):
template <int NT>
__global__ void __launch_bounds__(NT, 1) level_kernel(Args Ap, int j0, int j1) {
  __shared__ Args A;
  if (threadIdx.x == 0) A = Ap;
  __syncthreads();
  const Smem S = smem_view(lp_max_of(A), tw_max_of(A));
  grid_sync_init();
  march_body(A, S, j0, j1);
}

// ------------------------------------------------------------------------------------------------
// setup: tables, spectrum of W's embedding, Bluestein kernels, eigenvalues of s(W), s(Q)
// ------------------------------------------------------------------------------------------------
struct SetupArgs {
  const double *omega;   // WSGD weights omega_0..omega_{n+1}
  double2 *What, *LamW, *LamQ, *BhI, *BhF, *chirpI, *twL;
  int precond;
};

// Entry t_d of the Toeplitz matrix (0: W_beta, 1: Q), d in (-n, n).
__device__ __forceinline__ double toe_entry(const double *omega, int which, int d) {
  if (which == 0) return d >= -1 ? omega[d + 1] : 0.0;
  return d == 1 ? -1.0 : (d == -1 ? 1.0 : 0.0);
}
// First column of the circulant approximation (Strang: central diagonals; T. Chan: optimal).
__device__ __forceinline__ double circ_col(const double *omega, int which, int kind, int n, int k) {
  if (k == 0) return toe_entry(omega, which, 0);
  if (kind == 1) return ((double)(n - k) * toe_entry(omega, which, k) + (double)k * toe_entry(omega, which, k - n)) / (double)n;
  return k <= n / 2 ? toe_entry(omega, which, k) : toe_entry(omega, which, k - n);
}

// Per-instance tables and spectra with the current team.
static __device__ void setup_body(const Args &A, const SetupArgs &T, const Smem &S) {
  const int n = A.n, L = A.cp.L;
  const int gt = team_tid(), gs = team_threads();
  // tables: twiddles e^{-2 pi i k/L} (and their FP32 copy), chirp e^{i pi (k^2 mod 2n)/n}
  for (int k = gt; k < L; k += gs) {
    double s, c;
    sincospi(-2.0 * (double)k / (double)L, &s, &c);
    T.twL[k] = make_double2(c, s);
    if (A.precision == kMixed) {
      A.twL32[k] = make_float2((float)c, (float)s);
      A.twLff[k] = to_ffc(make_double2(c, s));
    }
  }
  for (int k = gt; k < n; k += gs) {
    const long long k2 = ((long long)k * (long long)k) % (2ll * n);
    double s, c;
    sincospi((double)k2 / (double)n, &s, &c);
    T.chirpI[k] = make_double2(c, s);
  }
  if (!grid_sync(A)) return;
  // spectrum of the L-embedding of W_beta: t_0 = omega_1 ... t_{n-1} = omega_n, t_{-1} = omega_0
  col_pass<false, true, double2>(A, S, A.twL, A.cp.lg1, A.cp.lg2, 1, A.cap_col, nullptr, A.Y1,
                                 [&](int m, double2) -> double2 {
                                   double v[2];
#pragma unroll
                                   for (int h = 0; h < 2; ++h) {
                                     const int i = 2 * m + h;
                                     v[h] = i < n ? T.omega[i + 1] : (i == L - 1 ? T.omega[0] : 0.0);
                                   }
                                   return make_double2(v[0], v[1]);
                                 });
  if (!grid_sync(A)) return;
  row_pass<1, double2>(A, S, A.twL, A.Y1, nullptr, nullptr, T.What, 1.0, -1);
  if (!grid_sync(A)) return;
  // Bluestein kernels: b_d = e^{-+ i pi d^2/n} placed circularly (|d| < n), spectra scaled for
  // the inverse (1/(L n)) and forward (1/L) n-point DFTs.
  for (int pass = 0; pass < 2; ++pass) {
    col_pass<false, true, double2>(A, S, A.twL, A.bp.lg1, A.bp.lg2, 0, A.cap_bcol, nullptr, A.Y1,
                                   [&](int m, double2) -> double2 {
                                     int d = m < n ? m : (m > L - n ? L - m : -1);
                                     if (d < 0) return make_double2(0.0, 0.0);
                                     const double2 c = T.chirpI[d];
                                     return pass == 0 ? cconj(c) : c;
                                   });
    if (!grid_sync(A)) return;
    crow_pass<1>(A, S, nullptr, pass == 0 ? T.BhI : T.BhF,
                 pass == 0 ? 1.0 / ((double)L * (double)n) : 1.0 / (double)L);
    if (!grid_sync(A)) return;
  }
  // eigenvalues of s(W_beta) and s(Q): forward n-point DFT by Bluestein
  for (int which = 0; which < 2; ++which) {
    col_pass<false, true, double2>(A, S, A.twL, A.bp.lg1, A.bp.lg2, 0, A.cap_bcol, nullptr, A.Y1,
                                   [&](int m, double2) -> double2 {
                                     if (m >= n) return make_double2(0.0, 0.0);
                                     const double c = circ_col(T.omega, which, T.precond, n, m);
                                     return cscale(cconj(T.chirpI[m]), c);
                                   });
    if (!grid_sync(A)) return;
    crow_pass<0>(A, S, T.BhF, nullptr, 1.0);
    if (!grid_sync(A)) return;
    double2 *out = which == 0 ? T.LamW : T.LamQ;
    col_pass<true, false, double2>(A, S, A.twL, A.bp.lg1, A.bp.lg2, 0, A.cap_bcol, A.Y2, nullptr,
                                   [&](int m, double2 z) -> double2 {
                                     if (m < n) out[m] = cmulc(z, T.chirpI[m]);
                                     return z;
                                   });
    if (!grid_sync(A)) return;
  }
}

// ------------------------------------------------------------------------------------------------
// batched instances: each CTA takes whole instances from a work queue and runs them with a
// one-CTA team (no grid barriers); per-instance data in Args, per-CTA work arrays patched in.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void patch_cta_scratch(Args &A, const CtaScratch &C) {
  A.x = C.x; A.r = C.r; A.rt = C.rt; A.p = C.p; A.q = C.q; A.uu = C.uu; A.vh = C.vh; A.H = C.H;
  A.xb = C.xb;
  A.SA = C.SA; A.SB = C.SB; A.SP = C.SP; A.Y1 = C.Y1; A.Y2 = C.Y2; A.Y3 = C.Y3; A.cprime = C.cprime;
  A.partials = C.partials; A.bar = C.bar;
  A.g = C.g; A.x32 = C.x32; A.r32 = C.r32; A.rt32 = C.rt32; A.p32 = C.p32; A.q32 = C.q32;
  A.uu32 = C.uu32; A.vh32 = C.vh32; A.SA32 = C.SA32; A.SP32 = C.SP32; A.Y1f = C.Y1f; A.Y2f = C.Y2f;
  A.xff = C.xff; A.rff = C.rff; A.rtff = C.rtff; A.pff = C.pff; A.qff = C.qff; A.uuff = C.uuff;
  A.vhff = C.vhff; A.SAff = C.SAff; A.SPff = C.SPff; A.Y1ff = C.Y1ff; A.Y2ff = C.Y2ff;
  A.x32b = C.x32b; A.xffb = C.xffb;
}

// One instance's weights (Lemma 2) and level tables (Lemma 1) with a one-CTA team; constant
// coefficients gamma, d+, d- given in the instance's lv_q/lv_kp/lv_km slots as raw values.
static __device__ void instance_tables(const Args &A, double *omega, double *gtmp, double alpha,
                                double beta, double tau, double h, double gam, double dp, double dm) {
  const int n = A.n, M = A.M;
  for (int k = 1 + threadIdx.x; k <= n + 1; k += blockDim.x)
    omega[k] = __dadd_rn(1.0, -__ddiv_rn(beta + 1.0, (double)k));
  __syncthreads();
  if (threadIdx.x == 0) {
    double gk = 1.0;
    gtmp[0] = gk;
    for (int k = 1; k <= n + 1; ++k) {
      gk = __dmul_rn(omega[k], gk);
      gtmp[k] = gk;
    }
  }
  __syncthreads();
  double lam1, lam0, lamm1;
  wsgd_lambdas(beta, lam1, lam0, lamm1);
  for (int k = threadIdx.x; k <= n + 1; k += blockDim.x) {
    double w = __dmul_rn(lam1, gtmp[k]);
    if (k >= 1) w = __dadd_rn(w, __dmul_rn(lam0, gtmp[k - 1]));
    if (k >= 2) w = __dadd_rn(w, __dmul_rn(lamm1, gtmp[k - 2]));
    omega[k] = w;
  }
  const double sigma = 1.0 - alpha / 2.0;
  const double denom = pow(tau, alpha) * tgamma(2.0 - alpha);
  const double hb = pow(h, beta);
  double *hc = const_cast<double *>(A.hc), *hl = const_cast<double *>(A.hl);
  double *eta = const_cast<double *>(A.lv_eta), *q = const_cast<double *>(A.lv_q);
  double *kp = const_cast<double *>(A.lv_kp), *km = const_cast<double *>(A.lv_km);
  int *ns = const_cast<int *>(A.lv_newsym);
  for (int l = threadIdx.x; l <= M; l += blockDim.x) {
    const double al = l21_a(alpha, sigma, l), bl = l21_b(alpha, sigma, l);
    hl[l] = al - bl;
    hc[l] = l >= 1 ? al + l21_b(alpha, sigma, l + 1) - bl : 0.0;
    if (l < M) {
      const double c0 = l == 0 ? l21_a(alpha, sigma, 0) : l21_a(alpha, sigma, 0) + l21_b(alpha, sigma, 1);
      eta[l] = c0 / denom;
      q[l] = gam / (2.0 * h);
      kp[l] = dp / hb;
      km[l] = dm / hb;
      ns[l] = l <= 1;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ int next_instance(const BatchArgs &B) {
  __shared__ int s_i;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned k = atomicAdd(B.next, 1u);
    s_i = k < (unsigned)B.count ? B.order[k] : -1;
  }
  __syncthreads();
  return s_i;
}

// a_l, b_l of Lemma 1 and the history coefficients hc[m] = a_m + b_{m+1} - b_m, hl[j] = a_j - b_j;
// per level eta_j = c^{(j)}_0 / (tau^alpha Gamma(2-alpha)) and the scaled coefficients.
__device__ __forceinline__ double l21_a(double alpha, double sigma, int l) {
  if (l == 0) return pow(sigma, 1.0 - alpha);
  return pow(l + sigma, 1.0 - alpha) - pow(l - 1 + sigma, 1.0 - alpha);
}
__device__ __forceinline__ double l21_b(double alpha, double sigma, int l) {
  if (l == 0) return 0.0;
  return (pow(l + sigma, 2.0 - alpha) - pow(l - 1 + sigma, 2.0 - alpha)) / (2.0 - alpha) -
         0.5 * (pow(l + sigma, 1.0 - alpha) + pow(l - 1 + sigma, 1.0 - alpha));
}


// Cooperative launch of a whole-grid kernel with `threads` per CTA.
static inline int coop_launch_n(const void *fn, int grid, int threads, size_t smem, cudaStream_t st,
                                void **args) {
  cudaError_t e = cudaLaunchCooperativeKernel(fn, grid, threads, args, smem, st);
  return e == cudaSuccess ? kOK : kECuda;
}

}  // namespace tsf
