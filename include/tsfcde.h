/*
 * tsfcde.h -- C ABI of the GB300 solver for the time-space fractional convection-diffusion
 * equation (TSFCDE) of Gu, Huang, Ji, Carpentieri and Alikhanov (arXiv:1603.00279).
 *
 * Problem (Eq. (1.1)): Caputo d^alpha_t u = gamma(t) u_x + d_+(t) aD^beta_x u + d_-(t) xD^beta_b u
 * + f(x,t) on [a,b] x (0,T], u(x,0) = phi(x), u(a,t) = u(b,t) = 0, alpha in (0,1], beta in (1,2],
 * d_+- >= 0.
 *
 * Method: the implicit difference scheme Eq. (2.1) (L2-1_sigma in time, Lemma 1; two-sided
 * weighted-shifted Grunwald operators in space, Lemma 2), written per level as the nonsymmetric
 * Toeplitz system Eq. (3.3), A^{(j+sigma)} u^{j+1} = B^{(j+sigma)} u^j - history + f^{j+sigma}
 * (the history term is subtracted, as in Eq. (3.1)), and solved level by level as in Algorithm
 * "Practical implementation of IDS": the right-hand side is assembled with an FFT Toeplitz
 * product and the system is solved with CGS preconditioned by the circulant P^{(j+sigma)} of
 * Eq. (3.7).
 *
 * Conventions shared by every entry point:
 *   - N is the number of INTERIOR grid points (the paper's N-1): h = (b-a)/(N+1),
 *     x_i = a + i h for i = 1..N; tau = T/M, sigma = 1 - alpha/2.
 *   - Vectors passed in or out hold the N interior values in natural order, float64, in HOST
 *     memory unless an argument says otherwise.  The caller owns every buffer it passes; the
 *     library owns all device memory it allocates and frees it in tsfcde_free().
 *   - Every call returns a status (TSFCDE_OK = 0 or one of the TSFCDE_E_* codes below);
 *     tsfcde_strerror() turns it into text.  A context stays valid after E_NOT_CONVERGED; after
 *     any other error it may only be freed.
 *   - Calls on one context must not overlap; different contexts are independent.
 *   - All device work runs on CUDA device 0 of the calling process unless `device` in the
 *     options says otherwise.
 */
#ifndef TSFCDE_H
#define TSFCDE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------------------------- */
#define TSFCDE_OK 0
#define TSFCDE_E_INVALID_ARG 1      /* an argument is out of the ranges of Eq. (1.1) or NULL     */
#define TSFCDE_E_NOMEM 2            /* device or host allocation failed                          */
#define TSFCDE_E_CUDA 3             /* a CUDA runtime call failed                                */
#define TSFCDE_E_NONFINITE 4        /* a callback or an iterate produced NaN/Inf                 */
#define TSFCDE_E_NOT_CONVERGED 5    /* CGS reached maxit on some level (state stays valid)       */
#define TSFCDE_E_BREAKDOWN 6        /* CGS breakdown: rho = 0 or (r~, A p^) = 0                  */
#define TSFCDE_E_SINGULAR_PRECOND 7 /* an eigenvalue of the circulant P vanished (Theorem 4)      */
#define TSFCDE_E_TIMEOUT 8          /* a device-wide barrier wait ran out of its bound            */
#define TSFCDE_E_STATE 9            /* stepping past level M, or a call in the wrong state        */
#define TSFCDE_E_NO_DEVICE 10       /* no CUDA device / library built without a usable GPU        */
#define TSFCDE_E_BOUNDS 11          /* libtsfcde_checked.so only (built with -DTSFCDE_CHECKED): a
                                       device index outside its array was caught and redirected
                                       to element 0 instead of being accessed; see
                                       tsfcde_checked_report()                                  */

/* ---- callbacks (host functions, called only during setup, on the caller's thread) ----------- */
/* gamma(t), d_plus(t), d_minus(t) of Eq. (1.1); called at t_{j+sigma} = (j+sigma) tau. */
typedef double (*tsfcde_coef_fn)(double t, void *user);
/* Vectorized field: out[i] = F(x[i], t) for i < n.  The library passes its own mesh x_i = a + i h
 * (i = 1..N, Section 2.1).  phi is called once with t = 0; f is called once per level with
 * t = t_{j+sigma} (Eq. (2.1) evaluates f at t_{j+sigma}). */
typedef void (*tsfcde_field_fn)(double t, const double *x, double *out, int64_t n, void *user);

/* ---- options -------------------------------------------------------------------------------- */
#define TSFCDE_PRECOND_STRANG 0 /* Strang circulant s(.) of Eq. (3.7) (the paper's choice)       */
#define TSFCDE_PRECOND_TCHAN 1  /* T. Chan's optimal circulant in place of s(.)                  */
#define TSFCDE_PRECOND_NONE 2   /* plain CGS                                                     */

#define TSFCDE_FP64 0  /* every step in float64                                             */
#define TSFCDE_MIXED 1 /* iterative refinement: residual r = g - A x, solution update, history
                          sum and all spectra/weights in float64; CGS on A d = r in float32 or
                          float-float (FFTs, matvecs and preconditioner in that precision,
                          spectra rounded from float64), chosen per level (inner_precision);
                          see TSFCDE_INNER_AUTO for the stopping and escalation rules       */

typedef struct tsfcde_options {
  int32_t precision;      /* TSFCDE_FP64 (default) or TSFCDE_MIXED                         */
  int32_t preconditioner; /* TSFCDE_PRECOND_*; default STRANG                               */
  double tol;             /* CGS stop: ||r_k||_2 / ||r_0||_2 < tol (Section 4); default 1e-12 */
  int32_t maxit;          /* CGS iterations per level before E_NOT_CONVERGED; default 2000.
                             A level that reaches it keeps its minimum-residual iterate.    */
  int32_t device;         /* CUDA device ordinal; default 0                                 */
  /* Separable source f(x,t) = sum_r T_r(t) X_r(x) (used when source_rank > 0, in which case the
   * f callback of tsfcde_setup must be NULL).  Both arrays hold source_rank host callbacks and
   * are read during setup only: the library calls source_space[r] once on its mesh x_i
   * (t argument 0) and source_time[r] once per level at t_{j+sigma}, with tsfcde_setup's `user`;
   * the device rebuilds f^{j+sigma}_i = sum_r T_r(t_{j+sigma}) X_r(x_i) at every level from these
   * R (N + M) values instead of an M x N table. */
  int32_t source_rank;
  const tsfcde_field_fn *source_space;
  const tsfcde_coef_fn *source_time;
  int32_t levels_per_launch; /* device launches cover at most this many levels; 0 = no limit */
  void *stream;              /* cudaStream_t to run on (e.g. a PyTorch stream); NULL = the
                                library creates and owns a non-blocking stream               */
  double inner_tol;          /* MIXED: relative residual reduction of each inner (float32 or
                                float-float) solve; default 1e-3: short inner solves with more
                                refinement steps took fewer iterations overall than 1e-5 on
                                every workload measured (CGS restarts are cheap, its erratic
                                late convergence is not)                                    */
  int32_t inner_maxit;       /* MIXED: inner CGS iterations per refinement step; default 1000 */
  int32_t outer_maxit;       /* MIXED: refinement steps per level before escalation; default 12 */
  int32_t barrier_spin_log2; /* a device-wide barrier wait gives up after 2^k polls and the call
                                returns TSFCDE_E_TIMEOUT; default 23 (a few seconds)           */
  int32_t test_skip_arrival; /* testing hook, 0 normally: when 1, CTA 0 skips its first barrier
                                arrival in the next launch only, so every wait of that launch
                                runs into its bound and the call returns TSFCDE_E_TIMEOUT     */
  int32_t inner_precision;   /* MIXED inner solve: TSFCDE_INNER_AUTO (default), _FP32, _FF    */
  int32_t autotune;          /* 1: at setup, time the candidate FFT splits N/2 = N1 x N2 (N1 =
                                N2/2, N2, 2 N2) and per-pass chunk sizes on the level operator
                                product and keep the fastest (see tsfcde_get_plan); 0: default
                                plan (N1 <= N2, N1 >= N2/2, chunks of 4096 values)            */
  int32_t algorithm;         /* TSFCDE_ALG_IDS (default) or TSFCDE_ALG_IDS_CONST, below        */
  int32_t test_inject;       /* testing hook, 0 normally (TSFCDE_INJECT_*, below): makes one
                                failure path reachable from the host with valid inputs        */
  int32_t fast_history;      /* 0 (default): the history sum of Lemma 1 summed directly at every
                                level, O(j N) per level.  1: the same sum as a blocked
                                convolution in time: increments in blocks of 128 levels, whose
                                2 x 128-point FFT spectra (stored once per block, 2 x 129 x N
                                values per block, about twice the history ring) are combined
                                with the kernel's spectra once per block of levels; the terms of
                                the level's own block are summed directly.  Equal to the direct
                                sum up to rounding (FFT convolution: a relative error of a few
                                u64 log2(256) per element).  Used when M > 128 and 2N >= 256;
                                otherwise the direct sum runs.  Single contexts only.        */
} tsfcde_options;

/* Testing hooks (tsfcde_options.test_inject).  Valid problems cannot reach these failure paths
 * (Theorems 1 and 4 keep A and P nonsingular, and a level's first CGS denominator is positive),
 * so a host-set hook stands in for the condition; nothing faults on the GPU.
 *   NOMEM:     tsfcde_setup / tsfcde_batch_setup report their device allocation as failed
 *              (no allocation is attempted) and return TSFCDE_E_NOMEM after releasing
 *              everything;
 *   BREAKDOWN: the first CGS iteration of the first level advanced by a context sees
 *              (r~, A p^) = 0 and the step returns TSFCDE_E_BREAKDOWN;
 *   SINGULAR:  the first level's preconditioner check sees a vanishing eigenvalue of P and the
 *              step returns TSFCDE_E_SINGULAR_PRECOND. */
#define TSFCDE_INJECT_NONE 0
#define TSFCDE_INJECT_NOMEM 1
#define TSFCDE_INJECT_BREAKDOWN 2
#define TSFCDE_INJECT_SINGULAR 3

/* Level algorithm.
 * TSFCDE_ALG_IDS: Algorithm "Practical implementation of IDS" -- every level solved by the
 *   circulant-preconditioned CGS.
 * TSFCDE_ALG_IDS_CONST: Algorithm "Practical implementation of IDS with constant coefficients"
 *   (Section 3.2), for gamma, d_+ and d_- constant in t.  Then A^{(j+sigma)} = A for every
 *   j >= 1 (Eq. (3.4)).  Level 0 is solved by CGS as usual.  At level 1 the two systems
 *   A x = e_1 and A y = e_N of Eq. (3.5) are solved by the preconditioned CGS, each refined once
 *   with the inverse they define.  Every level j >= 1 then computes u^{j+1} = A^{-1} g by the
 *   Gohberg-Semencul formula (Eq. (3.6), Section 3.1): Algorithm "Compute z = A^{-1} v", four
 *   triangular Toeplitz products by FFT, with no Krylov iterations.  The level's FP64 residual ||g - A u^{j+1}|| / ||g|| is
 *   measured.  While it is above both tol and 64 u64 kappa_eff, the level is refined,
 *   u += A^{-1}(g - A u), at most twice.  A level still above both is reported as
 *   TSFCDE_E_NOT_CONVERGED with its state kept.
 *   tsfcde_setup returns TSFCDE_E_INVALID_ARG if gamma, d_+ or d_- differ between two levels
 *   j, j' >= 1; it returns TSFCDE_E_BREAKDOWN from the step if xi_0 = (A^{-1})_{11} is zero. */
#define TSFCDE_ALG_IDS 0
#define TSFCDE_ALG_IDS_CONST 1

/* Inner precision of TSFCDE_MIXED.  AUTO estimates per level kappa_eff = max|A^| / eta_j <=
 * 1 + sigma ((kappa_+ + kappa_-) 2|omega_1| + 2|q|) / eta_j (Remark 3.1 bounds the eigenvalues
 * of s(W_beta) by 2|omega_1|) and runs the inner CGS in float32 when u32 * kappa_eff < 1e-3,
 * otherwise in float-float (pairs of floats, ~48-bit significands, on the FP32 pipe).  A level
 * whose float64 residual stops halving below 64 u64 kappa_eff (the float64 floor of r = g - Ax)
 * is accepted; above that it is finished by the float64 CGS. */
#define TSFCDE_INNER_AUTO 0
#define TSFCDE_INNER_FP32 1
#define TSFCDE_INNER_FF 2

/* Fill `opt` with the defaults above (the paper's settings: Strang, tol 1e-12, x0 = 0). */
void tsfcde_default_options(tsfcde_options *opt);

/* ---- statistics ----------------------------------------------------------------------------- */
typedef struct tsfcde_stats {
  int64_t level;            /* current level j: the context holds u^j                       */
  int64_t levels_advanced;  /* levels advanced by the call that filled this struct          */
  int64_t total_iterations; /* CGS iterations summed over those levels                      */
  int32_t max_iterations;   /* largest per-level CGS iteration count among them             */
  int32_t min_iterations;   /* smallest                                                     */
  double max_residual;      /* largest final ||r||/||r_0|| among them                       */
  int32_t status;           /* worst device status seen (a TSFCDE_* code)                   */
  int32_t device_launches;  /* kernel launches the call made                                */
  double device_ms;         /* device time of those launches (CUDA events on their stream)  */
  int64_t outer_iterations; /* MIXED: refinement steps summed over the levels advanced      */
  int32_t escalated_levels; /* MIXED: levels finished by the float64 CGS                    */
  int32_t gsf_levels;       /* IDS_CONST: levels solved by the Gohberg-Semencul formula; for
                               these, iterations count the two generator solves (level 1 only)
                               and outer_iterations the applications of A^{-1} (1 + refinements) */
  int32_t floor_levels;     /* MIXED / IDS_CONST (info, not an error): levels whose float64
                               residual was accepted at its floor 64 u64 kappa_eff, above tol,
                               because refinement no longer reduced it                       */
  int32_t pad_;
} tsfcde_stats;

typedef struct tsfcde_ctx tsfcde_ctx;

/* ---- life cycle ----------------------------------------------------------------------------- */

/* Build a solver for one TSFCDE instance (Eq. (1.1) on the mesh of Section 2.1).
 *   out       receives the context (set to NULL on failure).
 *   a < b, T > 0, N >= 1 interior points, M >= 1 levels, 0 < alpha <= 1, 1 < beta <= 2.
 *   gamma, d_plus, d_minus: required; d_plus, d_minus must be >= 0 at every t_{j+sigma}.
 *   phi: required (initial value u^0_i = phi(x_i), Eq. (2.1)).
 *   f: source, or NULL for f = 0 or for a separable source given through `opt`.
 *   user: passed through to every callback.  opt: NULL for the defaults.
 * Allocates on the device: O(N) vectors and spectra, the O(M N) history of increments
 * u^{s+1} - u^s (FP64) that the L2-1_sigma sum of Lemma 1 reads at every level, and, when f is a
 * callback, the M x N source table.  Computes on the device: the WSGD weights (Lemma 2), the
 * L2-1_sigma coefficients (Lemma 1), the Toeplitz spectra of the circulant embedding, and the
 * eigenvalues of the circulant approximations s(Q), s(W_beta).  Leaves the context at level 0. */
int tsfcde_setup(tsfcde_ctx **out, double a, double b, double T, int64_t N, int64_t M,
                 double alpha, double beta, tsfcde_coef_fn gamma, tsfcde_coef_fn d_plus,
                 tsfcde_coef_fn d_minus, tsfcde_field_fn phi, tsfcde_field_fn f, void *user,
                 const tsfcde_options *opt);

/* Advance `nsteps` levels (Algorithm "Practical implementation of IDS", one loop trip per
 * level): history sum of Lemma 1, B u^j by FFT, + f, then preconditioned CGS for A u^{j+1} = g
 * from a zero initial guess (Section 4).  Fails with E_STATE if the march would pass level M.
 * `stats` may be NULL.  Runs asynchronously to nothing: returns when the levels are done. */
int tsfcde_step(tsfcde_ctx *ctx, int64_t nsteps, tsfcde_stats *stats);

/* Advance to level M and copy u^M (N values) to the host buffer u_out (may be NULL). */
int tsfcde_solve(tsfcde_ctx *ctx, double *u_out, tsfcde_stats *stats);

/* Copy level u^j of the current march to the host buffer u_out (N values), for any
 * 0 <= j <= current level (E_INVALID_ARG otherwise).  Algorithm "Practical implementation of IDS"
 * produces every level; the context keeps u^0 of the march, the current level u^c and the ring of
 * increments d^s = u^{s+1} - u^s (s < c) that the history sum of Lemma 1 reads, so u^j is rebuilt
 * on the device by the shorter of the two sums u^0 + sum_{s<j} d^s and u^c - sum_{j<=s<c} d^s,
 * in FP64 in a fixed order.  j = 0 and j = c return the stored vectors exactly; in between the
 * rebuilt level differs from the march's own u^j by at most (number of terms) * u64 * sum |d^s|
 * per element.  Does not change the march state. */
int tsfcde_get_level(tsfcde_ctx *ctx, int64_t j, double *u_out);

/* The current level c of the march (the context holds u^c). */
int tsfcde_level(tsfcde_ctx *ctx, int64_t *level);

/* The spatial weights the context computed at setup, for k = 0..N+1 (N+2 host values each; either
 * pointer may be NULL): g_out[k] = g_k, the Grunwald weights (-1)^k binom(beta, k) by the
 * recurrence g_k = (1 - (beta+1)/k) g_{k-1} of Lemma 3, and omega_out[k] = omega_k, the WSGD
 * weights of Lemma 2 (omega_0 = lambda_1 g_0, omega_1 = lambda_1 g_1 + lambda_0 g_0,
 * omega_k = lambda_1 g_k + lambda_0 g_{k-1} + lambda_{-1} g_{k-2}).  Every operation is a single
 * IEEE-754 binary64 operation, rounded to nearest, evaluated left to right (no contraction into
 * fused multiply-adds), so the values are reproducible bit for bit on any conforming host. */
int tsfcde_get_weights(tsfcde_ctx *ctx, double *g_out, double *omega_out);

/* Return to level 0.  u0: N host values to use as u^0 (copied host to device), or NULL for
 * phi(x_i) (restored from a device copy made at setup; no host transfer). */
int tsfcde_reset(tsfcde_ctx *ctx, const double *u0);

/* Per-level CGS iteration counts and final relative residuals of the levels advanced so far:
 * iters[j] and resid[j] for j < count <= current level (either pointer may be NULL). */
int tsfcde_get_history(tsfcde_ctx *ctx, int32_t *iters, double *resid, int64_t count);

/* Diagnostic products with the level-j operators (Eq. (3.3), Eq. (3.7)), computed by the same
 * device kernels as the march: op = 0: y = A^{(j+sigma)} x, 1: y = B^{(j+sigma)} x,
 * 2: y = (P^{(j+sigma)})^{-1} x, 3: y = A^{-1} x by the Gohberg-Semencul formula (TSFCDE_ALG_IDS_CONST
 * only, after a march has passed level 1; j is ignored; TSFCDE_E_STATE before that).
 * x, y: N host values.  Does not change the march state. */
#define TSFCDE_OP_A 0
#define TSFCDE_OP_B 1
#define TSFCDE_OP_PINV 2
#define TSFCDE_OP_AINV_GS 3
int tsfcde_apply(tsfcde_ctx *ctx, int32_t op, int64_t j, const double *x, double *y);

/* Operator product that allocates nothing (no counterpart in the paper; an addition of this
 * library).  For callers that cannot call cudaMalloc -- code running inside another runtime's
 * memory pool or allocator hooks, processes whose device memory is reserved up front, or
 * latency-critical paths that must not allocate -- this computes y = A x (op = TSFCDE_OP_A) or
 * y = B x (op = TSFCDE_OP_B) for one level of Eq. (3.3), A = eta I - sigma L,
 * B = eta I + (1 - sigma) L, L = q Q + kappa_plus W_beta + kappa_minus W_beta^T, from the
 * level's scalars alone, without a context.
 *   N: interior points, 1 <= N <= 16383 (larger N returns TSFCDE_E_INVALID_ARG).
 *   beta in (1,2]; sigma = 1 - alpha/2; eta = eta_j; q = gamma/(2h); kappa_pm = d_pm / h^beta.
 *   x, y: N float64 values in DEVICE memory, owned by the caller.  stream: cudaStream_t or NULL.
 * All scratch (WSGD weights, twiddles, spectra, FFT work arrays, barrier words) lives in one
 * fixed 3 MiB file-scope device array that each device holds from library load until process
 * exit.  The first call on a device looks up that array's address and sets the kernel's
 * shared-memory limit.  Every call reuses the array: calls that overlap on the GPU race and
 * must be serialised by the caller.  Each call copies its status word to the host and returns
 * after the product is complete (it synchronises `stream`). */
int tsfcde_apply_operator_static(int64_t N, double beta, double sigma, double eta, double q,
                                 double kappa_plus, double kappa_minus, int32_t op,
                                 const double *x, double *y, void *stream);

/* ---- batched instances ----------------------------------------------------------------------
 * Many independent TSFCDE instances with their own N, alpha, beta and constant coefficients,
 * advanced together: each device CTA takes whole instances from a work queue (largest first)
 * and runs their level solves with CTA-local barriers only.  All instances share M and the
 * options (preconditioner, tol, maxit, precision).  f = 0 for batched instances. */
typedef struct tsfcde_instance {
  double a, b, T;         /* domain [a,b], final time T                                     */
  int64_t N;              /* interior points, 1 <= N <= 16383                               */
  double alpha, beta;     /* orders, as in tsfcde_setup                                      */
  double gamma, d_plus, d_minus;   /* constant coefficients (d_plus, d_minus >= 0)          */
  tsfcde_field_fn phi;    /* initial value: called once during tsfcde_batch_setup with t = 0 on
                             the instance's mesh x_i = a + i h, i = 1..N (u^0_i = phi(x_i))   */
  void *user;             /* passed through to phi                                          */
} tsfcde_instance;

typedef struct tsfcde_batch tsfcde_batch;

/* Set up `count` instances with M levels each.  Device memory: per instance its state, history
 * of increments (M x N FP64) and spectra; per CTA the work arrays of the largest instance. */
int tsfcde_batch_setup(tsfcde_batch **out, int64_t count, const tsfcde_instance *inst, int64_t M,
                       const tsfcde_options *opt);
/* Advance every instance by nsteps levels (one device launch).  stats sums over instances. */
int tsfcde_batch_step(tsfcde_batch *b, int64_t nsteps, tsfcde_stats *stats);
/* Copy level u^j of instance i (N_i host values), for any 0 <= j <= the batch's current level,
 * rebuilt from the instance's u^0, current level and ring of increments exactly as
 * tsfcde_get_level does. */
int tsfcde_batch_get_level(tsfcde_batch *b, int64_t i, int64_t j, double *u_out);
/* The batch's current level (every instance is at the same level). */
int tsfcde_batch_level(tsfcde_batch *b, int64_t *level);
/* Per-level CGS iterations and final residuals of instance i, levels 0..count-1. */
int tsfcde_batch_get_history(tsfcde_batch *b, int64_t i, int32_t *iters, double *resid, int64_t count);
/* Every instance back to level 0 with its u^0 (device copy, no host transfer). */
int tsfcde_batch_reset(tsfcde_batch *b);
/* Replace every instance's u^0 with u0_all (host; the N_i values of instance 0, then 1, ...,
 * concatenated: sum N_i doubles) and go back to level 0. */
int tsfcde_batch_set_initial(tsfcde_batch *b, const double *u0_all);
/* Copy every instance's current level to u_all (host, concatenated like u0_all). */
int tsfcde_batch_get_all(tsfcde_batch *b, double *u_all);
/* Advance every instance to level M (tsfcde_batch_step) and copy every u^M to u_all (host,
 * concatenated like u0_all; NULL skips the copy).  Returns the step's status; the copy is made
 * after E_NOT_CONVERGED too. */
int tsfcde_batch_solve(tsfcde_batch *b, double *u_all, tsfcde_stats *stats);
/* Release everything.  NULL is allowed. */
void tsfcde_batch_free(tsfcde_batch *b);
/* The batched launch's plan.  budget: complex values per shared-memory chunk (1024, 2048 or
 * 4096; it sets the shared memory per CTA, hence the CTAs per SM); n1_ge_n2: 1 when every
 * instance splits its half-length transform with N1 >= N2, 0 for N1 <= N2; ctas: CTAs of the
 * launch; best_ms: the tuner's time for the first two levels of every instance (0 without
 * tuning).  With opt->autotune = 1, tsfcde_batch_setup times every candidate on those two levels
 * (the states then go back to level 0) and keeps the fastest; otherwise budget 2048, N1 <= N2. */
int tsfcde_batch_get_plan(tsfcde_batch *b, int32_t *budget, int32_t *n1_ge_n2, int32_t *ctas,
                          double *best_ms);

/* The FFT plan in use: the split N/2 = N1 x N2 of the half-length transform, the per-pass chunk
 * budget (complex values per shared-memory buffer), and the autotuner's best time per operator
 * product in microseconds (0 when autotune was off).  Any pointer may be NULL. */
int tsfcde_get_plan(tsfcde_ctx *ctx, int32_t *N1, int32_t *N2, int32_t *budget, double *best_us);

/* Diagnostic: the history sum of Lemma 1 for level j, H_i = sum_{s<j} c^{(j)}_{j-s} (u^{s+1}_i -
 * u^s_i) (before the scaling tau^-alpha / Gamma(2-alpha)), computed by the same device phases the
 * march uses, in its own launch with the march's launch shape.  method: TSFCDE_HISTORY_CONTEXT
 * (0) sums as the march does (the blocked FFT convolution when fast_history is on), 
 * TSFCDE_HISTORY_DIRECT (1) always sums directly, term by term in order of s.  Requires
 * 1 <= j <= current level (the increments up to level j must be committed).  H_out: N host
 * values, or NULL (device work only, e.g. for timing).  Does not change the march state. */
#define TSFCDE_HISTORY_CONTEXT 0
#define TSFCDE_HISTORY_DIRECT 1
int tsfcde_history_sum(tsfcde_ctx *ctx, int64_t j, int32_t method, double *H_out);

/* Release everything the context holds.  NULL is allowed. */
void tsfcde_free(tsfcde_ctx *ctx);

/* TSFCDE_CHECKED builds: the first index violation the last launch of `ctx` caught (site number
 * of the checked access and the index, truncated to 32 bits); both 0 when none was caught or in a
 * normal build.  Reads the context's status words. */
int tsfcde_checked_report(tsfcde_ctx *ctx, int32_t *site, int32_t *index);

/* Measurement aid, no counterpart in the paper: the FP64 fused multiply-add throughput of CUDA
 * device `device` in TFLOP/s (2 flops per FMA), from a kernel of independent FMA chains timed
 * with CUDA events (about 0.1 s).  The level kernels are bound by this unit; benchmarks report
 * their algorithmic FP64 rate against it beside the peak derived from unit counts and clocks. */
int tsfcde_measure_fp64(int32_t device, double *tflops);

/* Static text for a status code. */
const char *tsfcde_strerror(int status);

/* Library version string. */
const char *tsfcde_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TSFCDE_H */
