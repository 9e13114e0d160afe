"""Parity at the workloads' full sizes, in the launch shape the benchmark times (one launch over
the levels, autotuned plan), on the first 8 levels.

Dense elimination cannot run at these sizes (34 GB per level at n = 65535), so the oracle checks
sampled rows of each level's equation (Eq. (3.1)), g - A u^{j+1} = 0, evaluated row by row from the
GPU's own level vectors (oracle.level_equation_rows, O(n) per row).  The bound for row i is derived
from the arithmetic:
    |r_i| <= rho_j ||g||_2 + 8 u64 log2(L) (||A|| ||u^{j+1}||_2 + ||B|| ||u^j||_2 + ||hist||_2)
             + sqrt(n) u64 ||A|| ||u^{j+1}||_inf
  rho_j: the relative residual the level's stopping rule allows, computed here and not read from
  the GPU: tol = 1e-12 for an FP64 CGS level (its recursive residual must drop below tol), and
  max(tol, 64 u64 kappa_j) for a mixed-precision level, which may be accepted at the FP64 floor
  of r = g - A x, with kappa_j = ||A||_rowsum / eta_j >= max|A^| / eta_j (every eigenvalue of a
  Toeplitz matrix is bounded by its largest absolute row sum).  The GPU's own reported residual
  must also lie below rho_j.  The second term is the rounding of FP64 FFT Toeplitz products of
  length L (normwise, about u log2 L ||T|| ||v||); the last is the oracle's own FP64 dot product.
  ||A||, ||B|| are bounded by the largest absolute row sum of the Toeplitz matrices.  Conditioning makes elementwise agreement
  to 1e-10 unattainable at these sizes (u64 kappa_eff ~ 1e-7 at n = 65535), which is why the
  residual and not the solution is checked; where the oracle can run (batch instances with
  n <= 1100) the solution is compared to elimination at 1e-10.
"""
import math

import numpy as np
import pytest

import oracle as O
import tsfcde_workloads as W
from gpu_common import rel_l2, solver_module

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53
LEVELS = 8


def _rows(n, seed):
    rng = np.random.default_rng(seed)
    fixed = [0, 1, 2, n // 7, n // 3, n // 2, n - 3, n - 2, n - 1]
    return sorted(set([i for i in fixed if 0 <= i < n] + list(rng.integers(0, n, 8))))


def _row_sum_bound(prob, j):
    """max_i sum_k |A_ik| and the same for B (Toeplitz: eta, sigma, kappa_pm, q, sum |omega|)."""
    e, q, kp, km = O.level_scalars(prob, j)
    sigma = 1.0 - prob.alpha / 2.0
    sw = float(np.abs(O.wsgd_weights(prob.beta, prob.n + 1)).sum())
    Lsum = (abs(kp) + abs(km)) * sw + 2.0 * abs(q)
    return abs(e) + sigma * Lsum, abs(e) + (1.0 - sigma) * Lsum


def _allowed_residual(prob, j, precision, tol=1e-12):
    """The relative residual a level may stop at, from the oracle's scalars (module docstring)."""
    e, _, _, _ = O.level_scalars(prob, j)
    nA, _ = _row_sum_bound(prob, j)
    if precision == "fp64":
        return tol
    return max(tol, 64.0 * U64 * nA / abs(e))


def _check_levels(prob, levels, resid, seed=0, label="", precision="fp64", first=0):
    """Sampled rows of levels first..len(levels)-2 against the derived bound; returns the largest
    observed |r_i| / bound_i."""
    n = prob.n
    L = max(8, 1 << math.ceil(math.log2(2 * n)))
    rows = _rows(n, seed)
    hs = prob.tau ** (-prob.alpha) / math.gamma(2.0 - prob.alpha)
    x = prob.grid()
    sigma = 1.0 - prob.alpha / 2.0
    worst = 0.0
    for j in range(first, len(levels) - 1):
        g, Au = O.level_equation_rows(prob, j, rows, levels[:j + 1], levels[j + 1])
        nA, nB = _row_sum_bound(prob, j)
        H = np.zeros(n)
        if j >= 1:
            c = O.c_coeffs(prob.alpha, j)
            for s in range(j):
                H += c[j - s] * (levels[s + 1] - levels[s])
        fn = (np.linalg.norm(prob.f(x, (j + sigma) * prob.tau)) if prob.f is not None else 0.0)
        un, uj = np.linalg.norm(levels[j + 1]), np.linalg.norm(levels[j])
        gnorm = nB * uj + hs * np.linalg.norm(H) + fn
        rho = _allowed_residual(prob, j, precision)
        assert resid[j] <= rho, (label, j, resid[j], rho)   # the GPU's claim, held to the rule
        bound = (rho * gnorm + 8 * U64 * math.log2(L) * (nA * un + nB * uj + hs * np.linalg.norm(H))
                 + math.sqrt(n) * U64 * nA * np.abs(levels[j + 1]).max())
        ratio = float(np.abs(g - Au).max() / bound)
        worst = max(worst, ratio)
        assert ratio <= 1.0, (label, j, ratio)
    print(f"{label}: largest sampled |r_i| / bound = {worst:.3g}")
    return worst


def _march_levels(s, nlev):
    out = [s.get_level()[0]]
    for _ in range(nlev):
        s.step(1)
        out.append(s.get_level()[0])
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_large_workload_full_size(precision):
    """n = 65535, M = 1024, T. Chan: first 8 levels, FP64 (as specified) and mixed.  The mixed
    march is held to the level equations: its gap to the FP64 march (about 2e-6) is the
    conditioning of this size, u64 kappa_eff, not an error of either."""
    P = solver_module()
    prob = W.config_large()
    s = P.Solver.from_problem(prob, source="separable", autotune=True, precision=precision)
    st = s.step(LEVELS)                           # one launch, as timed
    one = s.get_level()[0]
    assert st["device_launches"] == 1
    s.reset()
    levels = _march_levels(s, LEVELS)
    assert np.array_equal(one, levels[-1])        # deterministic: same plan, same passes
    _, rs = s.history(LEVELS)
    s.close()
    _check_levels(prob, levels, rs, seed=1, label=f"large n=65535 {precision}", precision=precision)
    # manufactured solution: the scheme's error at t_8 is far below ||u||
    ex = prob.exact(prob.grid(), LEVELS * prob.tau)
    assert rel_l2(levels[-1], ex) < 1e-5


def test_precision_workload_full_size_mixed_vs_fp64():
    """n = 2^20 - 1, M = 512: mixed within 1e-8 of the FP64 GPU path on each of the first 8
    levels, and both satisfy the level equations."""
    P = solver_module()
    prob = W.config_mixed()
    runs = {}
    for prec in ["fp64", "mixed"]:
        s = P.Solver.from_problem(prob, source="separable", precision=prec, autotune=True)
        runs[prec] = (_march_levels(s, LEVELS), s.history(LEVELS)[1])
        s.close()
    a, b = runs["fp64"][0], runs["mixed"][0]
    gaps = [rel_l2(b[j], a[j]) for j in range(1, LEVELS + 1)]
    assert max(gaps) <= 1e-8, gaps
    for prec, (lv, rs) in runs.items():
        _check_levels(prob, lv, rs, seed=2, label=f"precision workload {prec}", precision=prec)


@pytest.mark.parametrize("algorithm,precision,tol", [("ids", "fp64", 1e-10), ("ids-const", "fp64", 1e-10),
                                                     ("ids", "mixed", 1e-8)])
def test_batch_workload_full_size(algorithm, precision, tol):
    """4096 instances (n from 255 to 16383), first 8 levels in one launch: every instance with
    n <= 1100 against elimination (a seeded sample of 24; 1e-10 in FP64, 1e-8 mixed), and the
    equations of levels 0..7 for the 6 largest instances."""
    P = solver_module()
    probs = W.config_batch(M=LEVELS)
    b = P.Batch(probs, LEVELS, algorithm=algorithm, precision=precision)
    b.step(LEVELS)
    final = [b.get_level(i)[0] for i in range(len(probs))]
    small = [i for i, p in enumerate(probs) if p.n <= 1100]
    pick = sorted(np.random.default_rng(5).choice(small, size=24, replace=False))
    for i in pick:
        ref = O.run(probs[i])
        assert rel_l2(final[i], ref[-1]) <= tol, (i, probs[i].n)
    big = sorted(range(len(probs)), key=lambda i: -probs[i].n)[:6]
    b.reset()
    lv = {i: [b.get_level(i)[0]] for i in big}
    for _ in range(LEVELS):
        b.step(1)
        for i in big:
            lv[i].append(b.get_level(i)[0])
    for i in big:
        assert np.array_equal(lv[i][-1], final[i])
        _, rs = b.history(i, LEVELS)
        _check_levels(probs[i], lv[i], rs, seed=i, label=f"batch {algorithm} {precision} n={probs[i].n}",
                      precision="mixed" if (precision == "mixed" or algorithm == "ids-const") else "fp64")
    b.close()


def test_history_workload_full_size():
    """n = 2^18 - 1, M = 8192 (17 GB history ring): first 8 levels."""
    P = solver_module()
    prob = W.config_history()[0]
    s = P.Solver.from_problem(prob, source="separable", autotune=True)
    s.step(LEVELS)
    one = s.get_level()[0]
    s.reset()
    levels = _march_levels(s, LEVELS)
    assert np.array_equal(one, levels[-1])
    _, rs = s.history(LEVELS)
    s.close()
    _check_levels(prob, levels, rs, seed=3, label="history n=262143")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_largest_supported_n(precision):
    """N = 2^22 - 1, the largest the ABI accepts (FFT half-length 2^22, 4096-point Bluestein rows,
    about 193 KB of shared memory per CTA, 512 threads per CTA): 3 levels of the small workload's
    coefficients against the row-wise level equations and the manufactured solution."""
    P = solver_module()
    prob = W.config_small(n=(1 << 22) - 1, M=3)
    s = P.Solver.from_problem(prob, source="separable", precision=precision)
    levels = _march_levels(s, prob.M)
    _, rs = s.history(prob.M)
    s.close()
    _check_levels(prob, levels, rs, seed=4, label=f"n=2^22-1 {precision}", precision=precision)
    if precision == "fp64":
        # at tau = 1/3 the scheme's time error dominates and hardly depends on n: the error
        # against the manufactured solution matches the oracle's at n = 1023 (0.01154; h^2
        # terms move it by about 3e-6).  kappa_eff ~ 1e11 here, so the mixed march, which may
        # stop at its FP64 residual floor 64 u64 kappa_eff, is held to the level equations only.
        small = W.config_small(n=1023, M=3)
        e_ref = rel_l2(O.run(small)[-1], small.exact(small.grid(), small.T))
        e_gpu = rel_l2(levels[-1], prob.exact(prob.grid(), prob.T))
        print(f"n=2^22-1: error vs exact {e_gpu:.6g}, oracle at n=1023 {e_ref:.6g}, "
              f"difference {abs(e_gpu - e_ref):.3g}")
        assert abs(e_gpu - e_ref) < 5e-5, (e_gpu, e_ref)


def test_large_workload_whole_march_and_its_levels_at_maxit():
    """n = 65535, M = 1024, T. Chan (as specified), FP64, maxit 2000: the whole march (about
    50 s).  T. Chan's circulant misses A's smallest eigenvalues at this size
    (test_gpu_spectrum.py), so CGS needs hundreds of iterations and a level may stop at maxit,
    returning its minimum-residual iterate with E_NOT_CONVERGED and the state kept.  Such
    levels must be few and still near tol; every other level below tol; and the solution at T
    must carry the same error against the manufactured solution as the Strang-preconditioned
    march of the same problem (whose levels all converge).  Measured: one level at maxit with
    residual 1.31e-12; errors at T 1.332e-7 (T. Chan) and 1.320e-7 (Strang), the two solutions
    1.26e-9 apart.  That gap is the FP64 rounding of two different solves of levels whose
    kappa_eff is about 4.5e8, about 1 % of the scheme's error; the test allows 5 %."""
    P = solver_module()
    prob = W.config_large()
    s = P.Solver.from_problem(prob, source="separable", autotune=True, levels_per_launch=64)
    st = s.step(prob.M)
    its, rs = s.history(prob.M)
    u_t = s.get_level()[0]
    s.close()
    at_max = its >= 2000
    print(f"T. Chan: {int(at_max.sum())} levels at maxit, residuals there {rs[at_max]}, "
          f"largest elsewhere {rs[~at_max].max():.3g}, mean iterations {its.mean():.1f}")
    assert st["status"] == (5 if at_max.any() else 0)
    assert at_max.sum() <= 4
    assert (rs[~at_max] < prob.tol).all()
    assert (rs[at_max] < 10 * prob.tol).all()
    with P.Solver.from_problem(prob, source="separable", autotune=True, levels_per_launch=64,
                               preconditioner="strang") as s2:
        u_s = s2.solve()
        its2, rs2 = s2.history(prob.M)
    assert (its2 < 2000).all() and (rs2 < prob.tol).all()
    ex = prob.exact(prob.grid(), prob.T)
    e_t, e_s = rel_l2(u_t, ex), rel_l2(u_s, ex)
    gap = rel_l2(u_t, u_s)
    print(f"error vs exact at T: T. Chan {e_t:.6g}, Strang {e_s:.6g}; gap between the two {gap:.3g}")
    assert abs(e_t - e_s) <= 0.05 * e_s
    assert gap <= 0.05 * e_s
