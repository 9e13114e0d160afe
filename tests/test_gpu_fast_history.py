"""Fast history: the history sum of Lemma 1 as a blocked convolution in time (tsfcde_options
fast_history = 1; blocks of B = 128 levels, 2B-point FFTs along time).

* Same ring, two methods: at every level checked, the context's fast sum and the direct
  term-by-term sum (tsfcde_history_sum with method DIRECT) of the same increments agree within
  the rounding bound of an FFT convolution, derived here: per point and block p, the 2B-point
  circular convolution errs by at most about c u64 log2(2B) ||w||_2 ||d_p||_2 (w the kernel
  window, d_p the block's increments), summed over the blocks, plus the direct sum's own
  rounding; c = 16 leaves a margin over the textbook constant.
* The march with fast history against the oracle's elimination march (1e-10 at every level
  checked) and against the GPU march with the direct sum.
"""
import math

import numpy as np
import pytest

import oracle as O
import tsfcde_workloads as W
from gpu_common import rel_l2, solver_module

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53
B = 128


def _fft_bound(prob, levels, j):
    """Per-point bound on |H_fast - H_direct| at level j >= B (module docstring)."""
    c = O.c_coeffs(prob.alpha, j)              # c[m] = c^{(j)}_m, m = 0..j
    d = np.diff(np.array(levels[:j + 1]), axis=0)   # d^s, s < j (from the levels read back)
    q = j // B
    far = np.zeros(prob.n)
    for p in range(q):
        m = q - p
        lags = np.arange((m - 1) * B, (m + 1) * B)
        w = np.array([c[l] if 1 <= l < j else 0.0 for l in lags])
        blk = d[p * B:(p + 1) * B].copy()
        if p == 0:
            blk[0] = 0.0                        # d^0 enters through the endpoint term
        far += np.linalg.norm(w) * np.linalg.norm(blk, axis=0)
    direct = np.abs(c[j - np.arange(j)][:, None] * d).sum(axis=0)
    return 16 * U64 * math.log2(2 * B) * far + 4 * U64 * direct + 1e-300


@pytest.mark.parametrize("n,M,precond", [(127, 300, "strang"), (1023, 400, "strang")])
def test_fast_history_equals_direct_sum_on_the_same_ring(n, M, precond):
    """n = 127 runs the one-CTA march, n = 1023 the whole grid; levels up to the third block."""
    P = solver_module()
    prob = W.config_small(n=n, M=M, preconditioner=precond)
    s = P.Solver.from_problem(prob, fast_history=True)
    s.step(M)
    levels = [s.get_level(k)[0] for k in range(M + 1)]
    worst, rel = 0.0, 0.0
    for j in (1, 2, B - 1, B, B + 1, 2 * B - 1, 2 * B, 2 * B + 7, M - 1, M):
        hf = s.history_sum(j)
        hd = s.history_sum(j, direct=True)
        if j < B:
            assert np.array_equal(hf, hd), j     # below the first block both are the direct sum
            continue
        ratio = float(np.max(np.abs(hf - hd) / _fft_bound(prob, levels, j)))
        worst = max(worst, ratio)
        rel = max(rel, float(np.linalg.norm(hf - hd) / np.linalg.norm(hd)))
        assert ratio <= 1.0, (j, ratio)
    print(f"n={n}: largest |fast - direct| / bound {worst:.3g}, largest relative gap {rel:.3g}")
    s.close()


@pytest.mark.parametrize("n,M", [(127, 300), (511, 280)])
def test_fast_history_march_matches_oracle(n, M):
    """Every 20th level and the last within 1e-10 of elimination; the direct-sum march on the GPU
    within 1e-12 at every level."""
    P = solver_module()
    prob = W.config_small(n=n, M=M)
    ref = O.run(prob)
    sf = P.Solver.from_problem(prob, fast_history=True)
    sd = P.Solver.from_problem(prob)
    sf.step(M)
    sd.step(M)
    for j in list(range(0, M + 1, 20)) + [M]:
        uf, ud = sf.get_level(j)[0], sd.get_level(j)[0]
        assert rel_l2(uf, ref[j]) <= 1e-10, (j, rel_l2(uf, ref[j]))
        assert rel_l2(uf, ud) <= 1e-12, (j, rel_l2(uf, ud))
    # a launch boundary inside a block rebuilds the block's far part: levels in chunks of 50
    sc = P.Solver.from_problem(prob, fast_history=True, levels_per_launch=50)
    sc.step(M)
    assert rel_l2(sc.get_level(M)[0], sf.get_level(M)[0]) <= 1e-13
    for o in (sf, sd, sc):
        o.close()


def test_fast_history_history_workload_full_size():
    """n = 2^18 - 1, M = 8192 (the history-dominated workload's first instance) with fast
    history: levels up to 2B + 2 (two block boundaries crossed); sampled rows of the level
    equations of levels 2B .. 2B+1 checked by the oracle row by row (the history evaluated
    directly by the oracle from the levels), and the fast sum against the direct sum on the same
    ring at j = 2B + 1."""
    from test_gpu_fullsize import _check_levels
    P = solver_module()
    prob = W.config_history()[0]
    s = P.Solver.from_problem(prob, source="separable", fast_history=True, autotune=True)
    J = 2 * B + 2
    s.step(J)
    levels = [s.get_level(k)[0] for k in range(J + 1)]
    hf = s.history_sum(2 * B + 1)
    hd = s.history_sum(2 * B + 1, direct=True)
    assert float(np.max(np.abs(hf - hd) / _fft_bound(prob, levels, 2 * B + 1))) <= 1.0
    _, rs = s.history(J)
    s.close()
    # the oracle's row check needs levels 0..j+1 for level j; the equations of levels 2B and
    # 2B + 1 are evaluated (O(j n) per row for the history)
    _check_levels(prob, levels, rs, seed=9, label="history n=262143, fast history",
                  precision="fp64", first=2 * B)
