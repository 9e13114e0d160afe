"""Constant-coefficient path (TSFCDE_ALG_IDS_CONST) against the oracle.

Algorithm "Practical implementation of IDS with constant coefficients" (Section 3.2): level 0 by
the preconditioned CGS; levels j >= 1 by the Gohberg-Semencul formula (Eq. (3.6)) applied
as in Algorithm "Compute z = A^{-1} v".  The level solutions are the same as the plain scheme's,
so the oracle is the plain elimination march (oracle.run); FP64 tolerance 1e-10 per level, as for
the CGS path.  The generators x = A^{-1} e_1, y = A^{-1} e_n are checked through op 3
(y = A^{-1} x) against LAPACK's solve on the level matrix.
"""
import numpy as np
import pytest

import oracle as O
import tsfcde_workloads as W
from gpu_common import rel_l2, solver_module

pytestmark = pytest.mark.gpu


def _march(P, prob, **kw):
    s = P.Solver.from_problem(prob, algorithm="ids-const", **kw)
    levels = [s.get_level()[0]]
    stats = []
    for _ in range(prob.M):
        stats.append(s.step(1))
        levels.append(s.get_level()[0])
    return s, levels, stats


def _batch_instance(n, M, idx=0, seed=1603):
    return W.config_batch(count=idx + 1, M=M, seed=seed, n_lo=n, n_hi=n)[idx]


@pytest.mark.parametrize("n,precond", [(255, "strang"), (511, "strang"), (511, "tchan"),
                                       (1023, "strang")])
def test_const_march_matches_oracle_every_level(n, precond):
    """n = 255 runs the one-CTA march, n >= 511 the whole-grid march."""
    P = solver_module()
    prob = _batch_instance(n, 12, idx=2)
    ref = O.run(prob)
    s, got, stats = _march(P, prob, preconditioner=precond)
    gaps = [rel_l2(got[j], ref[j]) for j in range(prob.M + 1)]
    assert max(gaps) <= 1e-10, gaps
    assert stats[0]["gsf_levels"] == 0 and all(st["gsf_levels"] == 1 for st in stats[1:])
    # level 1 reports the two generator solves; later levels run no Krylov iteration
    it, rs = s.history(prob.M)
    assert it[1] > 0 and np.all(it[2:] == 0)
    assert np.all(rs[1:] < 1e-9)
    s.close()


def test_const_one_launch_equals_stepwise_and_oracle():
    P = solver_module()
    prob = _batch_instance(700, 10, idx=5)
    s1 = P.Solver.from_problem(prob, algorithm="ids-const")
    st = s1.step(prob.M)
    u1 = s1.get_level()[0]
    assert st["gsf_levels"] == prob.M - 1 and st["device_launches"] == 1
    s2 = P.Solver.from_problem(prob, algorithm="ids-const", levels_per_launch=1)
    s2.step(prob.M)
    u2 = s2.get_level()[0]
    assert np.array_equal(u1, u2)   # same passes, deterministic reductions
    ref = O.run(prob)
    assert rel_l2(u1, ref[-1]) <= 1e-10
    s1.close()
    s2.close()


def test_const_matches_cgs_path():
    P = solver_module()
    prob = _batch_instance(2047, 16, idx=1)
    a = P.Solver.from_problem(prob)
    b = P.Solver.from_problem(prob, algorithm="ids-const")
    ua, ub = a.solve(), b.solve()
    assert rel_l2(ub, ua) <= 1e-10
    a.close()
    b.close()


@pytest.mark.parametrize("n", [1, 2, 3, 8, 33])
def test_const_tiny_sizes(n):
    P = solver_module()
    prob = _batch_instance(n, 6, idx=0) if n >= 3 else W.example1(n, 6, 0.4, 1.5)
    ref = O.run(prob)
    s, got, _ = _march(P, prob)
    assert max(rel_l2(got[j], ref[j]) for j in range(prob.M + 1)) <= 1e-10
    s.close()


def test_gs_inverse_operator_matches_lapack():
    P = solver_module()
    prob = _batch_instance(600, 4, idx=3)
    s = P.Solver.from_problem(prob, algorithm="ids-const")
    v = np.random.default_rng(11).standard_normal(prob.n)
    with pytest.raises(P.TsfcdeError) as e:
        s.apply("Ainv_gs", 0, v)            # generators not built yet
    assert e.value.status == 9
    s.step(2)
    A, _ = O.level_matrices(prob, 1)
    z = s.apply("Ainv_gs", 0, v)
    assert rel_l2(z, np.linalg.solve(A, v)) <= 1e-11
    # A (A^{-1} v) = v through the library's own operator product
    assert rel_l2(s.apply("A", 1, z), v) <= 1e-11
    s.close()


def test_const_rejects_time_dependent_coefficients():
    P = solver_module()
    prob = W.config_small(M=4)              # d_+ = 1 + t varies between levels
    with pytest.raises(P.TsfcdeError) as e:
        P.Solver.from_problem(prob, algorithm="ids-const")
    assert e.value.status == 1


def test_const_example1_table1():
    """Paper Example 1 (constant coefficients) at N = M = 128 by the constant-coefficient
    algorithm: Table 1's error 1.6010e-5 (alpha = 0.1, beta = 1.8) to 0.5 %."""
    P = solver_module()
    prob = W.example1(127, 128, 0.1, 1.8)
    s, levels, _ = _march(P, prob)
    e2, em = O.errors_vs_exact(prob, levels)
    assert abs(e2 / 1.6010e-5 - 1) < 0.005 and abs(em / 2.3815e-5 - 1) < 0.005
    s.close()


def test_const_reset_reruns_identically():
    P = solver_module()
    prob = _batch_instance(1023, 8, idx=4)
    s = P.Solver.from_problem(prob, algorithm="ids-const")
    u1 = s.solve().copy()
    s.reset()
    u2 = s.solve()
    assert np.array_equal(u1, u2)
    s.close()


def test_const_mixed_level0_then_gs():
    """Mixed precision changes only level 0 (the only CGS level); later levels are FP64 GS."""
    P = solver_module()
    prob = _batch_instance(1023, 8, idx=6)
    ref = O.run(prob)
    s, got, _ = _march(P, prob, precision="mixed")
    assert max(rel_l2(got[j], ref[j]) for j in range(prob.M + 1)) <= 1e-8
    s.close()


def test_const_batch_matches_oracle():
    P = solver_module()
    probs = W.config_batch(count=6, M=8, n_lo=255, n_hi=1100)
    b = P.Batch(probs, 8, algorithm="ids-const")
    st = b.step(8)
    assert st["gsf_levels"] == 6 * 7
    for i, p in enumerate(probs):
        ref = O.run(p)
        assert rel_l2(b.get_level(i)[0], ref[-1]) <= 1e-10, i
    b.close()


@pytest.mark.parametrize("M", [1, 2, 3])
def test_const_shortest_marches(M):
    """M = 1 has no level j >= 1 (plain CGS only); M = 2 builds the generators for its single
    Gohberg-Semencul level; M = 3 uses them once more."""
    # with tau = T/M this large, eta_j is small and the levels are far worse conditioned than in
    # the marches above: the bound is 1e-10, or the forward error the stopping rules allow,
    # sum_j cond(A_j) rho_j, from the oracle's dense matrices (rho_j = tol for the CGS level 0,
    # max(tol, 64 u64 ||A||_1 / eta) for the Gohberg-Semencul levels)
    def bound(q, _unused=None, tol=1e-12):
        tot = 0.0
        for j in range(q.M):
            A = O.level_matrices(q, j)[0]
            rho = tol if j == 0 else max(tol, 64 * 2.0 ** -53 * np.abs(A).sum(axis=1).max()
                                         / O.level_scalars(q, j)[0])
            tot += np.linalg.cond(A) * rho
        return max(1e-10, tot)

    P = solver_module()
    prob = _batch_instance(300, M, idx=1)
    ref = O.run(prob)
    s = P.Solver.from_problem(prob, algorithm="ids-const")
    st = s.step(M)
    assert st["gsf_levels"] == M - 1
    assert rel_l2(s.get_level()[0], ref[-1]) <= bound(prob, st["max_residual"])
    s.close()
    probs = W.config_batch(count=3, M=M, n_lo=255, n_hi=1100)
    b = P.Batch(probs, M, algorithm="ids-const")
    st = b.step(M)
    assert st["gsf_levels"] == 3 * (M - 1)
    for i, q in enumerate(probs):
        _, rs = b.history(i, M)
        assert rel_l2(b.get_level(i)[0], O.run(q)[-1]) <= bound(q, float(rs.max()))
    b.close()
