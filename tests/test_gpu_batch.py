"""Batched instances (one CTA per instance, CTA-local level solves) against the FP64 oracle, per
instance, at several levels; and against the single-instance GPU path."""
import numpy as np
import pytest

import oracle as O
import tsfcde_workloads as W
from gpu_common import rel_l2, solver_module

pytestmark = pytest.mark.gpu


def _small_batch(count=24, M=12, seed=5):
    return W.config_batch(count=count, M=M, seed=seed, n_lo=7, n_hi=300)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-8)])
def test_batch_against_oracle(precision, tol):
    P = solver_module()
    probs = _small_batch()
    M = probs[0].M
    refs = [O.run(p) for p in probs]
    with P.Batch(probs, M, precision=precision) as b:
        for j0, j1 in ((0, 1), (1, 5), (5, M)):    # several calls: commit across launches
            b.step(j1 - j0)
            for i, p in enumerate(probs):
                u, lev = b.get_level(i)
                assert lev == j1
                assert rel_l2(u, refs[i][j1]) <= tol, (i, p.n, j1, rel_l2(u, refs[i][j1]))
        it, rs = b.history(0, M)
        assert np.all(it > 0) and np.all(rs < 1e-12)


def test_batch_equals_single_instance_path():
    P = solver_module()
    probs = W.config_batch(count=6, M=8, seed=11, n_lo=255, n_hi=4095)
    with P.Batch(probs, 8) as b:
        b.step(8)
        got = [b.get_level(i)[0] for i in range(len(probs))]
    for i, p in enumerate(probs):
        with P.Solver(p.a, p.b, p.T, p.n, 8, p.alpha, p.beta, p.gamma, p.d_plus, p.d_minus,
                      p.phi) as s:
            ref = s.solve()
        assert rel_l2(got[i], ref) <= 1e-10


def test_batch_reset_and_tchan():
    P = solver_module()
    probs = _small_batch(count=9, M=6, seed=3)
    refs = [O.run(p) for p in probs]
    with P.Batch(probs, 6, preconditioner="tchan") as b:
        b.step(6)
        b.reset()
        b.step(6)
        for i in range(len(probs)):
            assert rel_l2(b.get_level(i)[0], refs[i][6]) <= 1e-10


@pytest.mark.parametrize("algorithm", ["ids", "ids-const"])
def test_autotuned_batch_plan_matches_oracle(algorithm):
    """The batch plan tuner tries chunk budgets and split orientations on the first two levels;
    the states then restart from level 0 and the march with the kept plan matches elimination
    within 1e-10, or, where the instance's conditioning does not allow 1e-10, within the forward
    error its stopping rule allows: each level's relative residual is below tol (PCGS) or below
    max(tol, 64 u64 kappa) (constant-coefficient levels), so each level's relative error is at
    most cond(A) times that, summed over the M levels.  cond(A) comes from the oracle's dense A,
    so the bound uses nothing the GPU reported."""
    P = solver_module()
    probs = W.config_batch(count=12, M=6, seed=7, n_lo=200, n_hi=2100)
    b = P.Batch(probs, 6, algorithm=algorithm, autotune=True)
    plan = b.plan()
    assert plan["budget"] in (1024, 2048, 4096) and plan["best_ms"] > 0 and plan["ctas"] >= 152
    assert b.get_level(0)[1] == 0
    b.step(6)
    for i, q in enumerate(probs):
        ref = O.run(q)
        bound = _stopping_rule_bound(q, algorithm)
        gap = rel_l2(b.get_level(i)[0], ref[-1])
        print(f"instance {i} n={q.n}: gap {gap:.3g}, bound {bound:.3g}")
        assert gap <= bound, (i, q.n, gap, bound)
    b.close()


def _stopping_rule_bound(q, algorithm, tol=1e-12):
    """max(1e-10, sum over levels of cond(A_j) * rho_j) with rho_j the residual the level's
    stopping rule allows (tol for PCGS; max(tol, 64 u64 ||A_j||_1 / eta_j) for a
    Gohberg-Semencul level), all from the oracle's dense level matrices."""
    tot = 0.0
    for j in range(q.M):
        A = O.level_matrices(q, j)[0]
        rho = tol
        if algorithm == "ids-const" and j >= 1:
            rho = max(tol, 64 * 2.0 ** -53 * np.abs(A).sum(axis=1).max() / O.level_scalars(q, j)[0])
        tot += np.linalg.cond(A) * rho
    return max(1e-10, tot)


def test_contexts_of_different_sizes_coexist():
    """A context set up after another with smaller instances must not lower the shared-memory
    limit the first one launches with (the limit is a per-kernel, process-wide attribute)."""
    P = solver_module()
    big = W.config_batch(count=3, M=3, seed=3, n_lo=8000, n_hi=16383)
    small = W.config_batch(count=3, M=3, seed=4, n_lo=15, n_hi=40)
    b1 = P.Batch(big, 3)
    b2 = P.Batch(small, 3)
    b2.step(3)
    b1.step(3)
    s1 = P.Solver.from_problem(W.config_small(n=255, M=3))
    s2 = P.Solver.from_problem(W.config_small(n=31, M=3))
    s2.step(3)
    s1.step(3)
    for i, q in enumerate(small):
        assert rel_l2(b2.get_level(i)[0], O.run(q)[-1]) <= 1e-10
    assert rel_l2(s1.get_level()[0], O.run(W.config_small(n=255, M=3))[-1]) <= 1e-10
    for o in (b1, b2, s1, s2):
        o.close()


def test_batch_solve_equals_step_and_get():
    P = solver_module()
    probs = W.config_batch(count=5, M=6, n_lo=255, n_hi=1100)
    b = P.Batch(probs, 6)
    u = b.solve()
    assert b.last_stats["level"] == 6 and len(u) == len(probs)
    b.reset()
    b.step(6)
    for i in range(len(probs)):
        assert np.array_equal(u[i], b.get_level(i)[0])
        assert rel_l2(u[i], O.run(probs[i])[-1]) <= 1e-10
    b.close()


def test_contexts_release_device_memory():
    """Creating and freeing contexts and batches returns their device memory."""
    torch = pytest.importorskip("torch")
    P = solver_module()
    probs = W.config_batch(count=64, M=4, n_lo=255, n_hi=4095)
    # warm: library load, kernel modules and the first allocations of the process
    P.Batch(probs, 4).close()
    P.Solver.from_problem(W.config_small(n=65535, M=4)).close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(8):
        b = P.Batch(probs, 4)
        b.step(2)
        b.close()
        s = P.Solver.from_problem(W.config_small(n=65535, M=4))
        s.step(2)
        s.close()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (16 << 20), (free0 - free1) / 2**20
