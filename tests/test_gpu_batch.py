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
    the states then restart from level 0 and the march with the kept plan matches elimination."""
    P = solver_module()
    probs = W.config_batch(count=12, M=6, seed=7, n_lo=200, n_hi=2100)
    b = P.Batch(probs, 6, algorithm=algorithm, autotune=True)
    plan = b.plan()
    assert plan["budget"] in (1024, 2048, 4096) and plan["best_ms"] > 0 and plan["ctas"] >= 152
    assert b.get_level(0)[1] == 0
    b.step(6)
    for i, q in enumerate(probs):
        ref = O.run(q)
        assert rel_l2(b.get_level(i)[0], ref[-1]) <= 1e-10, (i, q.n)
    b.close()
