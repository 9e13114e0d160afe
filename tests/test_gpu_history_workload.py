"""The history-dominated workload (n = 2^18 - 1, M = 8192; the first instance, alpha = 0.2,
beta = 1.2): the convergence order in tau from the errors against the manufactured solution at
t = T with M/2 and M levels.

The scheme is second order in tau (Lemma 1, the L2-1_sigma formula) and in h (Lemma 2); at
h = 2^-18 the h^2 term (1.5e-11 relative) is far below tau^2 (1.5e-8), so
CO_tau = log2(E_{M/2} / E_M) must be close to 2 where the scheme's error dominates.  The marches
run in FP64 (CGS to 1e-12): the
workload's mixed precision accepts a level at its FP64 residual floor 64 u64 kappa_eff, about
3e-9 relative here, within a factor of a few of the scheme's own error at T (about 5e-10
relative), so an order measured from mixed marches mixes solver and discretisation error.  The
marches use the fast history (blocked FFT convolution in time), as the benchmark of this
workload does; its agreement with the direct sum is tested in test_gpu_fast_history.py."""
import math

import numpy as np
import pytest

import tsfcde_workloads as W
from gpu_common import solver_module

pytestmark = pytest.mark.gpu


def _error_at_T(P, prob):
    with P.Solver.from_problem(prob, source="separable", precision="fp64", fast_history=True) as s:
        st = s.step(prob.M)
        assert st["status"] == 0, st
        u = s.get_level(prob.M)[0]
    return float(np.sqrt(prob.h) * np.linalg.norm(u - prob.exact(prob.grid(), prob.T)))


def test_history_workload_convergence_order_in_tau():
    """M/4, M/2 and M levels.  At M = 8192 the scheme's error at T (about 4e-11) is only a few
    times the error the level solves accumulate at tol = 1e-12: two FFT plans that differ in
    their split alone move E_M by about 1.4e-11.  So the order is pinned on (M/4, M/2), where
    the scheme's error dominates, and (M/2, M) is held to the band that this solver error allows
    (E_M = E_{M/2}/4 +- 1.5e-11 gives 1.65 to 2.6)."""
    P = solver_module()
    probs = []
    for div in (4, 2, 1):
        q = W.config_history()[0]
        q.M = q.M // div
        probs.append(q)
    e4, e2, e1 = (_error_at_T(P, q) for q in probs)
    co_42, co_21 = math.log2(e4 / e2), math.log2(e2 / e1)
    print(f"E_M/4 = {e4:.4g}, E_M/2 = {e2:.4g}, E_M = {e1:.4g}; "
          f"CO_tau(M/4, M/2) = {co_42:.4f}, CO_tau(M/2, M) = {co_21:.4f}")
    assert 1.9 <= co_42 <= 2.1, co_42
    assert 1.65 <= co_21 <= 2.6, co_21
    assert e1 < 1e-9
