"""The history-dominated workload (n = 2^18 - 1, M = 8192; the first instance, alpha = 0.2,
beta = 1.2): the convergence order in tau from the errors against the manufactured solution at
t = T with M/4, M/2 and M levels.

The scheme is second order in tau (Lemma 1, the L2-1_sigma formula) and in h (Lemma 2).  The
marches run in FP64 (CGS to 1e-12; the workload's mixed march gives the same errors to five
digits) with the fast history (blocked FFT convolution in time), as the benchmark of this
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
    """M/4, M/2 and M levels.  The error at T is E(tau) = C tau^2 + E_inf: E_inf, the part that
    does not shrink with tau (the h^2 term and the FP64 rounding of the level solves, about
    kappa(A) u64 on the smooth mode that A^{-1} amplifies most), is about a third of C tau^2 at
    M = 8192.  It does not depend on the CGS tolerance (tol 1e-13 leaves every E unchanged to
    five digits) but on the rounding order: two FFT plans that differ only in their split shift
    E at M/4, M/2 and M alike by 1.4e-11.  So the order is measured by the three-level estimate
    log2((E_{M/4} - E_{M/2}) / (E_{M/2} - E_M)), in which E_inf cancels (2.002 and 2.000 with
    the two plans); the two-level order of (M/4, M/2) is held to the band that |E_inf| <= 1.5e-11
    allows (1.8 to 2.2)."""
    P = solver_module()
    probs = []
    for div in (4, 2, 1):
        q = W.config_history()[0]
        q.M = q.M // div
        probs.append(q)
    e4, e2, e1 = (_error_at_T(P, q) for q in probs)
    co3 = math.log2((e4 - e2) / (e2 - e1))
    co_42, co_21 = math.log2(e4 / e2), math.log2(e2 / e1)
    print(f"E_M/4 = {e4:.6g}, E_M/2 = {e2:.6g}, E_M = {e1:.6g}; three-level CO_tau = {co3:.4f}; "
          f"CO_tau(M/4, M/2) = {co_42:.4f}, CO_tau(M/2, M) = {co_21:.4f}")
    assert 1.95 <= co3 <= 2.05, co3
    assert 1.8 <= co_42 <= 2.2, co_42
    assert e1 < e2 < e4 and e1 < 1e-10
