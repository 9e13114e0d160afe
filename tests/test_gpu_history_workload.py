"""The history-dominated workload as specified (n = 2^18 - 1, M = 8192, mixed precision with FP64
history; the first instance, alpha = 0.2, beta = 1.2): the convergence order in tau from the
errors against the manufactured solution at t = T with M/2 and M levels.

The scheme is second order in tau (Lemma 1, the L2-1_sigma formula) and in h (Lemma 2); at
h = 2^-18 the h^2 term (1.5e-11 relative) is far below tau^2 (1.5e-8), so
CO_tau = log2(E_{M/2} / E_M) must be close to 2.  The marches use the fast history (blocked FFT
convolution in time), which the benchmark of this workload uses; its agreement with the direct
sum is tested in test_gpu_fast_history.py."""
import math

import numpy as np
import pytest

import tsfcde_workloads as W
from gpu_common import solver_module

pytestmark = pytest.mark.gpu


def _error_at_T(P, prob):
    with P.Solver.from_problem(prob, source="separable", precision="mixed", fast_history=True) as s:
        st = s.step(prob.M)
        assert st["status"] == 0, st
        u = s.get_level(prob.M)[0]
    return float(np.sqrt(prob.h) * np.linalg.norm(u - prob.exact(prob.grid(), prob.T)))


def test_history_workload_convergence_order_in_tau():
    P = solver_module()
    full = W.config_history()[0]
    half = W.config_history()[0]
    half.M = full.M // 2
    e_full, e_half = _error_at_T(P, full), _error_at_T(P, half)
    co = math.log2(e_half / e_full)
    print(f"E_M/2 = {e_half:.4g}, E_M = {e_full:.4g}, CO_tau = {co:.4f}")
    assert 1.9 <= co <= 2.15, co
    # against the solution's size (u(., T) ~ 2 X, ||X||_L2 ~ 0.03): the scheme's error at M
    assert e_full < 1e-9
