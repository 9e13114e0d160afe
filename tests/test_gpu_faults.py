"""Failure detection without any GPU fault: bounded device waits report E_TIMEOUT and leave the
context usable; breakdown/argument errors surface as status codes."""
import numpy as np
import pytest

import oracle as O
import tsfcde_workloads as W
from gpu_common import rel_l2, solver_module

pytestmark = pytest.mark.gpu


def test_barrier_wait_times_out_and_context_recovers():
    """CTA 0 skips its first grid-barrier arrival (testing hook, one launch only); every other
    CTA's wait runs into its bound (2^16 polls) and the call returns E_TIMEOUT.  The same
    context then resets and marches normally, matching the oracle.  n=511 (FFT half-length 512)
    so that the march runs on the whole grid: up to half-length 256 it runs in one CTA, which
    has no grid barrier."""
    P = solver_module()
    prob = W.config_small(n=511, M=6)
    s = P.Solver.from_problem(prob, barrier_spin_log2=16, test_skip_arrival=True)
    with pytest.raises(P.TsfcdeError) as e:
        s.step(1)
    assert e.value.status == 8                     # TSFCDE_E_TIMEOUT
    assert s.get_level()[1] == 0                   # the failed call advanced nothing
    s.reset()
    for _ in range(prob.M):
        s.step(1)
    ref = O.run(prob)
    assert rel_l2(s.get_level()[0], ref[-1]) <= 1e-10
    s.close()


def test_maxit_reports_not_converged_and_keeps_state():
    P = solver_module()
    prob = W.config_small(M=3, preconditioner="none")
    s = P.Solver.from_problem(prob, maxit=2)
    st = s.step(3)
    assert st["status"] == 5 and st["max_iterations"] == 2   # E_NOT_CONVERGED, state kept
    assert s.get_level()[1] == 3
    s.close()


def test_stepping_past_M_is_a_state_error():
    P = solver_module()
    prob = W.config_small(M=2)
    s = P.Solver.from_problem(prob)
    s.step(2)
    with pytest.raises(P.TsfcdeError) as e:
        s.step(1)
    assert e.value.status == 9
    s.close()
