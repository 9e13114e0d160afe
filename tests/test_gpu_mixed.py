"""Mixed precision (FP32 inner CGS inside FP64 iterative refinement) against the FP64 oracle and
the FP64 GPU path: relative L2 gap <= 1e-8 per level."""
import numpy as np
import pytest

import oracle as O
import tsfcde_workloads as W
from gpu_common import rel_l2, solver_module

pytestmark = pytest.mark.gpu


def _levels(P, prob, nlev, **kw):
    s = P.Solver.from_problem(prob, source="separable", **kw)
    out = [s.get_level()[0]]
    stats = []
    for _ in range(nlev):
        stats.append(s.step(1))
        out.append(s.get_level()[0])
    s.close()
    return out, stats


@pytest.mark.parametrize("precond", ["strang", "tchan"])
def test_mixed_small_config_every_level(precond):
    P = solver_module()
    prob = W.config_small(preconditioner=precond)
    ref = O.run(prob)
    got, st = _levels(P, prob, prob.M, precision="mixed")
    assert max(rel_l2(got[j], ref[j]) for j in range(prob.M + 1)) <= 1e-8
    assert sum(s["outer_iterations"] for s in st) >= prob.M


def test_mixed_parameters_of_the_precision_workload():
    """alpha = 0.8, beta = 1.5, gamma = 1, d+- = (1 +- t/2)/2 at n = 1023: first 8 levels."""
    P = solver_module()
    prob = W.config_mixed(n=1023, M=512)
    ref = O.run(prob, levels=8)
    got, st = _levels(P, prob, 8, precision="mixed")
    assert max(rel_l2(got[j], ref[j]) for j in range(9)) <= 1e-8
    assert sum(s["escalated_levels"] for s in st) == 0


def test_mixed_matches_fp64_gpu_path():
    P = solver_module()
    prob = W.config_mixed(n=4095, M=64)
    a, _ = _levels(P, prob, 16, precision="fp64")
    b, st = _levels(P, prob, 16, precision="mixed")
    assert max(rel_l2(b[j], a[j]) for j in range(17)) <= 1e-8


def test_mixed_escalates_when_fp32_cannot_converge():
    """beta = 1.9, alpha = 0.3 at n = 4095 with the inner solve forced to FP32 (u32 * kappa_eff
    ~ 0.3: each refinement step gains little) and one refinement step allowed: the levels must be
    finished by the FP64 CGS from the current iterate and still match FP64."""
    P = solver_module()
    prob = W.config_large(n=4095, M=1024, preconditioner="strang")
    a, _ = _levels(P, prob, 6, precision="fp64")
    b, st = _levels(P, prob, 6, precision="mixed", inner="fp32", outer_maxit=1)
    assert max(rel_l2(b[j], a[j]) for j in range(7)) <= 1e-8
    assert sum(s["escalated_levels"] for s in st) >= 1


@pytest.mark.parametrize("n,precond", [(4095, "strang"), (4095, "tchan"), (65535, "strang")])
def test_float_float_inner_where_fp32_fails(n, precond):
    """Same operator family (beta = 1.9), float-float inner solve: no escalation, and the result
    matches the FP64 GPU path to 1e-8."""
    P = solver_module()
    prob = W.config_large(n=n, M=1024, preconditioner=precond)
    a, _ = _levels(P, prob, 4, precision="fp64")
    b, st = _levels(P, prob, 4, precision="mixed", inner="ff")
    assert max(rel_l2(b[j], a[j]) for j in range(5)) <= 1e-8
    assert sum(s["escalated_levels"] for s in st) == 0


def test_float_float_small_config_every_level():
    P = solver_module()
    prob = W.config_small()
    ref = O.run(prob)
    got, st = _levels(P, prob, prob.M, precision="mixed", inner="ff")
    assert max(rel_l2(got[j], ref[j]) for j in range(prob.M + 1)) <= 1e-8
    assert sum(s["escalated_levels"] for s in st) == 0


def test_mixed_tchan_large_never_worse_than_fp64():
    """T. Chan at n = 65535 (hundreds of CGS iterations per solve, irregular convergence): inner
    solves that fail to converge return their minimum-residual iterate, so no refinement step can
    make x worse; every level must still match the FP64 path to 1e-8."""
    P = solver_module()
    prob = W.config_large(n=65535, M=1024, preconditioner="tchan")
    a, _ = _levels(P, prob, 6, precision="fp64")
    b, st = _levels(P, prob, 6, precision="mixed")
    assert max(rel_l2(b[j], a[j]) for j in range(7)) <= 1e-8
    assert max(s["max_residual"] for s in st) < 1e-6


def test_floor_flag_marks_levels_accepted_above_tol():
    """Each mixed level either reaches tol, or is accepted at its FP64 residual floor (counted in
    floor_levels, residual between tol and the floor), or is finished by the FP64 CGS.  tol is
    set to 1e-15, below the floor 64 u64 kappa_eff of computing g - A x in FP64 (about 1e-7 at
    n = 2^20 - 1, beta = 1.5), so the floor rule must act: at most 64 u64 kappa_eff, and no
    level may be left above it."""
    P = solver_module()
    prob = W.config_mixed(M=8)              # n = 2^20 - 1
    tol = 1e-15
    s = P.Solver.from_problem(prob, source="separable", precision="mixed", tol=tol)
    floors = 0
    for _ in range(4):
        st = s.step(1)
        assert st["floor_levels"] in (0, 1) and st["escalated_levels"] in (0, 1)
        assert st["floor_levels"] + st["escalated_levels"] <= 1
        if st["floor_levels"]:
            floors += 1
            assert tol <= st["max_residual"] < 1e-6
        elif not st["escalated_levels"]:
            assert st["max_residual"] < tol
    s.close()
    assert floors >= 1
