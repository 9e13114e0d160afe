"""tsfcde_apply_operator_static: the operator product for callers that cannot allocate device
memory (it keeps all scratch in a fixed file-scope device array).  Checked against the
context-based tsfcde_apply on two calls in a row, at the tolerance of the other operator tests.
This file is collected last on purpose."""
import numpy as np
import pytest

import oracle as O
import tsfcde_workloads as W
from gpu_common import solver_module

pytestmark = pytest.mark.gpu


def _static_product(P, torch, prob, j, op, x):
    sigma = 1.0 - prob.alpha / 2.0
    eta, q, kp, km = O.level_scalars(prob, j)
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.full((prob.n,), float("nan"), dtype=torch.float64, device="cuda")
    P.apply_operator_static(prob.n, prob.beta, sigma, eta, q, kp, km, op, xd.data_ptr(),
                            yd.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return yd.cpu().numpy()


def test_static_operator_matches_context_apply_twice():
    torch = pytest.importorskip("torch")
    P = solver_module()
    cases = [(W.example2(1000, 16, 0.7, 1.45), 9, "A"), (W.config_small(n=257, M=8), 3, "B")]
    rng = np.random.default_rng(7)
    for prob, j, op in cases:   # two calls in a row, different sizes and operators
        x = rng.standard_normal(prob.n)
        with P.Solver.from_problem(prob) as s:
            ref = s.apply(op, j, x)
        y = _static_product(P, torch, prob, j, op, x)
        A, B = O.level_matrices(prob, j)
        scale = np.linalg.norm(A if op == "A" else B, 2) * np.linalg.norm(x)
        assert np.all(np.isfinite(y))
        assert np.linalg.norm(y - ref) <= 1e-12 * scale, np.linalg.norm(y - ref) / scale


def test_static_operator_rejects_oversize():
    torch = pytest.importorskip("torch")
    P = solver_module()
    xd = torch.zeros(16384, dtype=torch.float64, device="cuda")
    with pytest.raises(P.TsfcdeError) as e:
        P.apply_operator_static(16384, 1.5, 0.7, 1.0, 0.0, 1.0, 1.0, "A", xd.data_ptr(),
                                xd.data_ptr())
    assert e.value.status == 1
