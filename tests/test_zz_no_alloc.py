"""tsfcde_apply_operator_static: the operator product for callers that cannot allocate device
memory (it keeps all scratch in a fixed file-scope device array).  Checked, on calls in a row of
different sizes and operators, against the oracle's product of the level matrix with x, row by
row (Eq. (3.3)), and against the context-based tsfcde_apply, at the tolerance of the other
operator tests (1e-12 ||op|| ||x||).  The sizes cover the smallest plans (N = 1 and 2, where the
FFT length is clamped to 8), odd and even N, and the largest N the fixed array allows (16383).
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
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _oracle_product(prob, j, op, x):
    """(op x, an upper bound of ||op||_2): rows of A or B from the oracle (O(n) each)."""
    w = O.wsgd_weights(prob.beta, prob.n + 1)
    y = np.empty(prob.n)
    norm = 0.0
    for i in range(prob.n):
        Arow, Brow = O.level_row(prob, j, i, w)
        row = Arow if op == "A" else Brow
        y[i] = row @ x
        norm = max(norm, float(np.abs(row).sum()))
    return y, norm            # Toeplitz: ||T||_2 <= ||T||_1 = ||T||_inf


def test_static_operator_matches_oracle_and_context_apply():
    torch = pytest.importorskip("torch")
    P = solver_module()
    cases = [(W.example2(1000, 16, 0.7, 1.45), 9, "A"), (W.config_small(n=257, M=8), 3, "B"),
             (W.config_small(n=1, M=4), 1, "A"), (W.config_small(n=2, M=4), 2, "B"),
             (W.config_mixed(n=16383, M=8), 5, "A"), (W.config_large(n=16383, M=8), 0, "B")]
    rng = np.random.default_rng(7)
    for prob, j, op in cases:   # calls in a row, different sizes and operators
        x = rng.standard_normal(prob.n)
        y = _static_product(P, torch, prob, j, op, x)
        assert np.all(np.isfinite(y)), prob.n
        ref, nrm = _oracle_product(prob, j, op, x)
        scale = nrm * np.linalg.norm(x)
        gap = np.linalg.norm(y - ref) / scale
        print(f"N={prob.n} op={op}: |y - oracle| / (||op|| ||x||) = {gap:.3g}")
        assert gap <= 1e-12, (prob.n, gap)
        with P.Solver.from_problem(prob) as s:
            ctx = s.apply(op, j, x)
        assert np.linalg.norm(y - ctx) <= 1e-12 * scale, (prob.n, np.linalg.norm(y - ctx) / scale)


def test_static_operator_rejects_oversize():
    torch = pytest.importorskip("torch")
    P = solver_module()
    xd = torch.zeros(16384, dtype=torch.float64, device="cuda")
    with pytest.raises(P.TsfcdeError) as e:
        P.apply_operator_static(16384, 1.5, 0.7, 1.0, 0.0, 1.0, 1.0, "A", xd.data_ptr(),
                                xd.data_ptr())
    assert e.value.status == 1
