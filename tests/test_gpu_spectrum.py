"""Spectrum of the preconditioned level matrix through the library's own operators (Figs. 1-2,
Section 4): P^{-1} A assembled column by column from tsfcde_apply (A, then P^{-1}) at Example 1,
N = M = 128, alpha = 0.9, beta = 1.8, and its eigenvalues compared with the oracle's dense
P^{-1} A."""
import numpy as np
import pytest

import oracle as O
import tsfcde_workloads as W
from gpu_common import solver_module

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precond", ["strang", "tchan"])
@pytest.mark.parametrize("j", [0, 1])
def test_preconditioned_spectrum_through_the_library(precond, j):
    P = solver_module()
    prob = W.example1(127, 128, 0.9, 1.8)
    s = P.Solver.from_problem(prob, preconditioner=precond)
    n = prob.n
    G = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        G[:, k] = s.apply("Pinv", j, s.apply("A", j, e))
    s.close()
    A, _ = O.level_matrices(prob, j)
    ref = np.linalg.solve(O.preconditioner_matrix(prob, j, precond), A)
    assert np.linalg.norm(G - ref) <= 1e-12 * np.linalg.norm(ref)
    lam = np.linalg.eigvals(G)
    lam_ref = np.linalg.eigvals(ref)
    # every eigenvalue has a partner in the other spectrum (nearest-neighbour, both ways)
    dist = np.abs(lam[:, None] - lam_ref[None, :])
    assert dist.min(axis=1).max() <= 1e-8 and dist.min(axis=0).max() <= 1e-8
    out = int((np.abs(lam - 1.0) > 1e-3).sum())
    if precond == "strang":
        assert 6 <= out <= 10, out
    assert np.abs(lam).min() > 0.5


def test_tchan_eigenvalue_gap_on_the_large_workload_through_the_library():
    """n = 65535, alpha = 0.3, beta = 1.9, tau = 1/1024 (the large workload), level 0: the
    eigenvalues of P are read back as 1 / FFT(P^{-1} e_0) (P is circulant).  T. Chan's smallest
    |Lambda_P| is thousands of times eta (its zero-frequency eigenvalue is the mean row sum of the
    level operator) while Strang's stays within 20 % of eta; on sin(pi x), where A is near its
    smallest eigenvalue, the Rayleigh quotient of P^{-1} A is below 1e-3 for T. Chan and of order
    1 for Strang; and the march's CGS needs over ten times Strang's iterations per level."""
    P = solver_module()
    prob = W.config_large()
    n = prob.n
    eta = O.eta(prob.alpha, prob.tau, 0)
    e0 = np.zeros(n)
    e0[0] = 1.0
    v = np.sin(np.pi * prob.grid())
    res = {}
    for kind in ("strang", "tchan"):
        with P.Solver.from_problem(prob, source="separable", preconditioner=kind) as s:
            lam = 1.0 / np.fft.fft(s.apply("Pinv", 0, e0))
            rq = float(v @ s.apply("Pinv", 0, s.apply("A", 0, v)) / (v @ v))
            st = s.step(2)
        res[kind] = (float(np.abs(lam).min()), rq, st["total_iterations"] / 2)
    print({k: tuple(f"{x:.4g}" for x in r) for k, r in res.items()})
    assert eta <= res["strang"][0] <= 1.2 * eta, res
    assert res["tchan"][0] >= 1e3 * eta, res
    assert 1.0 <= res["strang"][1] <= 3.0 and res["tchan"][1] <= 1e-3, res
    assert res["tchan"][2] >= 10 * res["strang"][2], res
