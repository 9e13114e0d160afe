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
