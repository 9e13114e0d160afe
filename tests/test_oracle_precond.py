"""Pins of the oracle's circulant preconditioners (Eq. (3.7)) and its dense PCGS."""
import numpy as np
import pytest
from scipy.linalg import toeplitz

import oracle as O
import tsfcde_workloads as W


def _rand_toeplitz(n, seed):
    rng = np.random.default_rng(seed)
    col, row = rng.standard_normal(n), rng.standard_normal(n)
    row[0] = col[0]
    return toeplitz(col, row)


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_circulant_fixed_points(n):
    c = np.random.default_rng(n).standard_normal(n)
    C = O.circulant_from_column(c)
    np.testing.assert_allclose(O.strang_column(C), c)
    np.testing.assert_allclose(O.tchan_column(C), c)


def test_strang_copies_central_diagonals():
    T = _rand_toeplitz(7, 3)
    t = O.toeplitz_diagonals(T)
    c = O.strang_column(T)
    np.testing.assert_array_equal(c, [t[0], t[1], t[2], t[3], t[-3], t[-2], t[-1]])


@pytest.mark.parametrize("n", [4, 7])
def test_tchan_is_frobenius_optimal(n):
    """T. Chan's circulant minimises ||C - T||_F over circulants: least squares in the basis of
    the n cyclic shift matrices."""
    T = _rand_toeplitz(n, n)
    basis = [O.circulant_from_column(np.eye(n)[k]) for k in range(n)]
    Amat = np.stack([b.ravel() for b in basis], axis=1)
    coef = np.linalg.lstsq(Amat, T.ravel(), rcond=None)[0]
    np.testing.assert_allclose(O.tchan_column(T), coef, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("kind", ["strang", "tchan"])
def test_preconditioner_is_circulant_approx_of_A(kind):
    """Eq. (3.7) applies s(.) to Q, W, W^T term by term; s is linear, so P = s(A)."""
    p = W.config_small(n=21, M=8, preconditioner=kind)
    A, _ = O.level_matrices(p, 2)
    col = O.strang_column if kind == "strang" else O.tchan_column
    np.testing.assert_allclose(O.preconditioner_matrix(p, 2), O.circulant_from_column(col(A)),
                               rtol=1e-12, atol=1e-9)


@pytest.mark.parametrize("kind", ["strang", "tchan"])
@pytest.mark.parametrize("n", [5, 8, 21])
def test_transpose_term_reading(kind, n):
    """s(W)^T (used for the W^T term, as the conj(Lambda_beta) of the diagonalisation after
    Eq. (3.7) states) equals the circulant approximation of W^T for odd n and for T. Chan;
    its eigenvalues are the conjugates of those of s(W)."""
    W_ = O.matrix_W(1.6, n)
    col = O.strang_column if kind == "strang" else O.tchan_column
    sW = O.circulant_from_column(col(W_))
    direct = O.circulant_from_column(col(W_.T))
    if n % 2 == 1 or kind == "tchan":
        np.testing.assert_allclose(sW.T, direct, atol=1e-15)
    lam = np.fft.fft(col(W_))
    lamT = np.fft.fft(sW.T[:, 0])
    np.testing.assert_allclose(lamT, np.conj(lam), atol=1e-13)


@pytest.mark.parametrize("kind", ["strang", "tchan"])
def test_preconditioner_nonsingular(kind):
    """Theorem 4: Re(Lambda_P) > 0."""
    p = W.config_small(n=63, M=16, preconditioner=kind)
    P = O.preconditioner_matrix(p, 0)
    lam = np.linalg.eigvals(P)
    assert np.min(lam.real) > 0


def _level_rhs(p, lv, j):
    import math
    A, B = O.level_matrices(p, j)
    sigma = 1 - p.alpha / 2
    g = B @ lv[j] + p.f(p.grid(), (j + sigma) * p.tau)
    c = O.c_coeffs(p.alpha, j)
    hist = sum(c[j - s] * (lv[s + 1] - lv[s]) for s in range(j)) if j else 0.0
    return A, g - p.tau ** (-p.alpha) / math.gamma(2 - p.alpha) * hist


@pytest.mark.parametrize("maker,beta,j", [(W.example1, 1.8, 0), (W.example1, 1.8, 1),
                                          (W.example1, 1.8, 40), (W.example2, 1.5, 64),
                                          (W.example2, 1.5, 127)])
def test_pcgs_iterations_in_paper_range(maker, beta, j):
    """Section 3.2 / Figs. 1-4: Strang-preconditioned CGS needs 6-10 iterations at N = M = 128,
    alpha = 0.9 (Example 2's first levels have d+- ~ sin t ~ 0 and need fewer); the solution
    equals the GE solution."""
    p = maker(127, 128, 0.9, beta)
    lv = O.run(p, levels=j + 1)
    A, g = _level_rhs(p, lv, j)
    sol, its, _ = O.pcgs(A, g, O.preconditioner_matrix(p, j, "strang"))
    assert 6 <= its <= 10, its
    np.testing.assert_allclose(sol, lv[j + 1], rtol=1e-10, atol=1e-13)


def test_pcgs_without_preconditioner_is_slow():
    p = W.example1(127, 128, 0.9, 1.8)
    A, B = O.level_matrices(p, 0)
    g = B @ p.phi(p.grid())
    _, its, _ = O.pcgs(A, g, None, maxit=60)
    assert its == 60


@pytest.mark.parametrize("j", [0, 1])
def test_preconditioned_spectrum_clusters_at_one(j):
    """Figs. 1-2 (Section 4): Example 1 at N = M = 128, alpha = 0.9, beta = 1.8, levels j = 0, 1.
    The eigenvalues of P^{-1} A (Strang) cluster at 1 except for about 6-10 outliers and stay
    away from 0, while those of A spread over two orders of magnitude.  Outlier reading:
    |lambda - 1| > 1e-3 (the paper gives no threshold)."""
    prob = W.example1(127, 128, 0.9, 1.8)
    A, _ = O.level_matrices(prob, j)
    P = O.preconditioner_matrix(prob, j, "strang")
    lam = np.linalg.eigvals(np.linalg.solve(P, A))
    lamA = np.abs(np.linalg.eigvals(A))
    outliers = int((np.abs(lam - 1.0) > 1e-3).sum())
    assert 6 <= outliers <= 10, outliers
    assert np.abs(lam).min() > 0.5
    assert lamA.max() / lamA.min() > 100.0


def test_tchan_misses_the_smallest_eigenvalues_on_the_large_workload():
    """The large workload's coefficients (alpha = 0.3, beta = 1.9, tau = 1/1024) at n = 1023.
    T. Chan's circulant averages each diagonal with its wrapped partner, so its zero-frequency
    eigenvalue is the mean row sum (1/n) 1^T P 1, which the boundary rows of the fractional
    operator make large: min|Lambda_P| is far above eta, while Strang's stays near eta.  On the
    smoothest mode sin(pi x), where A is near its smallest eigenvalue, P^{-1} A is then far below
    1 for T. Chan and of order 1 for Strang, and CGS needs several times Strang's iterations.
    (At n = 65535 the same gap grows to 6.9e4 against eta = 7.86.)"""
    p = W.config_large(n=1023, M=1024)
    A, B = O.level_matrices(p, 0)
    eta = O.eta(p.alpha, p.tau, 0)
    sigma = 1 - p.alpha / 2
    g = B @ p.phi(p.grid()) + p.f(p.grid(), sigma * p.tau)
    v = np.sin(np.pi * p.grid())
    out = {}
    for kind in ("strang", "tchan"):
        P = O.preconditioner_matrix(p, 0, kind)
        lam_min = float(np.abs(np.linalg.eigvals(P)).min())
        rq = float(v @ np.linalg.solve(P, A @ v) / (v @ v))
        x, its, _ = O.pcgs(A, g, P, maxit=500)
        np.testing.assert_allclose(x, np.linalg.solve(A, g), rtol=1e-9, atol=1e-12)
        out[kind] = (lam_min, rq, its)
    assert eta <= out["strang"][0] <= 1.2 * eta, out
    assert out["tchan"][0] >= 100.0 * eta, out
    assert 1.0 <= out["strang"][1] <= 3.0 and out["tchan"][1] <= 0.05, out
    assert out["tchan"][2] >= 2 * out["strang"][2], out
