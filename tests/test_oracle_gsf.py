"""Pins of the oracle's constant-coefficient path: the generator systems Eq. (3.5), the
Gohberg-Semencul formula Eq. (3.6) and Algorithm "Compute z = A^{-1} v" (Section 3.1), and
Algorithm "Practical implementation of IDS with constant coefficients" (Section 3.2).

What fixes them, other than the oracle itself:
  * exact rational arithmetic on tiny Toeplitz matrices: the formula must give the inverse
    exactly, entry for entry (brute force, no rounding);
  * LAPACK's inverse and solve on the scheme's own level matrices;
  * for a symmetric Toeplitz matrix, A^{-1} e_n is the reversal of A^{-1} e_1 (persymmetry);
  * the constant-coefficient march equals the plain elimination march level by level.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import tsfcde_workloads as W


def _frac_solve(A, B):
    """Gauss-Jordan elimination over the rationals: returns A^{-1} B (A, B lists of rows)."""
    n = len(A)
    m = len(B[0])
    M = [list(A[i]) + list(B[i]) for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * b for a, b in zip(M[r], M[c])]
    return [row[n:n + m] for row in M]


def _toeplitz_rows(t, n):
    """Rows of the Toeplitz matrix with T[i,k] = t[i-k] (t a dict over -(n-1)..n-1)."""
    return [[t[i - k] for k in range(n)] for i in range(n)]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_gs_inverse_is_exact_over_the_rationals(n):
    rng = np.random.default_rng(100 + n)
    t = {d: Fraction(int(rng.integers(-4, 5)), int(rng.integers(1, 4))) for d in range(-(n - 1), n)}
    t[0] = Fraction(3 * n + 7)   # diagonally dominant: nonsingular, xi_0 != 0
    A = _toeplitz_rows(t, n)
    I = [[Fraction(int(i == k)) for k in range(n)] for i in range(n)]
    Ainv = _frac_solve(A, I)
    x = [Ainv[i][0] for i in range(n)]        # A^{-1} e_1
    y = [Ainv[i][n - 1] for i in range(n)]    # A^{-1} e_n
    G = O.gs_inverse(x, y)
    assert G == Ainv


def test_gs_inverse_matches_lapack_on_level_matrix():
    prob = W.config_batch(count=2, M=4, n_lo=41, n_hi=41)[1]
    A, _ = O.level_matrices(prob, 1)
    x, y = O.gs_generators(A)
    G = np.array(O.gs_inverse(list(x), list(y)))
    ref = np.linalg.inv(A)
    assert np.linalg.norm(G - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("beta", [1.15, 1.6, 1.95])
def test_gs_apply_solves_the_level_system(beta):
    prob = W.example2(200, 8, 0.5, beta)
    A, _ = O.level_matrices(prob, 1)
    x, y = O.gs_generators(A)
    v = np.random.default_rng(7).standard_normal(prob.n)
    z = O.gs_apply(x, y, v)
    ref = np.linalg.solve(A, v)
    assert np.linalg.norm(z - ref) <= 1e-11 * np.linalg.norm(ref)


def test_generators_of_a_symmetric_toeplitz_are_reversals():
    """Symmetric Toeplitz A commutes with the reversal J, so A^{-1} e_n = J A^{-1} e_1."""
    n = 17
    prob = W.example2(n, 4, 0.5, 1.7)
    W_ = O.matrix_W(prob.beta, n)
    A = 5.0 * np.eye(n) - 0.5 * (W_ + W_.T)
    x, y = O.gs_generators(A)
    assert np.allclose(y, x[::-1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("idx", [0, 3])
def test_const_march_equals_plain_march(idx):
    prob = W.config_batch(count=4, M=10, n_lo=63, n_hi=255)[idx]
    a = O.run(prob)
    b = O.run_const(prob)
    assert len(a) == len(b) == prob.M + 1
    assert np.array_equal(a[1], b[1])   # level 0 is the same elimination
    gap = max(np.linalg.norm(a[j] - b[j]) / np.linalg.norm(a[j]) for j in range(1, prob.M + 1))
    assert gap <= 1e-11, gap


def test_a_misordered_factor_breaks_the_inverse():
    """A mistake in one factor (R_p's first row taken unreversed) breaks the inverse."""
    prob = W.config_batch(count=1, M=4, n_lo=15, n_hi=15)[0]
    A, _ = O.level_matrices(prob, 1)
    x, y = O.gs_generators(A)
    G = np.array(O.gs_inverse(list(x), list(y[::-1])))
    assert np.linalg.norm(G - np.linalg.inv(A)) > 1e-3 * np.linalg.norm(np.linalg.inv(A))
