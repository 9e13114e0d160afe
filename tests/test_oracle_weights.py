"""Pins of the oracle's space and time weights against closed forms (Lemmas 1-4)."""
import math

import numpy as np
import pytest
from scipy.special import binom

import oracle as O

BETAS = [1.1, 1.3, 1.5, 1.7, 1.9, 2.0]
ALPHAS = [0.1, 0.3, 0.5, 0.6, 0.9, 0.99]


@pytest.mark.parametrize("beta", BETAS)
def test_grunwald_closed_form(beta):
    # Lemma 2: g_k = (-1)^k binom(beta, k); Lemma 3 recurrence must reproduce it.
    g = O.grunwald_weights(beta, 60)
    ref = np.array([(-1) ** k * binom(beta, k) for k in range(61)])
    np.testing.assert_allclose(g, ref, rtol=1e-12, atol=1e-15)
    # partial sums: sum_{k<=m} g_k = (-1)^m binom(beta-1, m)
    ps = np.cumsum(g)
    ref_ps = np.array([(-1) ** m * binom(beta - 1, m) for m in range(61)])
    np.testing.assert_allclose(ps, ref_ps, rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("beta", [b for b in BETAS if b < 2.0])
def test_grunwald_lemma3_properties(beta):
    g = O.grunwald_weights(beta, 400)
    assert g[0] == 1.0 and abs(g[1] + beta) < 1e-15
    assert np.all(np.diff(g[2:]) < 0) and np.all(g[2:] > 0)
    assert np.all(np.cumsum(g)[2:] < 0)


@pytest.mark.parametrize("beta", [b for b in BETAS if b < 2.0])
def test_wsgd_lemma4_properties(beta):
    w = O.wsgd_weights(beta, 2000)
    lam1, lam0, lamm1 = O.wsgd_lambdas(beta)
    assert abs(lam1 + lam0 + lamm1 - 1.0) < 1e-15
    assert abs(w[0] - lam1) < 1e-15          # omega_0 = lambda_1 (Lemma 4 prints 1)
    assert w[1] < 0 and np.all(w[3:] > 0)
    assert w[0] + w[2] >= 0
    assert np.all(np.cumsum(w)[2:] < 0)      # sum_{k<=N} omega_k < 0 for N > 1
    assert abs(np.sum(w)) < 5e-3             # -> 0 as N -> infinity


@pytest.mark.parametrize("beta", BETAS)
def test_wsgd_generating_function(beta):
    # sum_k omega_k z^k = (lambda_1 + lambda_0 z + lambda_{-1} z^2) (1 - z)^beta, |z| < 1.
    w = O.wsgd_weights(beta, 300)
    lam1, lam0, lamm1 = O.wsgd_lambdas(beta)
    for z in (0.3, -0.5, 0.7):
        lhs = np.polynomial.polynomial.polyval(z, w)
        rhs = (lam1 + lam0 * z + lamm1 * z * z) * (1 - z) ** beta
        assert abs(lhs - rhs) < 1e-12


def test_wsgd_beta2_is_second_difference():
    w = O.wsgd_weights(2.0, 10)
    np.testing.assert_allclose(w, [1, -2, 1] + [0] * 8, atol=1e-15)


@pytest.mark.parametrize("beta", [1.2, 1.5, 1.9])
def test_wsgd_second_order_accuracy(beta):
    # Lemma 2: (1/h^beta) W v -> 0D_x^beta v and (1/h^beta) W^T v -> xD_1^beta v with O(h^2),
    # checked on v = x^4 (1-x)^4 against the Riemann-Liouville power rule.
    g = math.gamma
    coef = [1, -4, 6, -4, 1]

    def rl(x):
        return sum(c * g(p + 1) / g(p + 1 - beta) * x ** (p - beta) for c, p in zip(coef, range(4, 9)))

    errs = []
    for n in (255, 511, 1023):
        h = 1.0 / (n + 1)
        x = h * np.arange(1, n + 1)
        v = x ** 4 * (1 - x) ** 4
        Wm = O.matrix_W(beta, n)
        e = max(np.max(np.abs(Wm @ v / h ** beta - rl(x))),
                np.max(np.abs(Wm.T @ v / h ** beta - rl(1 - x))))
        errs.append(e)
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.8, orders


@pytest.mark.parametrize("alpha", ALPHAS + [1.0])
def test_l21sigma_exact_on_quadratics(alpha):
    # Lemma 1 is exact for u = 1, t, t^2 at t_{j+sigma}: Caputo of t is t^(1-a)/G(2-a),
    # of t^2 is 2 t^(2-a)/G(3-a).
    sigma = 1 - alpha / 2
    tau = 0.037
    for j in (0, 1, 2, 7, 20):
        ts = tau * np.arange(j + 2)
        tj = (j + sigma) * tau
        assert abs(O.caputo_l21sigma(alpha, tau, np.ones(j + 2), j)) < 1e-12
        ref1 = tj ** (1 - alpha) / math.gamma(2 - alpha)
        assert abs(O.caputo_l21sigma(alpha, tau, ts, j) - ref1) < 1e-12 * max(1, ref1)
        ref2 = 2 * tj ** (2 - alpha) / math.gamma(3 - alpha)
        assert abs(O.caputo_l21sigma(alpha, tau, ts ** 2, j) - ref2) < 1e-12 * max(1, ref2)


@pytest.mark.parametrize("alpha", ALPHAS)
def test_c_coefficients_properties(alpha):
    sigma = 1 - alpha / 2
    for j in (1, 2, 5, 40):
        c = O.c_coeffs(alpha, j)
        assert abs(c.sum() - (j + sigma) ** (1 - alpha)) < 1e-12   # telescoping of Lemma 1
        assert np.all(np.diff(c) < 0)                               # decreasing in m
        assert c[j] > (1 - alpha) / (2 * (j + sigma) ** alpha)


def test_alpha_one_is_backward_difference():
    a, b = O.l21sigma_ab(1.0, 10)
    assert a[0] == 1.0 and np.all(a[1:] == 0) and np.all(b == 0)
    c = O.c_coeffs(1.0, 5)
    np.testing.assert_array_equal(c, [1, 0, 0, 0, 0, 0])
