"""The seeded input recipes (no GPU).

* the batch workload: 4096 instances from PCG64 seed 1603, n odd and log-uniform in
  [255, 16383] with about half snapped to 2^k - 1 (sum of n about 1.59e7), alpha, beta and the
  constant coefficients in their stated ranges; the same instances on every call;
* the history workload: 16 instances of n = 2^18 - 1, M = 8192, each of the 8 (alpha, beta)
  pairs twice;
* the manufactured sources, checked against the definitions they stand for, by quadrature:
  the Caputo derivative of Eq. (1.2) of t^2 and t^(2+alpha), and the left Riemann-Liouville
  derivative of Eq. (1.3) of X(x) = x^2 (1-x)^2; the right one of Eq. (1.4) by the symmetry
  X(x) = X(1-x); and the four separable factors summing to f.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import tsfcde_workloads as W


def test_batch_recipe():
    a = W.config_batch()
    b = W.config_batch()
    assert len(a) == 4096
    ns = np.array([p.n for p in a])
    assert np.array_equal(ns, [p.n for p in b])
    assert [p.alpha for p in a] == [p.alpha for p in b]
    assert (ns % 2 == 1).all() and ns.min() >= 255 and ns.max() <= 16383
    snapped = np.mean([((n + 1) & n) == 0 for n in ns])
    assert 0.45 <= snapped <= 0.6, snapped
    assert 1.5e7 <= ns.sum() <= 1.7e7, ns.sum()
    for p in a[:200]:
        assert 0.1 <= p.alpha <= 0.95 and 1.1 <= p.beta <= 1.95
        assert 0.2 <= p.d_plus(0.3) <= 2.0 and 0.2 <= p.d_minus(0.7) <= 2.0
        assert -1.0 <= p.gamma(0.5) <= 1.0
        assert p.d_plus(0.0) == p.d_plus(1.0) and p.constant_coefficients and p.f is None
        assert p.M == 256
    # log-uniform: the geometric middle of the range splits the instances roughly in half
    mid = math.sqrt(255 * 16383)
    assert 0.35 <= np.mean(ns < mid) <= 0.65


def test_history_recipe():
    ps = W.config_history()
    assert len(ps) == 16
    assert all(p.n == (1 << 18) - 1 and p.M == 8192 for p in ps)
    pairs = [(p.alpha, p.beta) for p in ps]
    assert sorted(set(pairs)) == sorted((a, b) for a in (0.2, 0.5, 0.9, 0.99) for b in (1.2, 1.8))
    assert all(pairs.count(q) == 2 for q in set(pairs))


def _caputo(dg, alpha, t):
    """Caputo derivative of Eq. (1.2), 1/Gamma(1-alpha) int_0^t g'(s) (t-s)^(-alpha) ds, by
    quadrature with the algebraic end-point weight (dg = g')."""
    val, _ = integrate.quad(dg, 0.0, t, weight="alg", wvar=(0.0, -alpha), epsabs=1e-13,
                            epsrel=1e-11)
    return val / math.gamma(1.0 - alpha)


@pytest.mark.parametrize("alpha", [0.2, 0.6, 0.9])
@pytest.mark.parametrize("t", [0.3, 1.0])
def test_caputo_closed_forms(alpha, t):
    f2, _, _ = W.manufactured_t2(alpha, 1.5, lambda s: 0.0, lambda s: 0.0, lambda s: 0.0)
    fa, _, _ = W.manufactured_t2alpha(alpha, 1.5, lambda s: 0.0, lambda s: 0.0, lambda s: 0.0)
    x = np.array([0.5])
    X = W.X(x)[0]
    # with zero coefficients the source is exactly (Caputo T)(t) X(x)
    # u = (t^2 + 1) X and u = (t^(2+alpha) + 1) X, through their time derivatives
    assert f2(x, t)[0] / X == pytest.approx(_caputo(lambda s: 2.0 * s, alpha, t), rel=1e-9)
    assert fa(x, t)[0] / X == pytest.approx(
        _caputo(lambda s: (2.0 + alpha) * s ** (1.0 + alpha), alpha, t), rel=1e-9)


def _rl_left(g, beta, x):
    """Left Riemann-Liouville derivative of Eq. (1.3) of order beta in (1, 2):
    1/Gamma(2-beta) d^2/dx^2 int_0^x (x-s)^(1-beta) g(s) ds, the integral by quadrature with the
    algebraic end-point weight, the second derivative by a central difference."""
    def I(y):
        v, _ = integrate.quad(g, 0.0, y, weight="alg", wvar=(0.0, 1.0 - beta), epsabs=1e-14,
                              epsrel=1e-12)
        return v
    d = 1e-3
    return (I(x + d) - 2.0 * I(x) + I(x - d)) / (d * d) / math.gamma(2.0 - beta)


@pytest.mark.parametrize("beta", [1.2, 1.5, 1.8])
@pytest.mark.parametrize("x", [0.25, 0.6])
def test_riemann_liouville_closed_forms(beta, x):
    g = lambda s: s * s * (1 - s) ** 2
    ref = _rl_left(g, beta, x)
    assert W.rl_left_X(np.array([x]), beta)[0] == pytest.approx(ref, rel=2e-5, abs=1e-7)
    # right derivative of Eq. (1.4) at x is the left one of the reflected function at 1 - x
    ref_r = _rl_left(lambda s: g(1.0 - s), beta, 1.0 - x)
    assert W.rl_right_X(np.array([x]), beta)[0] == pytest.approx(ref_r, rel=2e-5, abs=1e-7)


@pytest.mark.parametrize("maker", [W.config_small, W.config_large, W.config_mixed,
                                   lambda: W.config_history()[5]])
def test_separable_factors_sum_to_the_source(maker):
    p = maker()
    x = np.linspace(0.01, 0.99, 37)
    for t in (0.0, 0.37, 1.0):
        f = p.f(x, t)
        s = sum(Tr(t) * Xr(x) for Tr, Xr in p.separable)
        np.testing.assert_allclose(s, f, rtol=1e-13, atol=1e-13 * np.abs(f).max())
