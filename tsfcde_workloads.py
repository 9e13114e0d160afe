"""Seeded synthetic inputs for the time-space fractional convection-diffusion equation (TSFCDE).

This module only describes *problems*: the domain, the orders alpha and beta, the coefficient
functions gamma(t), d_plus(t), d_minus(t), the initial value phi(x) and the source f(x, t) of
Eq. (1.1).  It holds none of the discretisation or solver arithmetic, so both the CPU oracle and
the GPU path can take their inputs from it.

Manufactured solutions.  For u(x, t) = T(t) X(x) with X(x) = x^2 (1 - x)^2 on [0, 1] the source
that makes u an exact solution of Eq. (1.1) is

    f = (Caputo_t^alpha T)(t) X(x)
        - T(t) [ gamma(t) X'(x) + d_plus(t) (0D_x^beta X)(x) + d_minus(t) (xD_1^beta X)(x) ],

with the Caputo derivative of Eq. (1.2) and the Riemann-Liouville derivatives of Eqs. (1.3)-(1.4)
applied to powers (D^beta x^p = Gamma(p+1)/Gamma(p+1-beta) x^(p-beta)); X is symmetric under
x -> 1-x, so the right-sided derivative is the left one evaluated at 1-x.  The source is a sum of
four separable terms f = sum_r T_r(t) X_r(x); `separable_source` returns them so the GPU path can
rebuild f on the device from 4 spatial profiles and 4 time tables.

Workloads (sizes are interior unknowns n, the paper's N-1):
  * `config_small`   n=127, M=64, alpha=0.6, beta=1.7, gamma=0.5, d+=1+t, d-=1-t/2, u=(t^2+1)X.
  * `config_large`   n=65535, M=1024, alpha=0.3, beta=1.9, same coefficient forms and solution.
  * `config_mixed`   n=2^20-1, M=512, alpha=0.8, beta=1.5, gamma=1, d+-=(1 +- t/2)/2.
  * `config_batch`   seeded instances with log-uniform n in [255, 16383] and constant coefficients.
  * `config_history` 16 instances of n=2^18-1, M=8192 (8 (alpha, beta) combinations, each twice).
  * `example1`/`example2`: the paper's Examples 1 and 2 (Section 4), u=(t^(2+alpha)+1)X.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

Coef = Callable[[float], float]
Field = Callable[[np.ndarray, float], np.ndarray]


@dataclass
class Problem:
    """One TSFCDE instance, Eq. (1.1): domain [a,b]x(0,T], n interior points, M time levels."""

    a: float
    b: float
    T: float
    n: int
    M: int
    alpha: float
    beta: float
    gamma: Coef
    d_plus: Coef
    d_minus: Coef
    phi: Callable[[np.ndarray], np.ndarray]
    f: Optional[Field]
    exact: Optional[Field] = None          # u(x, t) when known
    preconditioner: str = "strang"         # "strang" | "tchan" | "none"
    tol: float = 1e-12
    constant_coefficients: bool = False
    name: str = ""
    # separable form of f: list of (time function, spatial function)
    separable: Optional[List[tuple]] = field(default=None, repr=False)

    @property
    def h(self) -> float:
        return (self.b - self.a) / (self.n + 1)

    @property
    def tau(self) -> float:
        return self.T / self.M

    def grid(self) -> np.ndarray:
        """Interior nodes x_i = a + i h, i = 1..n (the mesh of Section 2.1)."""
        return self.a + self.h * np.arange(1, self.n + 1, dtype=np.float64)


# --------------------------------------------------------------------------------------------
# Closed forms used by manufactured solutions on [0, 1]
# --------------------------------------------------------------------------------------------

def X(x):
    return x * x * (1.0 - x) ** 2


def dX(x):
    return 2.0 * x * (1.0 - x) * (1.0 - 2.0 * x)


def rl_left_X(x, beta):
    """Left Riemann-Liouville derivative 0D_x^beta of x^2 - 2x^3 + x^4 (Eq. (1.3) on powers)."""
    g = math.gamma
    return (g(3.0) / g(3.0 - beta) * np.power(x, 2.0 - beta)
            - 2.0 * g(4.0) / g(4.0 - beta) * np.power(x, 3.0 - beta)
            + g(5.0) / g(5.0 - beta) * np.power(x, 4.0 - beta))


def rl_right_X(x, beta):
    """Right Riemann-Liouville derivative xD_1^beta of X (Eq. (1.4)); X(x) = X(1-x)."""
    return rl_left_X(1.0 - x, beta)


def _manufactured(alpha, beta, gamma, dp, dm, Tt, Tcap):
    """Source f and its separable factors for u = Tt(t) X(x)."""

    def f(x, t):
        x = np.asarray(x, dtype=np.float64)
        return (Tcap(t) * X(x)
                - Tt(t) * (gamma(t) * dX(x) + dp(t) * rl_left_X(x, beta)
                           + dm(t) * rl_right_X(x, beta)))

    sep = [
        (lambda t: Tcap(t), lambda x: X(x)),
        (lambda t: -Tt(t) * gamma(t), lambda x: dX(x)),
        (lambda t: -Tt(t) * dp(t), lambda x: rl_left_X(x, beta)),
        (lambda t: -Tt(t) * dm(t), lambda x: rl_right_X(x, beta)),
    ]

    def exact(x, t):
        return Tt(t) * X(np.asarray(x, dtype=np.float64))

    return f, sep, exact


def manufactured_t2(alpha, beta, gamma, dp, dm):
    """u = (t^2 + 1) X(x); Caputo derivative of t^2 is 2 t^(2-alpha) / Gamma(3-alpha)."""
    Tt = lambda t: t * t + 1.0
    Tcap = lambda t: 2.0 * t ** (2.0 - alpha) / math.gamma(3.0 - alpha)
    return _manufactured(alpha, beta, gamma, dp, dm, Tt, Tcap)


def manufactured_t2alpha(alpha, beta, gamma, dp, dm):
    """u = (t^(2+alpha) + 1) X(x) (Examples 1-2); Caputo of t^(2+alpha) is Gamma(3+alpha)/2 t^2."""
    Tt = lambda t: t ** (2.0 + alpha) + 1.0
    Tcap = lambda t: math.gamma(3.0 + alpha) / 2.0 * t * t
    return _manufactured(alpha, beta, gamma, dp, dm, Tt, Tcap)


def _make(n, M, alpha, beta, gamma, dp, dm, manuf, **kw):
    f, sep, exact = manuf(alpha, beta, gamma, dp, dm)
    return Problem(a=0.0, b=1.0, T=1.0, n=n, M=M, alpha=alpha, beta=beta, gamma=gamma,
                   d_plus=dp, d_minus=dm, phi=lambda x: exact(x, 0.0), f=f, exact=exact,
                   separable=sep, **kw)


# --------------------------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------------------------

def manufactured(n, M, alpha, beta, gamma=lambda t: 0.5, d_plus=lambda t: 1.0 + t,
                 d_minus=lambda t: 1.0 - 0.5 * t, preconditioner="strang", constant=False):
    """Any parameters with the manufactured solution u = (t^2+1) x^2 (1-x)^2 on [0, 1] and its
    analytic source (edge and degenerate cases of Eq. (1.1))."""
    return _make(n, M, alpha, beta, gamma, d_plus, d_minus, manufactured_t2,
                 preconditioner=preconditioner, constant_coefficients=constant, name="manufactured")


def config_small(n=127, M=64, alpha=0.6, beta=1.7, preconditioner="strang"):
    """Small FP64 instance: n=127, M=64, alpha=0.6, beta=1.7, gamma=0.5, d+=1+t, d-=1-t/2."""
    return _make(n, M, alpha, beta, lambda t: 0.5, lambda t: 1.0 + t, lambda t: 1.0 - 0.5 * t,
                 manufactured_t2, preconditioner=preconditioner, name="small")


def config_large(n=65535, M=1024, alpha=0.3, beta=1.9, preconditioner="tchan"):
    """Large FP64 instance: n=2^16-1, M=1024, alpha=0.3, beta=1.9, T. Chan preconditioner."""
    return _make(n, M, alpha, beta, lambda t: 0.5, lambda t: 1.0 + t, lambda t: 1.0 - 0.5 * t,
                 manufactured_t2, preconditioner=preconditioner, name="large")


def config_mixed(n=(1 << 20) - 1, M=512, alpha=0.8, beta=1.5, preconditioner="strang"):
    """Precision workload: n=2^20-1, M=512, alpha=0.8, beta=1.5, gamma=1, d+-=(1+-t/2)/2."""
    return _make(n, M, alpha, beta, lambda t: 1.0, lambda t: 0.5 * (1.0 + 0.5 * t),
                 lambda t: 0.5 * (1.0 - 0.5 * t), manufactured_t2,
                 preconditioner=preconditioner, name="mixed")


def config_history(n=(1 << 18) - 1, M=8192, preconditioner="strang"):
    """History-dominated workload: 16 instances, the 8 combinations of alpha in
    {0.2, 0.5, 0.9, 0.99} and beta in {1.2, 1.8}, each twice (16 instances from 8 combinations)."""
    combos = [(a, b) for a in (0.2, 0.5, 0.9, 0.99) for b in (1.2, 1.8)]
    combos = combos + combos
    return [_make(n, M, a, b, lambda t: 0.5, lambda t: 1.0 + t, lambda t: 1.0 - 0.5 * t,
                  manufactured_t2, preconditioner=preconditioner, name=f"history{i}")
            for i, (a, b) in enumerate(combos)]


def example1(n, M, alpha, beta=1.8):
    """Paper Example 1 (Section 4): d+=0.8, d-=0.5, gamma=-0.1, u=(t^(2+alpha)+1)X."""
    return _make(n, M, alpha, beta, lambda t: -0.1, lambda t: 0.8, lambda t: 0.5,
                 manufactured_t2alpha, constant_coefficients=True, name="example1")


def example2(n, M, alpha, beta=1.3):
    """Paper Example 2 (Section 4): d+=9 sin t, d-=4 sin t, gamma=-t, u=(t^(2+alpha)+1)X."""
    return _make(n, M, alpha, beta, lambda t: -t, lambda t: 9.0 * math.sin(t),
                 lambda t: 4.0 * math.sin(t), manufactured_t2alpha, name="example2")


def config_batch(count=4096, M=256, seed=1603, n_lo=255, n_hi=16383):
    """Independent constant-coefficient instances with uneven n (seeded, PCG64).

    n = odd(round(exp(U(ln n_lo, ln n_hi)))), half of them snapped to 2^k - 1; alpha ~ U(.1,.95),
    beta ~ U(1.1,1.95), d+- ~ U(.2,2), gamma ~ U(-1,1); phi = sum of 4 sine modes with U(-1,1)
    amplitudes; f = 0.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        n |= 1
        if rng.uniform() < 0.5:
            n = (1 << max(1, int(round(math.log2(n + 1))))) - 1
        n = min(max(n, n_lo), n_hi)
        alpha = float(rng.uniform(0.1, 0.95))
        beta = float(rng.uniform(1.1, 1.95))
        dp = float(rng.uniform(0.2, 2.0))
        dm = float(rng.uniform(0.2, 2.0))
        gm = float(rng.uniform(-1.0, 1.0))
        amps = rng.uniform(-1.0, 1.0, size=4)

        def phi(x, amps=amps):
            x = np.asarray(x, dtype=np.float64)
            return sum(amps[m] * np.sin((m + 1) * math.pi * x) for m in range(4))

        out.append(Problem(a=0.0, b=1.0, T=1.0, n=n, M=M, alpha=alpha, beta=beta,
                           gamma=(lambda t, g=gm: g), d_plus=(lambda t, d=dp: d),
                           d_minus=(lambda t, d=dm: d), phi=phi, f=None,
                           constant_coefficients=True, name=f"batch{i}"))
    return out
