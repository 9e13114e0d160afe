"""FP64 CPU oracle for the implicit difference scheme (IDS) of Gu, Huang, Ji, Carpentieri and
Alikhanov, "Fast iterative method with a second order implicit difference scheme for time-space
fractional convection-diffusion equations" (arXiv:1603.00279).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this module.  The product (the CUDA library and its binding) never calls it and shares no
code with it.

What it computes: the plain definition of the scheme.  Each time level of Eq. (2.1), written in
matrix form as Eq. (3.1)/(3.3), is assembled densely (Q and W_beta of Eq. (3.2)) and solved
exactly by Gaussian elimination with partial pivoting (LAPACK dgesv through numpy.linalg.solve),
level after level.  There is no FFT and no Krylov method on this path.  The circulant
preconditioners (Eq. (3.7), Strang and T. Chan) and a dense preconditioned CGS are also written
out densely, but only so that tests can pin iteration counts and preconditioner definitions; they
do not feed the level solutions.

For constant coefficients (Section 3.2) `run_const` follows Algorithm "Practical implementation of
IDS with constant coefficients": level 0 by elimination, every later level by the Gohberg-Semencul
formula (Eq. (3.6)) applied as in Algorithm "Compute z = A^{-1} v", with the two generator
systems of Eq. (3.5) solved by elimination and the four triangular Toeplitz factors formed densely.
It reaches the same level solutions as `run` up to rounding, which the tests check.

Notation follows the paper except that n = N - 1 is the number of interior unknowns,
h = (b - a) / (n + 1), tau = T / M, sigma = 1 - alpha/2.

Readings of the paper taken here (each is also listed in the design notes):
  * the history term is subtracted on the right-hand side (Eq. (3.1)); Eq. (3.3) prints "+",
    which contradicts Eq. (3.1) and the paper's own error tables;
  * gamma, d_+ and d_- and f are evaluated at t_{j+sigma} for every level, j = 0 included;
  * omega_0 = lambda_1 (Lemma 2), not 1 as Lemma 4 prints;
  * W_beta is the Toeplitz matrix W[i,k] = omega_{i-k+1} (zero when i-k+1 < 0), the reading of
    the garbled last row of the display in Eq. (3.2);
  * Strang: c_k = t_k for 0 <= k <= floor(n/2), c_k = t_{k-n} otherwise; T. Chan:
    c_k = ((n-k) t_k + k t_{k-n}) / n (neither is written out in the paper);
  * alpha = 1 is allowed: then sigma = 1/2, a_0 = 1, a_l = b_l = 0 and the scheme is
    Crank-Nicolson (remark after Eq. (2.1)).
"""
from __future__ import annotations

import math
from typing import Callable, Iterable, List, Optional

import numpy as np

# ----------------------------------------------------------------------------------------------
# Space weights: Lemma 2 (WSGD weights) and Lemma 3 (Grunwald weights)
# ----------------------------------------------------------------------------------------------


def grunwald_weights(beta: float, K: int) -> np.ndarray:
    """g_k = (-1)^k binom(beta, k), k = 0..K, by the recurrence g_k = (1 - (beta+1)/k) g_{k-1}
    (Lemma 3)."""
    g = np.empty(K + 1, dtype=np.float64)
    g[0] = 1.0
    for k in range(1, K + 1):
        g[k] = (1.0 - (beta + 1.0) / k) * g[k - 1]
    return g


def wsgd_lambdas(beta: float):
    """lambda_1, lambda_0, lambda_{-1} of Lemma 2."""
    lam1 = (beta * beta + 3.0 * beta + 2.0) / 12.0
    lam0 = (4.0 - beta * beta) / 6.0
    lamm1 = (beta * beta - 3.0 * beta + 2.0) / 12.0
    return lam1, lam0, lamm1


def wsgd_weights(beta: float, K: int) -> np.ndarray:
    """omega_k, k = 0..K (Lemma 2):
    omega_0 = lambda_1 g_0, omega_1 = lambda_1 g_1 + lambda_0 g_0,
    omega_k = lambda_1 g_k + lambda_0 g_{k-1} + lambda_{-1} g_{k-2} for k >= 2."""
    g = grunwald_weights(beta, K)
    lam1, lam0, lamm1 = wsgd_lambdas(beta)
    w = np.empty(K + 1, dtype=np.float64)
    w[0] = lam1 * g[0]
    if K >= 1:
        w[1] = lam1 * g[1] + lam0 * g[0]
    for k in range(2, K + 1):
        w[k] = lam1 * g[k] + lam0 * g[k - 1] + lamm1 * g[k - 2]
    return w


# ----------------------------------------------------------------------------------------------
# Time weights: Lemma 1 (the L2-1_sigma formula)
# ----------------------------------------------------------------------------------------------


def l21sigma_ab(alpha: float, K: int):
    """a_l and b_l of Lemma 1 for l = 0..K (b_0 is unused and set to 0)."""
    sigma = 1.0 - alpha / 2.0
    a = np.empty(K + 1, dtype=np.float64)
    b = np.zeros(K + 1, dtype=np.float64)
    a[0] = sigma ** (1.0 - alpha)
    for l in range(1, K + 1):
        a[l] = (l + sigma) ** (1.0 - alpha) - (l - 1 + sigma) ** (1.0 - alpha)
        b[l] = (((l + sigma) ** (2.0 - alpha) - (l - 1 + sigma) ** (2.0 - alpha)) / (2.0 - alpha)
                - 0.5 * ((l + sigma) ** (1.0 - alpha) + (l - 1 + sigma) ** (1.0 - alpha)))
    return a, b


def c_coeffs(alpha: float, j: int) -> np.ndarray:
    """c^{(alpha,sigma,j)}_m for m = 0..j (Lemma 1)."""
    a, b = l21sigma_ab(alpha, j + 1)
    c = np.empty(j + 1, dtype=np.float64)
    if j == 0:
        c[0] = a[0]
        return c
    c[0] = a[0] + b[1]
    for m in range(1, j):
        c[m] = a[m] + b[m + 1] - b[m]
    c[j] = a[j] - b[j]
    return c


def caputo_l21sigma(alpha: float, tau: float, values: np.ndarray, j: int) -> float:
    """Delta^alpha_{0,t_{j+sigma}} u of Lemma 1 for a scalar sequence u(t_0..t_{j+1})."""
    c = c_coeffs(alpha, j)
    s = sum(c[j - s] * (values[s + 1] - values[s]) for s in range(j + 1))
    return tau ** (-alpha) / math.gamma(2.0 - alpha) * s


# ----------------------------------------------------------------------------------------------
# Matrices of Eq. (3.2) and Eq. (3.3)
# ----------------------------------------------------------------------------------------------


def matrix_Q(n: int) -> np.ndarray:
    """Q of Eq. (3.2): +1 on the super-diagonal, -1 on the sub-diagonal."""
    return np.eye(n, k=1) - np.eye(n, k=-1)


def matrix_W(beta: float, n: int) -> np.ndarray:
    """W_beta of Eq. (3.2): W[i,k] = omega_{i-k+1} for i-k+1 >= 0, else 0."""
    w = wsgd_weights(beta, n + 1)
    d = np.arange(n)[:, None] - np.arange(n)[None, :] + 1      # d = i - k + 1
    return np.where(d >= 0, w[np.clip(d, 0, n + 1)], 0.0)


def eta(alpha: float, tau: float, j: int) -> float:
    """eta_j = c^{(j)}_0 / (tau^alpha Gamma(2-alpha)) (below Eq. (3.1))."""
    a, b = l21sigma_ab(alpha, 1)
    c0 = a[0] if j == 0 else a[0] + b[1]
    return c0 / (tau ** alpha * math.gamma(2.0 - alpha))


def level_scalars(prob, j: int):
    """(eta_j, q, kappa_+, kappa_-) at t_{j+sigma}: q = gamma/(2h), kappa_pm = d_pm / h^beta."""
    sigma = 1.0 - prob.alpha / 2.0
    t = (j + sigma) * prob.tau
    h = prob.h
    return (eta(prob.alpha, prob.tau, j), prob.gamma(t) / (2.0 * h),
            prob.d_plus(t) / h ** prob.beta, prob.d_minus(t) / h ** prob.beta)


def level_matrices(prob, j: int, Q=None, W=None):
    """A^{(j+sigma)} and B^{(j+sigma)} of Eq. (3.3)."""
    n = prob.n
    sigma = 1.0 - prob.alpha / 2.0
    if Q is None:
        Q = matrix_Q(n)
    if W is None:
        W = matrix_W(prob.beta, n)
    e, q, kp, km = level_scalars(prob, j)
    L = q * Q + kp * W + km * W.T
    I = np.eye(n)
    return e * I - sigma * L, e * I + (1.0 - sigma) * L


# ----------------------------------------------------------------------------------------------
# The time march (Algorithm "Practical implementation of IDS", solved exactly per level)
# ----------------------------------------------------------------------------------------------


def run(prob, levels: Optional[int] = None, source: Optional[Callable] = None,
        solve: Optional[Callable] = None) -> List[np.ndarray]:
    """Return [u^0, u^1, ..., u^levels] (interior values) for the problem `prob`.

    For j = 0..levels-1 (Eq. (3.1)):
        g = B^{(j+sigma)} u^j - tau^{-alpha}/Gamma(2-alpha) sum_{s<j} c^{(j)}_{j-s} (u^{s+1}-u^s)
            + f(x, t_{j+sigma})
        A^{(j+sigma)} u^{j+1} = g        (Gaussian elimination with partial pivoting)
    `solve(j, A, g)` replaces the elimination when given (see run_const).
    """
    M = prob.M if levels is None else levels
    n = prob.n
    x = prob.grid()
    sigma = 1.0 - prob.alpha / 2.0
    tau = prob.tau
    hist_scale = tau ** (-prob.alpha) / math.gamma(2.0 - prob.alpha)
    Q = matrix_Q(n)
    W = matrix_W(prob.beta, n)
    f = source if source is not None else prob.f
    u = [np.asarray(prob.phi(x), dtype=np.float64).copy()]
    for j in range(M):
        A, B = level_matrices(prob, j, Q, W)
        g = B @ u[j]
        if j >= 1:
            c = c_coeffs(prob.alpha, j)
            H = np.zeros(n)
            for s in range(j):
                H += c[j - s] * (u[s + 1] - u[s])
            g = g - hist_scale * H
        if f is not None:
            g = g + f(x, (j + sigma) * tau)
        u.append(np.linalg.solve(A, g) if solve is None else solve(j, A, g))
    return u


# ----------------------------------------------------------------------------------------------
# Rows of one level's equation without n x n matrices (checks at sizes where elimination is
# impossible)
# ----------------------------------------------------------------------------------------------


def level_row(prob, j: int, i: int, omega: Optional[np.ndarray] = None):
    """Row i of A^{(j+sigma)} and of B^{(j+sigma)} (Eq. (3.3)), entry by entry:
        L[i,k] = q Q[i,k] + kappa_+ omega_{i-k+1} + kappa_- omega_{k-i+1}
                 (Q[i,i+1] = 1, Q[i,i-1] = -1; omega_m = 0 for m < 0, Eq. (3.2)),
        A[i,:] = eta e_i - sigma L[i,:],  B[i,:] = eta e_i + (1 - sigma) L[i,:]."""
    n = prob.n
    sigma = 1.0 - prob.alpha / 2.0
    w = wsgd_weights(prob.beta, n + 1) if omega is None else omega
    e, q, kp, km = level_scalars(prob, j)
    k = np.arange(n)
    dW = i - k + 1                       # W[i,k] = omega_{i-k+1}
    dWt = k - i + 1                      # W^T[i,k] = W[k,i] = omega_{k-i+1}
    Lrow = kp * np.where(dW >= 0, w[np.clip(dW, 0, n + 1)], 0.0)
    Lrow = Lrow + km * np.where(dWt >= 0, w[np.clip(dWt, 0, n + 1)], 0.0)
    if i + 1 < n:
        Lrow[i + 1] += q
    if i - 1 >= 0:
        Lrow[i - 1] -= q
    Arow = -sigma * Lrow
    Brow = (1.0 - sigma) * Lrow
    Arow[i] += e
    Brow[i] += e
    return Arow, Brow


def level_equation_rows(prob, j: int, rows, levels: List[np.ndarray], u_next: np.ndarray,
                        source: Optional[Callable] = None):
    """Rows of the level-j equation of Eq. (3.1) evaluated at given level vectors u^0..u^j
    (`levels`) and u^{j+1} (`u_next`), O(n) work per row:
        g_i  = (B u^j)_i - tau^{-alpha}/Gamma(2-alpha) sum_{s<j} c^{(j)}_{j-s} (u^{s+1}_i - u^s_i)
               + f(x_i, t_{j+sigma}),
        Au_i = (A u^{j+1})_i.
    Returns (g, Au) over `rows`."""
    n = prob.n
    w = wsgd_weights(prob.beta, n + 1)
    sigma = 1.0 - prob.alpha / 2.0
    hist_scale = prob.tau ** (-prob.alpha) / math.gamma(2.0 - prob.alpha)
    c = c_coeffs(prob.alpha, j) if j >= 1 else None
    f = source if source is not None else prob.f
    x = prob.grid()
    g = np.empty(len(rows))
    Au = np.empty(len(rows))
    for r, i in enumerate(rows):
        Arow, Brow = level_row(prob, j, int(i), w)
        gi = float(Brow @ levels[j])
        if j >= 1:
            H = 0.0
            for s_ in range(j):
                H += c[j - s_] * (levels[s_ + 1][i] - levels[s_][i])
            gi -= hist_scale * H
        if f is not None:
            gi += float(np.asarray(f(x[i:i + 1], (j + sigma) * prob.tau))[0])
        g[r] = gi
        Au[r] = float(Arow @ u_next)
    return g, Au


# ----------------------------------------------------------------------------------------------
# Constant coefficients: the Gohberg-Semencul formula Eq. (3.6) and Algorithm "Compute
# z = A^{-1} v" (Section 3.1), and Algorithm "Practical implementation of IDS with constant
# coefficients" (Section 3.2).  Dense matrices throughout; no FFT.
# ----------------------------------------------------------------------------------------------


def gs_generators(A: np.ndarray):
    """x = A^{-1} e_1 and y = A^{-1} e_n, the two systems of Eq. (3.5), by Gaussian elimination."""
    n = A.shape[0]
    E = np.zeros((n, 2))
    E[0, 0] = 1.0
    E[n - 1, 1] = 1.0
    X = np.linalg.solve(A, E)
    return X[:, 0].copy(), X[:, 1].copy()


def gs_factors(x, y):
    """The four triangular Toeplitz matrices of the Gohberg-Semencul formula, entry by entry
    (generic element type, so exact rationals work):
        L_p [i,k] = xi_{i-k}          (i >= k)   lower, first column x
        R_p [i,k] = eta_{n-1-(k-i)}   (k >= i)   upper, first row (eta_{n-1}, ..., eta_0)
        L0_p[i,k] = eta_{i-k-1}       (i >  k)   strictly lower, first column (0, eta_0, ...)
        R0_p[i,k] = xi_{n-(k-i)}      (k >  i)   strictly upper, first row (0, xi_{n-1}, ..., xi_1)
    Returned as lists of rows."""
    n = len(x)
    zero = x[0] - x[0]
    Lp = [[x[i - k] if i >= k else zero for k in range(n)] for i in range(n)]
    Rp = [[y[n - 1 - (k - i)] if k >= i else zero for k in range(n)] for i in range(n)]
    L0 = [[y[i - k - 1] if i > k else zero for k in range(n)] for i in range(n)]
    R0 = [[x[n - (k - i)] if k > i else zero for k in range(n)] for i in range(n)]
    return Lp, Rp, L0, R0


def _matmul_rows(P, Q):
    n = len(P)
    return [[sum((P[i][m] * Q[m][k] for m in range(n)), P[0][0] - P[0][0]) for k in range(n)]
            for i in range(n)]


def gs_inverse(x, y):
    """A^{-1} = (L_p R_p - L0_p R0_p) / xi_0 (Gohberg-Semencul formula; requires xi_0 != 0).
    Plain loops over entries: for pins on small n, any element type with + - * /."""
    Lp, Rp, L0, R0 = gs_factors(x, y)
    P1 = _matmul_rows(Lp, Rp)
    P2 = _matmul_rows(L0, R0)
    n = len(x)
    return [[(P1[i][k] - P2[i][k]) / x[0] for k in range(n)] for i in range(n)]


def gs_apply(x: np.ndarray, y: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Algorithm "Compute z = A^{-1} v": z1 = R0_p v, z2 = R_p v, z3 = L0_p z1, z4 = L_p z2,
    z = (z4 - z3) / xi_0, with the triangular Toeplitz matrices formed densely (FP64)."""
    Lp, Rp, L0, R0 = (np.array(F, dtype=np.float64) for F in gs_factors(list(x), list(y)))
    z1 = R0 @ v
    z2 = Rp @ v
    z3 = L0 @ z1
    z4 = Lp @ z2
    return (z4 - z3) / x[0]


def run_const(prob, levels: Optional[int] = None, source: Optional[Callable] = None) -> List[np.ndarray]:
    """Algorithm "Practical implementation of IDS with constant coefficients": level 0 solves
    A^{(sigma)} u^1 = g^1 by elimination; every later level, whose matrix A is the same for
    j = 1..M-1 when gamma and d_+- are constant (Eq. (3.4)), computes u^{j+1} = A^{-1} g
    by Algorithm "Compute z = A^{-1} v" with the generators of that A."""
    gen = {}

    def solve(j, A, g):
        if j == 0:
            return np.linalg.solve(A, g)
        if "xy" not in gen:
            gen["xy"] = gs_generators(A)
        return gs_apply(gen["xy"][0], gen["xy"][1], g)

    return run(prob, levels, source, solve)


def l2_norm(v: np.ndarray, h: float) -> float:
    """Discrete L2 norm ||v|| = sqrt(h sum v_i^2) (Section 2.2)."""
    return math.sqrt(h * float(np.dot(v, v)))


def errors_vs_exact(prob, levels: List[np.ndarray]):
    """max_n ||E^n||_0 and max |E| over the grid (Section 4, Tables 1, 2, 5 and 6)."""
    x = prob.grid()
    e2, emax = 0.0, 0.0
    for j, u in enumerate(levels):
        E = u - prob.exact(x, j * prob.tau)
        e2 = max(e2, l2_norm(E, prob.h))
        emax = max(emax, float(np.max(np.abs(E))))
    return e2, emax


def convergence_order(e1: float, e2: float, h1: float, h2: float) -> float:
    """CO = log_{h1/h2}(E1/E2) (Section 4)."""
    return math.log(e1 / e2) / math.log(h1 / h2)


# ----------------------------------------------------------------------------------------------
# Circulant preconditioners (Eq. (3.7)) and dense preconditioned CGS, for pinning only
# ----------------------------------------------------------------------------------------------


def toeplitz_diagonals(T: np.ndarray) -> dict:
    """t_d = T[i, i-d] for d = -(n-1)..(n-1) of a Toeplitz matrix."""
    n = T.shape[0]
    return {d: T[max(d, 0), max(d, 0) - d] for d in range(-(n - 1), n)}


def circulant_from_column(c: np.ndarray) -> np.ndarray:
    n = len(c)
    C = np.empty((n, n), dtype=c.dtype)
    for i in range(n):
        for k in range(n):
            C[i, k] = c[(i - k) % n]
    return C


def strang_column(T: np.ndarray) -> np.ndarray:
    """First column of Strang's circulant s(T): copy the central diagonals."""
    n = T.shape[0]
    t = toeplitz_diagonals(T)
    c = np.empty(n)
    for k in range(n):
        c[k] = t[k] if k <= n // 2 else t[k - n]
    return c


def tchan_column(T: np.ndarray) -> np.ndarray:
    """First column of T. Chan's optimal circulant: c_k = ((n-k) t_k + k t_{k-n}) / n."""
    n = T.shape[0]
    t = toeplitz_diagonals(T)
    c = np.empty(n)
    c[0] = t[0]
    for k in range(1, n):
        c[k] = ((n - k) * t[k] + k * t[k - n]) / n
    return c


def preconditioner_matrix(prob, j: int, kind: Optional[str] = None) -> np.ndarray:
    """P^{(j+sigma)} of Eq. (3.7): eta I - sigma (q s(Q) + kappa_+ s(W) + kappa_- s(W^T)).

    The term for W^T is taken as s(W)^T, whose eigenvalues are the conjugates of those of s(W):
    the diagonalisation that follows Eq. (3.7) writes s(W^T) = F* conj(Lambda_beta) F.  For odd n
    (and for T. Chan's circulant at any n) s(W)^T equals the circulant approximation of W^T
    itself; for even n Strang's choice of the middle diagonal makes them differ, and the
    paper's eigenvalue formula is followed."""
    kind = kind or prob.preconditioner
    n = prob.n
    sigma = 1.0 - prob.alpha / 2.0
    e, q, kp, km = level_scalars(prob, j)
    col = strang_column if kind == "strang" else tchan_column
    Q, W = matrix_Q(n), matrix_W(prob.beta, n)
    sQ = circulant_from_column(col(Q))
    sW = circulant_from_column(col(W))
    return e * np.eye(n) - sigma * (q * sQ + kp * sW + km * sW.T)


def pcgs(A: np.ndarray, b: np.ndarray, P: Optional[np.ndarray], tol: float = 1e-12,
         maxit: int = 500):
    """Preconditioned conjugate gradient squared, zero initial guess (Section 4), in the form of
    Barrett et al., "Templates" (preconditioned CGS of Saad, pp. 241-244).  Stops when the
    recursively updated residual satisfies ||r_k|| / ||r_0|| < tol.  Returns (x, iterations,
    relative residual history)."""
    n = len(b)
    solveP = (lambda v: v) if P is None else (lambda v: np.linalg.solve(P, v))
    x = np.zeros(n)
    r = b.copy()
    rt = r.copy()
    nr0 = np.linalg.norm(r)
    hist = [1.0]
    if nr0 == 0.0:
        return x, 0, hist
    rho_old = 1.0
    p = q = None
    for it in range(1, maxit + 1):
        rho = float(rt @ r)
        if rho == 0.0:
            raise ArithmeticError("CGS breakdown: rho = 0")
        if it == 1:
            u = r.copy()
            p = u.copy()
        else:
            bet = rho / rho_old
            u = r + bet * q
            p = u + bet * (q + bet * p)
        ph = solveP(p)
        vh = A @ ph
        alpha = rho / float(rt @ vh)
        q = u - alpha * vh
        uh = solveP(u + q)
        x = x + alpha * uh
        r = r - alpha * (A @ uh)
        rho_old = rho
        rel = np.linalg.norm(r) / nr0
        hist.append(rel)
        if rel < tol:
            return x, it, hist
    return x, maxit, hist
