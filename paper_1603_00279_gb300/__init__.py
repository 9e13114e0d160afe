"""Python binding of libtsfcde (include/tsfcde.h): argument marshalling only.

Every step of the time march runs in the CUDA library; this module converts Python callables and
numpy arrays to the plain pointers of the C ABI and raises on error status.  If the compiled
library is missing, importing the functions raises: there is no CPU fallback.

    from paper_1603_00279_gb300 import Solver
    s = Solver(a, b, T, N, M, alpha, beta, gamma, d_plus, d_minus, phi, f, preconditioner="strang")
    u = s.solve()          # u^M at the N interior nodes
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Callable, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libtsfcde.so")
CHECKED_LIB_PATH = os.path.join(_HERE, "_lib", "checked", "libtsfcde_checked.so")

TSFCDE_OK = 0
STATUS_NAMES = {
    0: "OK", 1: "E_INVALID_ARG", 2: "E_NOMEM", 3: "E_CUDA", 4: "E_NONFINITE",
    5: "E_NOT_CONVERGED", 6: "E_BREAKDOWN", 7: "E_SINGULAR_PRECOND", 8: "E_TIMEOUT",
    9: "E_STATE", 10: "E_NO_DEVICE", 11: "E_BOUNDS",
}
PRECONDITIONERS = {"strang": 0, "tchan": 1, "none": 2}
PRECISIONS = {"fp64": 0, "mixed": 1}
INNER = {"auto": 0, "fp32": 1, "ff": 2}
OPS = {"A": 0, "B": 1, "Pinv": 2, "Ainv_gs": 3}
ALGORITHMS = {"ids": 0, "ids-const": 1}
INJECT = {None: 0, "nomem": 1, "breakdown": 2, "singular": 3}

COEF_FN = C.CFUNCTYPE(C.c_double, C.c_double, C.c_void_p)
FIELD_FN = C.CFUNCTYPE(None, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double),
                       C.c_int64, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("preconditioner", C.c_int32), ("tol", C.c_double),
                ("maxit", C.c_int32), ("device", C.c_int32), ("source_rank", C.c_int32),
                ("source_space", C.POINTER(FIELD_FN)), ("source_time", C.POINTER(COEF_FN)),
                ("levels_per_launch", C.c_int32), ("stream", C.c_void_p),
                ("inner_tol", C.c_double), ("inner_maxit", C.c_int32), ("outer_maxit", C.c_int32),
                ("barrier_spin_log2", C.c_int32), ("test_skip_arrival", C.c_int32),
                ("inner_precision", C.c_int32), ("autotune", C.c_int32),
                ("algorithm", C.c_int32), ("test_inject", C.c_int32),
                ("fast_history", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("level", C.c_int64), ("levels_advanced", C.c_int64),
                ("total_iterations", C.c_int64), ("max_iterations", C.c_int32),
                ("min_iterations", C.c_int32), ("max_residual", C.c_double),
                ("status", C.c_int32), ("device_launches", C.c_int32),
                ("device_ms", C.c_double), ("outer_iterations", C.c_int64),
                ("escalated_levels", C.c_int32), ("gsf_levels", C.c_int32),
                ("floor_levels", C.c_int32), ("pad_", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Instance(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("T", C.c_double), ("N", C.c_int64),
                ("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("d_plus", C.c_double), ("d_minus", C.c_double), ("phi", FIELD_FN),
                ("user", C.c_void_p)]


class TsfcdeError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({status})")
        self.status = status


_lib = None


def load_library(path: Optional[str] = None) -> C.CDLL:
    """Load libtsfcde.so (built by paper_1603_00279_gb300.build) and declare its signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libtsfcde.so not built ({p}); run paper_1603_00279_gb300.build.build()")
    lib = C.CDLL(p)
    vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    pd = C.POINTER(C.c_double)
    lib.tsfcde_default_options.argtypes = [C.POINTER(Options)]
    lib.tsfcde_default_options.restype = None
    lib.tsfcde_setup.argtypes = [C.POINTER(vp), dbl, dbl, dbl, i64, i64, dbl, dbl, COEF_FN, COEF_FN,
                                 COEF_FN, FIELD_FN, FIELD_FN, vp, C.POINTER(Options)]
    lib.tsfcde_setup.restype = C.c_int
    lib.tsfcde_step.argtypes = [vp, i64, C.POINTER(Stats)]
    lib.tsfcde_step.restype = C.c_int
    lib.tsfcde_solve.argtypes = [vp, pd, C.POINTER(Stats)]
    lib.tsfcde_solve.restype = C.c_int
    lib.tsfcde_get_level.argtypes = [vp, i64, pd]
    lib.tsfcde_get_level.restype = C.c_int
    lib.tsfcde_level.argtypes = [vp, C.POINTER(i64)]
    lib.tsfcde_level.restype = C.c_int
    lib.tsfcde_get_weights.argtypes = [vp, pd, pd]
    lib.tsfcde_get_weights.restype = C.c_int
    lib.tsfcde_reset.argtypes = [vp, pd]
    lib.tsfcde_reset.restype = C.c_int
    lib.tsfcde_get_history.argtypes = [vp, C.POINTER(i32), pd, i64]
    lib.tsfcde_get_history.restype = C.c_int
    lib.tsfcde_get_plan.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), pd]
    lib.tsfcde_get_plan.restype = C.c_int
    lib.tsfcde_history_sum.argtypes = [vp, i64, i32, pd]
    lib.tsfcde_history_sum.restype = C.c_int
    lib.tsfcde_apply.argtypes = [vp, i32, i64, pd, pd]
    lib.tsfcde_apply.restype = C.c_int
    lib.tsfcde_apply_operator_static.argtypes = [i64, dbl, dbl, dbl, dbl, dbl, dbl, i32, vp, vp, vp]
    lib.tsfcde_apply_operator_static.restype = C.c_int
    lib.tsfcde_batch_setup.argtypes = [C.POINTER(vp), i64, C.POINTER(Instance), i64, C.POINTER(Options)]
    lib.tsfcde_batch_setup.restype = C.c_int
    lib.tsfcde_batch_step.argtypes = [vp, i64, C.POINTER(Stats)]
    lib.tsfcde_batch_step.restype = C.c_int
    lib.tsfcde_batch_get_level.argtypes = [vp, i64, i64, pd]
    lib.tsfcde_batch_get_level.restype = C.c_int
    lib.tsfcde_batch_level.argtypes = [vp, C.POINTER(i64)]
    lib.tsfcde_batch_level.restype = C.c_int
    lib.tsfcde_batch_get_history.argtypes = [vp, i64, C.POINTER(i32), pd, i64]
    lib.tsfcde_batch_get_history.restype = C.c_int
    lib.tsfcde_batch_reset.argtypes = [vp]
    lib.tsfcde_batch_reset.restype = C.c_int
    lib.tsfcde_batch_set_initial.argtypes = [vp, vp]
    lib.tsfcde_batch_set_initial.restype = C.c_int
    lib.tsfcde_batch_get_all.argtypes = [vp, vp]
    lib.tsfcde_batch_solve.argtypes = [vp, vp, C.POINTER(Stats)]
    lib.tsfcde_batch_solve.restype = C.c_int
    lib.tsfcde_batch_get_plan.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                          C.POINTER(dbl)]
    lib.tsfcde_batch_get_plan.restype = C.c_int
    lib.tsfcde_batch_get_all.restype = C.c_int
    lib.tsfcde_batch_free.argtypes = [vp]
    lib.tsfcde_batch_free.restype = None
    lib.tsfcde_free.argtypes = [vp]
    lib.tsfcde_free.restype = None
    lib.tsfcde_strerror.argtypes = [C.c_int]
    lib.tsfcde_strerror.restype = C.c_char_p
    lib.tsfcde_version.argtypes = []
    lib.tsfcde_version.restype = C.c_char_p
    lib.tsfcde_checked_report.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
    lib.tsfcde_checked_report.restype = C.c_int
    lib.tsfcde_measure_fp64.argtypes = [i32, C.POINTER(dbl)]
    lib.tsfcde_measure_fp64.restype = C.c_int
    if path is None:
        _lib = lib
    return lib


_checked = None


def load_checked_library() -> C.CDLL:
    """libtsfcde_checked.so, the -DTSFCDE_CHECKED build (built by build.build(checked=True))."""
    global _checked
    if _checked is None:
        _checked = load_library(CHECKED_LIB_PATH)
    return _checked


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _check(st: int, where: str, allow_not_converged: bool = False):
    if st == TSFCDE_OK or (allow_not_converged and st == 5):
        return
    raise TsfcdeError(st, where)


class Solver:
    """One TSFCDE instance on the GPU (wraps tsfcde_setup ... tsfcde_free).

    gamma, d_plus, d_minus: callables t -> float.  phi: callable x (ndarray) -> ndarray.
    f: callable (x ndarray, t) -> ndarray, or None; alternatively `separable` = list of
    (T_r(t), X_r(x)) pairs passed as callbacks; the library samples them on its own mesh.
    test_inject: None, or "nomem" / "breakdown" / "singular" (tsfcde_options.test_inject).
    """

    def __init__(self, a, b, T, N, M, alpha, beta, gamma: Callable, d_plus: Callable,
                 d_minus: Callable, phi: Callable, f: Optional[Callable] = None,
                 separable=None, preconditioner: str = "strang", tol: float = 1e-12,
                 maxit: int = 2000, device: int = 0, levels_per_launch: int = 0,
                 stream: Optional[int] = None, precision: str = "fp64",
                 inner_tol: Optional[float] = None, inner_maxit: Optional[int] = None,
                 outer_maxit: Optional[int] = None, barrier_spin_log2: Optional[int] = None,
                 test_skip_arrival: bool = False, inner: str = "auto", autotune: bool = False,
                 algorithm: str = "ids", test_inject: Optional[str] = None,
                 fast_history: bool = False, lib: Optional[C.CDLL] = None):
        self.lib = lib if lib is not None else load_library()
        self.N, self.M = int(N), int(M)
        self._keep = []

        def coef(fn):
            cb = COEF_FN(lambda t, _u: float(fn(t)))
            self._keep.append(cb)
            return cb

        def field(fn, with_t):
            def call(t, xp, outp, n, _u):
                x = np.ctypeslib.as_array(xp, shape=(n,))
                out = np.ctypeslib.as_array(outp, shape=(n,))
                out[:] = np.broadcast_to(fn(x, t) if with_t else fn(x), (n,))
            cb = FIELD_FN(call)
            self._keep.append(cb)
            return cb

        opt = Options()
        self.lib.tsfcde_default_options(C.byref(opt))
        opt.preconditioner = PRECONDITIONERS[preconditioner]
        opt.tol = tol
        opt.maxit = maxit
        opt.device = device
        opt.levels_per_launch = levels_per_launch
        opt.stream = stream
        opt.precision = PRECISIONS[precision]
        if inner_tol is not None:
            opt.inner_tol = inner_tol
        if inner_maxit is not None:
            opt.inner_maxit = inner_maxit
        if outer_maxit is not None:
            opt.outer_maxit = outer_maxit
        if barrier_spin_log2 is not None:
            opt.barrier_spin_log2 = barrier_spin_log2
        opt.test_skip_arrival = 1 if test_skip_arrival else 0
        opt.inner_precision = INNER[inner]
        opt.autotune = 1 if autotune else 0
        opt.algorithm = ALGORITHMS[algorithm]
        opt.test_inject = INJECT[test_inject]
        opt.fast_history = 1 if fast_history else 0
        f_cb = FIELD_FN() if f is None else field(f, True)
        if separable is not None:
            if f is not None:
                raise ValueError("give either f or separable")
            spaces = (FIELD_FN * len(separable))(*[field(Xr, False) for _, Xr in separable])
            times = (COEF_FN * len(separable))(*[coef(Tr) for Tr, _ in separable])
            self._keep += [spaces, times]
            opt.source_rank = len(separable)
            opt.source_space = C.cast(spaces, C.POINTER(FIELD_FN))
            opt.source_time = C.cast(times, C.POINTER(COEF_FN))
        ctx = C.c_void_p()
        stt = self.lib.tsfcde_setup(C.byref(ctx), a, b, T, self.N, self.M, alpha, beta, coef(gamma),
                                    coef(d_plus), coef(d_minus), field(phi, False), f_cb, None,
                                    C.byref(opt))
        _check(stt, "tsfcde_setup")
        self.ctx = ctx

    @classmethod
    def from_problem(cls, prob, source: str = "callback", **kw):
        """Build from a tsfcde_workloads.Problem-like object."""
        f = prob.f if source == "callback" else None
        sep = prob.separable if source == "separable" else None
        if source == "separable" and sep is None:
            f = None
        return cls(prob.a, prob.b, prob.T, prob.n, prob.M, prob.alpha, prob.beta, prob.gamma,
                   prob.d_plus, prob.d_minus, prob.phi, f, separable=sep,
                   preconditioner=kw.pop("preconditioner", prob.preconditioner),
                   tol=kw.pop("tol", prob.tol), **kw)

    def step(self, nsteps: int = 1) -> dict:
        s = Stats()
        _check(self.lib.tsfcde_step(self.ctx, nsteps, C.byref(s)), "tsfcde_step", True)
        return s.as_dict()

    def solve(self, out: Optional[np.ndarray] = None, out_ptr: Optional[int] = None):
        """Advance to level M; copy u^M to `out` (numpy) or to the raw host address out_ptr."""
        s = Stats()
        if out_ptr is not None:
            p = C.cast(C.c_void_p(out_ptr), C.POINTER(C.c_double))
        else:
            out = np.empty(self.N) if out is None else out
            p = _dptr(out)
        _check(self.lib.tsfcde_solve(self.ctx, p, C.byref(s)), "tsfcde_solve", True)
        self.last_stats = s.as_dict()
        return out if out_ptr is None else None

    def level(self) -> int:
        """The current level j of the march."""
        j = C.c_int64()
        _check(self.lib.tsfcde_level(self.ctx, C.byref(j)), "tsfcde_level")
        return j.value

    def get_level(self, j: Optional[int] = None):
        """(u^j, j) for any j <= the current level (default: the current level)."""
        cur = self.level()
        j = cur if j is None else int(j)
        out = np.empty(self.N)
        _check(self.lib.tsfcde_get_level(self.ctx, j, _dptr(out)), "tsfcde_get_level")
        return out, j

    def weights(self):
        """(g_k, omega_k) for k = 0..N+1 as the library computed them (Lemmas 2-3)."""
        g = np.empty(self.N + 2)
        w = np.empty(self.N + 2)
        _check(self.lib.tsfcde_get_weights(self.ctx, _dptr(g), _dptr(w)), "tsfcde_get_weights")
        return g, w

    def reset(self, u0: Optional[np.ndarray] = None, u0_ptr: Optional[int] = None):
        """Back to level 0 with u^0 = u0 (numpy), the host address u0_ptr, or phi."""
        if u0_ptr is not None:
            p = C.cast(C.c_void_p(u0_ptr), C.POINTER(C.c_double))
        else:
            p = None if u0 is None else _dptr(np.ascontiguousarray(u0, dtype=np.float64))
        _check(self.lib.tsfcde_reset(self.ctx, p), "tsfcde_reset")

    def history(self, count: int):
        it = np.zeros(count, dtype=np.int32)
        rs = np.zeros(count)
        _check(self.lib.tsfcde_get_history(self.ctx, it.ctypes.data_as(C.POINTER(C.c_int32)),
                                           _dptr(rs), count), "tsfcde_get_history")
        return it, rs

    def plan(self) -> dict:
        """The FFT plan in use (autotuner's choice when autotune was requested)."""
        n1, n2, b = C.c_int32(), C.c_int32(), C.c_int32()
        us = C.c_double()
        _check(self.lib.tsfcde_get_plan(self.ctx, C.byref(n1), C.byref(n2), C.byref(b), C.byref(us)),
               "tsfcde_get_plan")
        return {"N1": n1.value, "N2": n2.value, "budget": b.value, "best_us": us.value}

    def checked_report(self):
        """(site, index) of the first index violation caught (checked build), or (0, 0)."""
        site, idx = C.c_int32(), C.c_int32()
        _check(self.lib.tsfcde_checked_report(self.ctx, C.byref(site), C.byref(idx)),
               "tsfcde_checked_report")
        return site.value, idx.value

    def history_sum(self, j: int, want: bool = True, direct: bool = False):
        """Lemma 1 history sum of level j (unscaled), by the march's device phases (direct=True:
        always the term-by-term sum)."""
        out = np.empty(self.N) if want else None
        _check(self.lib.tsfcde_history_sum(self.ctx, j, 1 if direct else 0,
                                           _dptr(out) if want else None), "tsfcde_history_sum")
        return out

    def apply(self, op: str, j: int, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.N)
        _check(self.lib.tsfcde_apply(self.ctx, OPS[op], j, _dptr(x), _dptr(y)), "tsfcde_apply")
        return y

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.tsfcde_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Independent constant-coefficient instances advanced together (tsfcde_batch_*).

    problems: objects with a, b, T, n, alpha, beta, gamma(t), d_plus(t), d_minus(t), phi(x)
    (coefficients are sampled once, at t = 0, since batched instances take constants); all
    share M."""

    def __init__(self, problems, M: int, preconditioner: str = "strang", tol: float = 1e-12,
                 maxit: int = 2000, precision: str = "fp64", device: int = 0,
                 stream: Optional[int] = None, inner: str = "auto", algorithm: str = "ids",
                 inner_tol: Optional[float] = None, autotune: bool = False,
                 test_inject: Optional[str] = None, lib: Optional[C.CDLL] = None):
        self.lib = lib if lib is not None else load_library()
        self.M = int(M)
        self.n = [int(p.n) for p in problems]
        self._keep = []

        def field(fn):
            def call(t, xp, outp, n, _u):
                x = np.ctypeslib.as_array(xp, shape=(n,))
                out = np.ctypeslib.as_array(outp, shape=(n,))
                out[:] = np.broadcast_to(fn(x), (n,))
            cb = FIELD_FN(call)
            self._keep.append(cb)
            return cb

        arr = (Instance * len(problems))()
        for k, p in enumerate(problems):
            arr[k] = Instance(p.a, p.b, p.T, p.n, p.alpha, p.beta, float(p.gamma(0.0)),
                              float(p.d_plus(0.0)), float(p.d_minus(0.0)), field(p.phi), None)
        opt = Options()
        self.lib.tsfcde_default_options(C.byref(opt))
        opt.preconditioner = PRECONDITIONERS[preconditioner]
        opt.tol = tol
        opt.maxit = maxit
        opt.precision = PRECISIONS[precision]
        opt.device = device
        opt.stream = stream
        opt.inner_precision = INNER[inner]
        opt.algorithm = ALGORITHMS[algorithm]
        if inner_tol is not None:
            opt.inner_tol = inner_tol
        opt.autotune = 1 if autotune else 0
        opt.test_inject = INJECT[test_inject]
        h = C.c_void_p()
        _check(self.lib.tsfcde_batch_setup(C.byref(h), len(problems), arr, self.M, C.byref(opt)),
               "tsfcde_batch_setup")
        self.h = h

    def step(self, nsteps: int = 1) -> dict:
        s = Stats()
        _check(self.lib.tsfcde_batch_step(self.h, nsteps, C.byref(s)), "tsfcde_batch_step", True)
        return s.as_dict()

    def solve(self) -> list:
        """Advance every instance to level M; returns the list of u^M (numpy arrays)."""
        st = Stats()
        out = np.empty(sum(self.n))
        _check(self.lib.tsfcde_batch_solve(self.h, _dptr(out), C.byref(st)), "tsfcde_batch_solve", True)
        self.last_stats = st.as_dict()
        parts, k = [], 0
        for n in self.n:
            parts.append(out[k:k + n].copy())
            k += n
        return parts

    def plan(self) -> dict:
        """The batched launch's plan (the tuner's choice when autotune was requested)."""
        bud, big, ctas = C.c_int32(), C.c_int32(), C.c_int32()
        ms = C.c_double()
        _check(self.lib.tsfcde_batch_get_plan(self.h, C.byref(bud), C.byref(big), C.byref(ctas),
                                              C.byref(ms)), "tsfcde_batch_get_plan")
        return {"budget": bud.value, "n1_ge_n2": bool(big.value), "ctas": ctas.value,
                "best_ms": ms.value}

    def level(self) -> int:
        """The batch's current level."""
        j = C.c_int64()
        _check(self.lib.tsfcde_batch_level(self.h, C.byref(j)), "tsfcde_batch_level")
        return j.value

    def get_level(self, i: int, j: Optional[int] = None):
        """(u^j of instance i, j) for any j <= the current level (default: the current level)."""
        j = self.level() if j is None else int(j)
        out = np.empty(self.n[i])
        _check(self.lib.tsfcde_batch_get_level(self.h, i, j, _dptr(out)), "tsfcde_batch_get_level")
        return out, j

    def history(self, i: int, count: int):
        it = np.zeros(count, dtype=np.int32)
        rs = np.zeros(count)
        _check(self.lib.tsfcde_batch_get_history(self.h, i, it.ctypes.data_as(C.POINTER(C.c_int32)),
                                                 _dptr(rs), count), "tsfcde_batch_get_history")
        return it, rs

    def reset(self):
        _check(self.lib.tsfcde_batch_reset(self.h), "tsfcde_batch_reset")

    def set_initial(self, u0_ptr: int):
        """New u^0 for every instance from the host address u0_ptr (sum N_i doubles)."""
        _check(self.lib.tsfcde_batch_set_initial(self.h, u0_ptr), "tsfcde_batch_set_initial")

    def get_all(self, u_ptr: int):
        """Every instance's current level into the host address u_ptr (sum N_i doubles)."""
        _check(self.lib.tsfcde_batch_get_all(self.h, u_ptr), "tsfcde_batch_get_all")

    def close(self):
        if getattr(self, "h", None):
            self.lib.tsfcde_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def apply_operator_static(N: int, beta: float, sigma: float, eta: float, q: float,
                          kappa_plus: float, kappa_minus: float, op: str, x_ptr: int, y_ptr: int,
                          stream: Optional[int] = None) -> None:
    """y = A x or B x of one level with no device allocation (tsfcde_apply_operator_static);
    x_ptr and y_ptr are device addresses of N float64 values."""
    st = load_library().tsfcde_apply_operator_static(N, beta, sigma, eta, q, kappa_plus,
                                                      kappa_minus, OPS[op], x_ptr, y_ptr, stream)
    _check(st, "tsfcde_apply_operator_static")


def measure_fp64(device: int = 0) -> float:
    """FP64 FMA throughput of the device in TFLOP/s (tsfcde_measure_fp64)."""
    v = C.c_double()
    _check(load_library().tsfcde_measure_fp64(device, C.byref(v)), "tsfcde_measure_fp64")
    return v.value


def strerror(status: int) -> str:
    return load_library().tsfcde_strerror(status).decode()
