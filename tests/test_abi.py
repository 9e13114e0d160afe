"""The C-ABI library builds, loads and exports every function include/tsfcde.h declares; argument
errors are reported before any device work (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tsfcde.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(tsfcde_[a-z_]+)\s*\(", src))
    return sorted(n for n in names if not n.endswith("_fn"))


def _lib():
    from paper_1603_00279_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_exports_every_declared_symbol():
    lib = _lib()
    names = _declared()
    assert {"tsfcde_setup", "tsfcde_step", "tsfcde_solve", "tsfcde_free"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_invalid_arguments_rejected_without_device():
    import paper_1603_00279_gb300 as P
    P.load_library()
    with pytest.raises(P.TsfcdeError) as e:
        P.Solver(0.0, 1.0, 1.0, 15, 4, 0.0, 1.5, lambda t: 0, lambda t: 1, lambda t: 1,
                 lambda x: x * 0)
    assert e.value.status == 1
    with pytest.raises(P.TsfcdeError) as e:
        P.Solver(0.0, 1.0, 1.0, 15, 4, 0.5, 1.0, lambda t: 0, lambda t: 1, lambda t: 1,
                 lambda x: x * 0)
    assert e.value.status == 1
    with pytest.raises(P.TsfcdeError) as e:
        P.Solver(1.0, 0.0, 1.0, 15, 4, 0.5, 1.5, lambda t: 0, lambda t: 1, lambda t: 1,
                 lambda x: x * 0)
    assert e.value.status == 1


def test_strerror_and_version():
    import paper_1603_00279_gb300 as P
    assert P.strerror(0) == "ok"
    assert "converge" in P.strerror(5)
    assert b"sm_103a" in P.load_library().tsfcde_version()


def test_invalid_options_rejected_without_device():
    """Option checks (algorithm, precision, preconditioner, tolerances, barrier bound) come before
    any device call, and the batch entry point checks the same options."""
    import paper_1603_00279_gb300 as P
    lib = P.load_library()
    base = dict(a=0.0, b=1.0, T=1.0, N=15, M=4, alpha=0.5, beta=1.5, gamma=lambda t: 0,
                d_plus=lambda t: 1, d_minus=lambda t: 1, phi=lambda x: x * 0)
    bad = [dict(preconditioner="nope")]
    for kw in bad:
        with pytest.raises(KeyError):
            P.Solver(**base, **kw)
    def opt_with(**fields):
        o = P.Options()
        lib.tsfcde_default_options(C.byref(o))
        for k, v in fields.items():
            setattr(o, k, v)
        return o
    coef = P.COEF_FN(lambda t, u: 1.0)
    phi = P.FIELD_FN(lambda t, x, out, n, u: None)
    for fields in [dict(algorithm=7), dict(algorithm=-1), dict(precision=3), dict(preconditioner=5),
                   dict(tol=0.0), dict(maxit=0), dict(barrier_spin_log2=2), dict(inner_precision=9),
                   dict(precision=1, inner_tol=2.0), dict(test_inject=4), dict(test_inject=-1),
                   dict(source_rank=2)]:
        o = opt_with(**fields)
        ctx = C.c_void_p()
        st = lib.tsfcde_setup(C.byref(ctx), 0.0, 1.0, 1.0, 15, 4, 0.5, 1.5, coef, coef, coef, phi,
                              P.FIELD_FN(), None, C.byref(o))
        assert st == 1, fields
        assert not ctx.value
    inst = (P.Instance * 1)(P.Instance(0.0, 1.0, 1.0, 15, 0.5, 1.5, 0.1, 1.0, 1.0, phi, None))
    for fields in [dict(algorithm=3), dict(precision=5), dict(maxit=0), dict(test_inject=2),
                   dict(test_inject=3)]:
        o = opt_with(**fields)
        h = C.c_void_p()
        assert lib.tsfcde_batch_setup(C.byref(h), 1, inst, 4, C.byref(o)) == 1, fields


def test_header_is_c99_and_links():
    """A plain C99 program compiled against include/tsfcde.h and linked to libtsfcde.so calls the
    entry points that need no device (defaults, strerror, version, argument checks, NULL frees)."""
    import shutil
    import subprocess
    import tempfile
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    from paper_1603_00279_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "abi_c_check")
        r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror",
                            "-I", os.path.join(ROOT, "include"),
                            os.path.join(ROOT, "tests", "abi_c_check.c"), "-o", exe,
                            "-L", libdir, "-ltsfcde", "-Wl,-rpath," + libdir],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
        assert r.returncode == 0 and "c abi ok" in r.stdout, (r.returncode, r.stdout, r.stderr)


def test_product_never_uses_the_oracle():
    """The package (binding, build, host helpers and CUDA sources) neither imports nor names the
    oracle: the product path is the CUDA library alone."""
    pkg = os.path.join(ROOT, "paper_1603_00279_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_lib" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
                assert "ids_oracle" not in src, f


def test_binding_fails_loudly_without_the_library():
    import paper_1603_00279_gb300 as P
    with pytest.raises(RuntimeError):
        P.load_library(os.path.join(ROOT, "paper_1603_00279_gb300", "_lib", "missing.so"))


def test_empty_and_oversize_problems_rejected_without_device():
    """N = 0, M = 0 and N beyond 2^22 - 1 are argument errors, as is an empty or oversize batch."""
    import paper_1603_00279_gb300 as P
    lib = P.load_library()
    opt = P.Options()
    lib.tsfcde_default_options(C.byref(opt))
    coef = P.COEF_FN(lambda t, u: 1.0)
    phi = P.FIELD_FN(lambda t, x, out, n, u: None)
    for N, M in [(0, 4), (15, 0), (1 << 22, 4), (-3, 4)]:
        ctx = C.c_void_p()
        st = lib.tsfcde_setup(C.byref(ctx), 0.0, 1.0, 1.0, N, M, 0.5, 1.5, coef, coef, coef, phi,
                              P.FIELD_FN(), None, C.byref(opt))
        assert st == 1 and not ctx.value, (N, M)
    h = C.c_void_p()
    assert lib.tsfcde_batch_setup(C.byref(h), 0, None, 4, C.byref(opt)) == 1
    big = (P.Instance * 1)(P.Instance(0.0, 1.0, 1.0, 16384, 0.5, 1.5, 0.1, 1.0, 1.0, phi, None))
    assert lib.tsfcde_batch_setup(C.byref(h), 1, big, 4, C.byref(opt)) == 1
    ok = (P.Instance * 1)(P.Instance(0.0, 1.0, 1.0, 15, 0.5, 1.5, 0.1, 1.0, 1.0, phi, None))
    assert lib.tsfcde_batch_setup(C.byref(h), 1, ok, 0, C.byref(opt)) == 1
    nophi = (P.Instance * 1)(P.Instance(0.0, 1.0, 1.0, 15, 0.5, 1.5, 0.1, 1.0, 1.0, P.FIELD_FN(), None))
    assert lib.tsfcde_batch_setup(C.byref(h), 1, nophi, 4, C.byref(opt)) == 1


def test_nonfinite_callbacks_rejected_before_any_device_work():
    """A coefficient, initial value, source or separable-source callback that returns NaN or Inf
    makes setup return E_NONFINITE (4).  Every callback is sampled on the host, on the library's
    own mesh, before any CUDA call, so this holds on a machine without a GPU; so does the batch's
    initial value."""
    import math
    import paper_1603_00279_gb300 as P
    P.load_library()
    base = dict(a=0.0, b=1.0, T=1.0, N=15, M=4, alpha=0.5, beta=1.5, gamma=lambda t: 0.5,
                d_plus=lambda t: 1.0, d_minus=lambda t: 1.0, phi=lambda x: x * (1 - x))
    nan = float("nan")
    cases = [dict(gamma=lambda t: nan if t > 0.3 else 0.5),
             dict(d_plus=lambda t: math.inf),
             dict(d_minus=lambda t: nan),
             dict(phi=lambda x: x / (x - x[3])),                       # Inf at one node
             dict(f=lambda x, t: np.where(x > 0.5, nan, 0.0)),
             dict(separable=[(lambda t: 1.0, lambda x: x), (lambda t: nan, lambda x: x)]),
             dict(separable=[(lambda t: 1.0, lambda x: np.log(x - 0.5))])]
    for kw in cases:
        args = dict(base, **kw)
        with pytest.raises(P.TsfcdeError) as e:
            P.Solver(**args)
        assert e.value.status == 4, kw
    # a negative diffusion coefficient at some t_{j+sigma} is an argument error, found on the host
    with pytest.raises(P.TsfcdeError) as e:
        P.Solver(**dict(base, d_minus=lambda t: 1.0 - 2.0 * t))
    assert e.value.status == 1

    class Q:
        a, b, T, n, alpha, beta = 0.0, 1.0, 1.0, 15, 0.5, 1.5
        gamma = staticmethod(lambda t: 0.1)
        d_plus = staticmethod(lambda t: 1.0)
        d_minus = staticmethod(lambda t: 1.0)
        phi = staticmethod(lambda x: np.where(x > 0.9, nan, x))
    with pytest.raises(P.TsfcdeError) as e:
        P.Batch([Q()], 4)
    assert e.value.status == 4


def test_separable_source_sampled_by_the_library_on_its_mesh():
    """The separable source's callbacks receive the library's mesh: X_r is called once with the N
    interior nodes x_i = a + i h, T_r once per level at t_{j+sigma} = (j + sigma) tau (Section 2.1
    and Eq. (2.1)).  Recorded on the host during setup, which then fails with a NaN on purpose so
    that no device is needed."""
    import paper_1603_00279_gb300 as P
    P.load_library()
    seen_x, seen_t = [], []

    def X(x):
        seen_x.append(np.array(x))
        return x

    def T(t):
        seen_t.append(t)
        return float("nan") if len(seen_t) == 5 else 1.0
    a, b, N, M, Tf, alpha = -1.0, 2.0, 11, 5, 0.5, 0.4
    with pytest.raises(P.TsfcdeError) as e:
        P.Solver(a, b, Tf, N, M, alpha, 1.5, lambda t: 0.0, lambda t: 1.0, lambda t: 1.0,
                 lambda x: 0 * x, separable=[(T, X)])
    assert e.value.status == 4
    h = (b - a) / (N + 1)
    assert len(seen_x) == 1 and np.array_equal(seen_x[0], a + h * np.arange(1, N + 1))
    sigma = 1.0 - alpha / 2.0
    assert seen_t == [(j + sigma) * (Tf / M) for j in range(M)]
