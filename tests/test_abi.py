"""The C-ABI library builds, loads and exports every function include/tsfcde.h declares; argument
errors are reported before any device work (no GPU needed)."""
import ctypes as C
import os
import re

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
