"""The index-checked build (libtsfcde_checked.so, -DTSFCDE_CHECKED): every checked device access
compares its index with its array's length; an index outside sets TSFCDE_E_BOUNDS and the
first failing site and index, and is redirected to element 0 instead of being accessed (no trap).
Tiny problems (N <= 16) through every kind of launch -- the one-CTA and whole-grid marches in
FP64 and mixed precision, the three preconditioners, the constant-coefficient algorithm, fast
history, the batch, the diagnostic products -- must report no violation and still match the
oracle."""
import numpy as np
import pytest

import oracle as O
import tsfcde_workloads as W
from gpu_common import rel_l2

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1603_00279_gb300 as P
    from paper_1603_00279_gb300 import build
    build.build(checked=True)
    return P, P.load_checked_library()


@pytest.mark.parametrize("n", [1, 2, 5, 16])
@pytest.mark.parametrize("kw", [dict(), dict(preconditioner="tchan"), dict(preconditioner="none"),
                                dict(precision="mixed"), dict(algorithm="ids-const")])
def test_checked_build_reports_no_violation(n, kw):
    P, lib = _lib()
    const = kw.get("algorithm") == "ids-const"
    prob = (W.config_batch(count=1, M=5, n_lo=n, n_hi=n, seed=3)[0] if const
            else W.config_small(n=n, M=5, preconditioner=kw.get("preconditioner", "strang")))
    ref = O.run(prob)
    args = {k: v for k, v in kw.items() if k != "preconditioner"}
    with P.Solver.from_problem(prob, lib=lib, preconditioner=kw.get("preconditioner", "strang"),
                               **args) as s:
        st = s.step(prob.M)
        assert st["status"] in (0, 5), st
        assert s.checked_report() == (0, 0)
        tol = 1e-4 if kw.get("preconditioner") == "none" else 1e-10
        assert rel_l2(s.get_level()[0], ref[-1]) <= tol
        for op in ("A", "B"):
            s.apply(op, 1, np.linspace(0.0, 1.0, n))
        s.history_sum(prob.M)
        assert s.checked_report() == (0, 0)


def test_checked_build_whole_grid_fast_history_and_batch():
    """n = 300 (whole grid, fast history past level 128), and a batch of three tiny instances."""
    P, lib = _lib()
    prob = W.config_small(n=300, M=140)
    with P.Solver.from_problem(prob, lib=lib, fast_history=True) as s:
        s.step(prob.M)
        assert s.checked_report() == (0, 0)
        assert rel_l2(s.get_level()[0], O.run(prob)[-1]) <= 1e-10
    probs = W.config_batch(count=3, M=4, n_lo=9, n_hi=16, seed=5)
    b = P.Batch(probs, 4, lib=lib)
    st = b.step(4)
    assert st["status"] == 0
    for i, q in enumerate(probs):
        assert rel_l2(b.get_level(i)[0], O.run(q)[-1]) <= 1e-10
    b.close()
