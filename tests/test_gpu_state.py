"""State access through the C ABI and the host-injected failure paths.

* tsfcde_get_level(ctx, j, out) for any j <= the current level, rebuilt on the device from u^0,
  the current level and the ring of increments, against the oracle's levels (Algorithm "Practical
  implementation of IDS" produces every level u^j);
* tsfcde_get_weights: the Grunwald weights of Lemma 3 and the WSGD weights of Lemma 2, bit for
  bit equal to a plain binary64 evaluation of the lemmas' formulas (the oracle's);
* failure codes that valid inputs cannot reach, set off from the host (tsfcde_options.test_inject)
  with nothing faulting on the GPU: E_NOMEM, E_BREAKDOWN, E_SINGULAR_PRECOND.
"""
import numpy as np
import pytest

import oracle as O
import tsfcde_workloads as W
from gpu_common import rel_l2, solver_module

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,M,source", [(127, 64, "callback"), (1023, 24, "separable")])
def test_get_level_any_j_matches_oracle(n, M, source):
    """n = 127 runs the one-CTA march, n = 1023 the whole-grid march.  After the whole march the
    levels 0, M/2 and M (and a few others) are read back through the C ABI and compared with the
    oracle's elimination march at 1e-10; levels 0 and M come back bit for bit as stored."""
    P = solver_module()
    prob = W.config_small(n=n, M=M)
    ref = O.run(prob)
    s = P.Solver.from_problem(prob, source=source)
    u0, j0 = s.get_level(0)
    assert j0 == 0 and np.array_equal(u0, prob.phi(prob.grid()))
    st = s.step(M)
    assert s.level() == M and st["levels_advanced"] == M
    for j in sorted({0, 1, M // 3, M // 2, M - 1, M}):
        u, jj = s.get_level(j)
        assert jj == j
        assert rel_l2(u, ref[j]) <= 1e-10, (j, rel_l2(u, ref[j]))
    assert np.array_equal(s.get_level(0)[0], u0)
    last = s.get_level()[0]
    assert np.array_equal(s.get_level(M)[0], last)
    with pytest.raises(P.TsfcdeError) as e:
        s.get_level(M + 1)
    assert e.value.status == 1
    # a reset with new initial values: level 0 of the new march is what was given
    u0b = 0.5 * u0
    s.reset(u0b)
    s.step(3)
    assert np.array_equal(s.get_level(0)[0], u0b)
    s.close()


def test_batch_get_level_any_j_matches_oracle():
    P = solver_module()
    probs = W.config_batch(count=3, M=6, n_lo=255, n_hi=700, seed=11)
    b = P.Batch(probs, 6)
    b.step(6)
    assert b.level() == 6
    for i, q in enumerate(probs):
        ref = O.run(q)
        for j in (0, 3, 6):
            u, jj = b.get_level(i, j)
            assert jj == j and rel_l2(u, ref[j]) <= 1e-10, (i, j)
        assert np.array_equal(b.get_level(i, 0)[0], q.phi(q.grid()))
    b.close()


@pytest.mark.parametrize("beta", [1.05, 1.3, 1.5, 1.7, 1.9, 2.0])
@pytest.mark.parametrize("n", [127, 4095])
def test_weights_bit_exact(beta, n):
    """g_k and omega_k (k = 0..n+1) as the library computed them equal the oracle's plain binary64
    evaluation of Lemma 3's recurrence and Lemma 2's combination bit for bit."""
    P = solver_module()
    prob = W.config_small(n=n, M=2, beta=beta)
    with P.Solver.from_problem(prob) as s:
        g, w = s.weights()
    assert np.array_equal(g, O.grunwald_weights(beta, n + 1))
    assert np.array_equal(w, O.wsgd_weights(beta, n + 1))


def test_injected_nomem_single_and_batch():
    """The setup's device allocation reported as failed: E_NOMEM, everything released, and the
    next setup works."""
    P = solver_module()
    prob = W.config_small(n=127, M=4)
    with pytest.raises(P.TsfcdeError) as e:
        P.Solver.from_problem(prob, test_inject="nomem")
    assert e.value.status == 2
    probs = W.config_batch(count=2, M=4, n_lo=255, n_hi=300)
    with pytest.raises(P.TsfcdeError) as e:
        P.Batch(probs, 4, test_inject="nomem")
    assert e.value.status == 2
    ref = O.run(prob)
    with P.Solver.from_problem(prob) as s:
        assert rel_l2(s.solve(), ref[-1]) <= 1e-10


@pytest.mark.parametrize("n", [127, 1023])
@pytest.mark.parametrize("kind,code", [("breakdown", 6), ("singular", 7)])
def test_injected_device_conditions(kind, code, n):
    """CGS breakdown ((r~, A p^) = 0) and a vanishing preconditioner eigenvalue, injected into the
    first launch: the step returns the code, the call ends normally (no fault, no hang) and a new
    context on the same device then matches the oracle."""
    P = solver_module()
    prob = W.config_small(n=n, M=4)
    s = P.Solver.from_problem(prob, test_inject=kind)
    with pytest.raises(P.TsfcdeError) as e:
        s.step(2)
    assert e.value.status == code
    s.close()
    ref = O.run(prob)
    with P.Solver.from_problem(prob) as s2:
        assert rel_l2(s2.solve(), ref[-1]) <= 1e-10
