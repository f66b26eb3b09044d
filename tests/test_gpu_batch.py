"""Persistent 1D batch execution (lelbm_run_batch, CUDA graph, autotuner, step budgets)."""
import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L, workloads as W
from paper_2508_06911_gb300.solver import Solver

import oracle as O
from parity_util import assert_close, oracle_1d_instance

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    O.build()


@pytest.mark.parametrize("precision", [L.LELBM_FP64, L.LELBM_MIXED])
def test_run_batch_equals_per_step_launches(precision):
    w = W.riemann_1d_batch(n_batch=40, seed_index=505, lmin=16, lmax=300)
    a = Solver.riemann1d(w, precision=precision)
    b = Solver.riemann1d(w, precision=precision)
    a.step(3)
    b.run_batch(3)
    tol = 3 * (STEP_TOL if precision == L.LELBM_FP64 else 1e-11)
    assert_close(b.get_moments(), a.get_moments(), tol, "run_batch vs step")
    sa, sb = a.stats(), b.stats()
    assert sa.cells == sb.cells
    a.close()
    b.close()


def test_run_batch_budgets_against_oracle():
    """Each instance stops after its own step count (run to t_end instance by instance)."""
    w = W.riemann_1d_batch(n_batch=8, seed_index=606, lmin=16, lmax=80)
    s = Solver.riemann1d(w)
    budgets = np.array([0, 1, 2, 3, 4, 5, 1, 2])
    s.set_steps(budgets)
    s.run_batch(3)   # instance b advances min(3, budget_b) steps
    s.run_batch(3)   # and the rest of its budget (up to 3 more)
    M = s.get_moments()
    for b in range(w.n_batch):
        first, n = s.instance(b)
        k = int(min(budgets[b], 6))
        ref = oracle_1d_instance(w, b, k)
        p = int(w.pads[b])
        assert_close(M[:, first:first + n], ref[:, p:p + n], max(k, 1) * STEP_TOL, f"instance {b}, {k} steps")
    s.close()


def test_autotune_keeps_state_and_picks_a_shape():
    w = W.riemann_1d_batch(n_batch=64, seed_index=707, lmin=32, lmax=400)
    s = Solver.riemann1d(w)
    M0 = s.get_moments()
    t = s.autotune(1)
    assert t.threads in (64, 128) and t.ms > 0
    np.testing.assert_array_equal(s.get_moments(), M0)
    ref = Solver.riemann1d(w)
    ref.step(2)
    s.run_batch(2)
    assert_close(s.get_moments(), ref.get_moments(), 2 * STEP_TOL, "tuned run_batch")
    s.close()
    ref.close()


def test_run_batch_rejects_2d():
    w = W.hot_box(2, 6, 0.5)
    s = Solver.grid2d(w)
    with pytest.raises(L.LelbmError):
        s.run_batch(1)
    s.close()
