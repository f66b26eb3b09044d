"""Stored warm start (Sec. II.D: each cell's multipliers kept as the precondition of
its next step) against the CPU oracle.

The warm start changes only where the Newton iteration begins.  The FP64 path still
stops at the same 1e-12 residual and applies its polishing update, so it must match
the oracle within the same 1e-12 per step, the mixed path within its 1e-11 and the
FP32 path within its 2e-5.  From the second step on, the stored start must take fewer
Newton updates than Eq. (IID13).
"""
import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L, workloads as W
from paper_2508_06911_gb300.solver import Solver

import oracle as O
from parity_util import assert_close, oracle_1d_instance, oracle_2d

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12
FP32_TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    O.build()


def mean_updates(st):
    h = np.array(st.newton_hist)
    return float((np.arange(64) * h).sum() / h.sum())


@pytest.mark.parametrize("precision,tol", [(L.LELBM_FP64, STEP_TOL), (L.LELBM_FP32, FP32_TOL)])
def test_stored_start_1d_matches_oracle_and_saves_updates(precision, tol):
    w = W.riemann_1d(n=400, seed_index=0)
    p = int(w.pads[0])
    a = Solver.riemann1d(w, precision=precision)
    b = Solver.riemann1d(w, precision=precision)
    b.set_warmstart(True)
    for s in (a, b):
        s.step(2)
        L.lelbm_reset_stats(s.h)
        s.step(3)
    ref = oracle_1d_instance(w, 0, 5)
    assert_close(b.get_moments()[:, p:p + 400], ref[:, p:p + 400], 5 * tol, "stored start, 5 steps")
    ma, mb = mean_updates(a.stats()), mean_updates(b.stats())
    assert mb < ma - 0.3, (ma, mb)
    assert b.stats().fallback_mx == 0
    a.close()
    b.close()


def test_stored_start_1d_batch_persistent():
    """The persistent batch kernel with the store, after an autotune (whose trial
    steps must leave the store as they found it)."""
    w = W.riemann_1d_batch(n_batch=10, seed_index=406, lmin=20, lmax=120)
    s = Solver.riemann1d(w)
    s.set_warmstart(True)
    s.autotune(1)
    s.run_batch(4)
    M = s.get_moments()
    for b in range(w.n_batch):
        first, n = s.instance(b)
        ref = oracle_1d_instance(w, b, 4)
        pb = int(w.pads[b])
        assert_close(M[:, first:first + n], ref[:, pb:pb + n], 4 * STEP_TOL, f"stored start, instance {b}")
    s.close()


@pytest.mark.parametrize("precision,tol", [(L.LELBM_FP64, STEP_TOL), (L.LELBM_MIXED, 1e-11), (L.LELBM_FP32, FP32_TOL)])
def test_stored_start_2d(precision, tol):
    w = W.random_smooth_2d(18, 14, seed_index=23, RT_lo=0.25, RT_hi=1.4, umag=0.7)
    s = Solver.grid2d(w, precision=precision)
    s.set_warmstart(True)
    s.step(3)
    assert_close(s.get_moments(), oracle_2d(w, 3), 3 * tol, "stored start 2D")
    s.close()


def test_stored_start_toggles():
    """Turning the store off frees it and restores the plain start; a new store
    starts at zero, i.e. from Eq. (IID13)."""
    w = W.riemann_1d(n=200, seed_index=3)
    s = Solver.riemann1d(w)
    s.set_warmstart(True)
    s.step(2)
    s.set_warmstart(False)
    L.lelbm_reset_stats(s.h)
    s.step(1)
    plain = mean_updates(s.stats())
    s.set_warmstart(True)
    L.lelbm_reset_stats(s.h)
    s.step(1)
    assert abs(mean_updates(s.stats()) - plain) < 0.2
    s.close()
