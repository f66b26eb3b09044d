"""Mixed-precision path (LELBM_MIXED) against the CPU oracle and the FP64 path.

The mixed path iterates the EPR Newton in FP32, corrects with one FP64 Newton pass and
accepts the multipliers only when the FP64 residual of the streamed populations is within
the same 1e-12 tolerance (thermal units) as the FP64 path; it does not apply the FP64
path's polishing update.  Per step it must therefore match the oracle within 1e-11 of each
moment's largest magnitude, and a full run within 1e-8 (L1 density error reported too).
"""
import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L, workloads as W
from paper_2508_06911_gb300.solver import Solver

import oracle as O
from parity_util import assert_close, interior_mask_2d, oracle_1d_instance, oracle_2d

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-11
RUN_TOL = 1e-8
MIXED = dict(precision=L.LELBM_MIXED)


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    O.build()


def test_mixed_1d_step_and_run():
    w = W.riemann_1d(n=400, seed_index=0)
    p = int(w.pads[0])
    s = Solver.riemann1d(w, **MIXED)
    s.step(1)
    M1 = s.get_moments()
    assert_close(M1[:, p:p + 400], oracle_1d_instance(w, 0, 1)[:, p:p + 400], STEP_TOL, "mixed 1D step")
    s.step(int(w.steps[0]) - 1)
    M = s.get_moments()
    st = s.stats()
    ref = oracle_1d_instance(w, 0, int(w.steps[0]))
    assert_close(M[:, p:p + 400], ref[:, p:p + 400], RUN_TOL, "mixed, 400-cell 1D Riemann problem, full run")
    l1 = np.abs(M[0, p:p + 400] - ref[0, p:p + 400]).sum() / np.abs(ref[0, p:p + 400]).sum()
    assert l1 < 1e-9, l1
    assert st.fallback_mx == 0 and st.points_32 > 0
    s.close()


def test_mixed_1d_batch():
    w = W.riemann_1d_batch(n_batch=10, seed_index=404, lmin=20, lmax=120)
    s = Solver.riemann1d(w, **MIXED)
    s.step(2)
    M = s.get_moments()
    for b in range(w.n_batch):
        first, n = s.instance(b)
        ref = oracle_1d_instance(w, b, 2)
        pb = int(w.pads[b])
        assert_close(M[:, first:first + n], ref[:, pb:pb + n], 2 * STEP_TOL, f"mixed instance {b}")
    s.close()


def test_mixed_2d_periodic_with_refinement():
    w = W.random_smooth_2d(18, 12, seed_index=17, RT_lo=0.25, RT_hi=1.3, umag=0.8)
    s = Solver.grid2d(w, **MIXED)
    s.step(2)
    assert_close(s.get_moments(), oracle_2d(w, 2), 2 * STEP_TOL, "mixed 2D periodic")
    s.close()


def test_mixed_2d_outflow_inflow():
    w = W.random_smooth_2d(14, 12, seed_index=18, RT_lo=0.5, RT_hi=2.5, umag=0.6, periodic=False)
    w.bc = (1, 0, 0, 0)
    w.inlet = (1.2, 0.9, 0.1, 0.8)
    s = Solver.grid2d(w, **MIXED)
    s.step(2)
    m = interior_mask_2d(w)
    assert_close(s.get_moments()[:, m], oracle_2d(w, 2)[:, m], 2 * STEP_TOL, "mixed 2D outflow/inflow")
    s.close()


def test_mixed_matches_fp64_path_on_2d_riemann():
    w = W.lax_liu_12(n=48)
    a = Solver.grid2d(w)
    b = Solver.grid2d(w, **MIXED)
    a.step(4)
    b.step(4)
    m = interior_mask_2d(w)
    assert_close(b.get_moments()[:, m], a.get_moments()[:, m], 4 * STEP_TOL, "mixed vs FP64, Lax-Liu 12")
    a.close()
    b.close()
