"""Full-length 2D runs through the C ABI.

- The FP64 path against the CPU oracle over 200 steps of configuration 12 of the 2D Riemann
  problem (Sec. V.D, Eq. VID1): within 1e-9 of each moment's largest magnitude after the
  run, the bound the FP64 path is held to.
- The mixed path (FP32 Newton, double-float correction and streaming judged at the FP64
  tolerance of Sec. II.D), from the learned warm start, against the FP64 path over the full
  2000 steps of the seeded four-quadrant problem at 1024^2 (the generator of the 4096^2
  benchmark workload): relative L1 density difference at most 1e-4.  The FP32 path's
  difference over the same run is printed beside it (it is not held to 1e-4 over thousands
  of 2D steps; see the FP32 path's description in include/lelbm.h).
"""
import os

import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L, workloads as W
from paper_2508_06911_gb300.solver import Solver

import oracle as O
from parity_util import assert_close, interior_mask_2d, max_rel_err, oracle_2d

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RUN_TOL = 1e-9
L1_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    O.build()


def l1_rel(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def test_fp64_2d_200_steps_match_oracle():
    w = W.lax_liu_12(n=48)
    nsteps = 200
    s = Solver.grid2d(w)
    s.step(nsteps)
    M = s.get_moments()
    st = s.stats()
    s.close()
    ref = oracle_2d(w, nsteps)
    m = interior_mask_2d(w)
    e = assert_close(M[:, m], ref[:, m], RUN_TOL, "FP64 Lax-Liu 12, 200 steps")
    print(f"FP64 vs oracle after {nsteps} steps: max rel {e:.2e}, L1 density {l1_rel(M[0, m], ref[0, m]):.2e}")
    assert st.fallback_mx == 0


def test_mixed_full_run_matches_fp64_riemann2d_1024():
    w = W.riemann_2d(n=1024, seed_index=2)
    nsteps = int(w.steps)
    assert nsteps == 2000
    weights = np.load(os.path.join(ROOT, "paper_2508_06911_gb300", "weights", "warmstart_2d_quadrants.npy"))
    m = interior_mask_2d(w)
    ref = Solver.grid2d(w)
    ref.step(nsteps)
    rho64 = ref.get_moments()[0, m]
    ref.close()
    mixed = Solver.grid2d(w, precision=L.LELBM_MIXED)
    L.lelbm_set_mlp(mixed.h, weights)
    mixed.step(nsteps)
    Mm = mixed.get_moments()
    st = mixed.stats()
    mixed.close()
    fp32 = Solver.grid2d(w, precision=L.LELBM_FP32)
    L.lelbm_set_mlp(fp32.h, weights)
    fp32.step(nsteps)
    rho32 = fp32.get_moments()[0, m]
    fp32.close()
    l1m, l1f = l1_rel(Mm[0, m], rho64), l1_rel(rho32, rho64)
    print(f"2000 steps at 1024^2: L1 density vs FP64 path: mixed {l1m:.2e}, FP32 {l1f:.2e}; "
          f"mixed judge misses {st.judge_redo}, FP64 fallbacks {st.points_f > 0}")
    assert np.all(np.isfinite(Mm))
    assert l1m <= L1_TOL
    assert st.fallback_mx == 0 and st.mlp_cells > 0
