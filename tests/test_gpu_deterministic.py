"""Deterministic moment streaming (lelbm_params.deterministic, 2D FP64 path) through the C ABI.

Moment streaming (Eq. IIE3) as a gather: each target cell sums what the cells within reach
send it, in a fixed order, instead of the FP64 atomic scatter.
- Parity: within 1e-12 of the oracle per step, as the scatter path, on periodic random
  states, cold states with refined children landing between cells (Eq. IIC10-IIC11, cloud in
  cell), padded boxes with inflow and outflow sides (Sec. III.A), and the hot box of
  Sec. IV.E on a grid smaller than the reach of its velocity set (a source reaches a target
  through several periodic images).
- Reproducibility: two handles stepping the same state on two streams at once, and a third
  stepping alone, end with the same bits after many steps; the atomic scatter does not
  guarantee that.
"""
import numpy as np
import pytest
import torch

from paper_2508_06911_gb300 import build, lelbm as L, workloads as W
from paper_2508_06911_gb300.solver import Solver

import oracle as O
from parity_util import assert_close, interior_mask_2d, oracle_2d

pytestmark = pytest.mark.gpu
STEP_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    O.build()


def gpu_steps(w, nsteps, stream=None, **numerics):
    s = Solver.grid2d(w, stream=stream, deterministic=1, **numerics)
    out = []
    for _ in range(nsteps):
        s.step(1)
        out.append(s.get_moments())
    st = s.stats()
    status = s.synchronize()
    s.close()
    return out, st, status


CASES = {
    "periodic": lambda: W.random_smooth_2d(24, 20, 31, 0.6, 2.5, 0.8),
    "refined": lambda: W.random_smooth_2d(20, 18, 32, 0.06, 0.3, 0.3),
    "padded": lambda: W.random_smooth_2d(22, 16, 33, 0.4, 1.2, 0.5, periodic=False),
    "hot-box-images": lambda: W.hot_box(2, 8, 0.5),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_gather_matches_oracle(case):
    w = CASES[case]()
    if case == "padded":
        w.bc = (1, 0, 0, 1)  # inflow at x- and y+
        w.inlet = (1.1, 0.3, -0.2, 0.8)
    nsteps = 3
    got, st, status = gpu_steps(w, nsteps)
    m = interior_mask_2d(w)
    # raw moments at |u| >> sqrt(RT) (the hot box, |u| / sqrt(RT) = 20) carry rounding of
    # order eps (|u| / sqrt(RT))^3 relative on both sides
    tol = 1e-11 if case == "hot-box-images" else STEP_TOL
    for k in range(nsteps):
        ref = oracle_2d(w, k + 1)
        e = assert_close(got[k][:, m], ref[:, m], tol * (k + 1), f"deterministic {case}, step {k + 1}")
        print(f"deterministic gather, {case}, step {k + 1}: max rel {e:.2e}")
        assert np.all(got[k][:, ~m] == 0.0)
    assert status == L.LELBM_OK and st.fallback_mx == 0
    assert st.points_ms > 0


def test_gather_rejects_what_it_does_not_cover():
    w = W.random_smooth_2d(8, 8, 34, 0.5, 1.0, 0.3)
    with pytest.raises(L.LelbmError):
        Solver.grid2d(w, deterministic=1, precision=L.LELBM_MIXED)


def test_same_bits_on_concurrent_streams():
    w = W.random_smooth_2d(96, 80, 35, 0.2, 2.0, 0.8)
    nsteps = 25
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a = Solver.grid2d(w, stream=s1.cuda_stream, deterministic=1)
    b = Solver.grid2d(w, stream=s2.cuda_stream, deterministic=1)
    for _ in range(nsteps):  # the two handles' kernels overlap on the GPU
        a.step(1)
        b.step(1)
    Ma, Mb = a.get_moments(), b.get_moments()
    a.close()
    b.close()
    alone, _, _ = gpu_steps(w, nsteps)
    assert np.array_equal(Ma, Mb)
    assert np.array_equal(Ma, alone[-1])
    # and the same physics as the atomic scatter, to rounding
    c = Solver.grid2d(w)
    c.step(nsteps)
    Mc = c.get_moments()
    c.close()
    m = interior_mask_2d(w)
    e = assert_close(Ma[:, m], Mc[:, m], 1e-11, "gather vs scatter")
    print(f"gather vs atomic scatter after {nsteps} steps: max rel {e:.2e}; bits equal across runs")
