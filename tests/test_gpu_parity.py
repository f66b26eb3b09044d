"""GPU (liblelbm, FP64 path) against the CPU oracle, through the C ABI.

Tolerances: the FP64 path must match the oracle within 1e-12 relative per step and
1e-9 after a full run (relative to each moment's largest magnitude over the grid).
"""
import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L, workloads as W
from paper_2508_06911_gb300.solver import Solver

import oracle as O
from parity_util import assert_close, interior_mask_2d, oracle_1d_instance, oracle_2d

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12
RUN_TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    O.build()


def gpu_1d(w, nsteps, periodic=False):
    bc = (2, 2, 2, 2) if periodic else (0, 0, 2, 2)
    s = Solver(1, int(w.lengths[0]), 1, K=w.K, nu=w.nu, Pr=w.Pr, bc=bc,
               pad=0 if periodic else int(w.pads[0]),
               lengths=w.lengths if w.n_batch > 1 else None,
               pads=None if (periodic or w.n_batch == 1) else w.pads)
    if periodic:
        rho, u, RT = (np.concatenate(x) for x in zip(*[w.primitives(b) for b in range(w.n_batch)]))
        s.set_state(rho, u[None, :], RT)
    else:
        s.set_state(*w.padded_fields())
    s.step(nsteps)
    M = s.get_moments()
    st = s.stats()
    return s, M, st


def test_1d_single_step():
    w = W.riemann_1d(n=150, seed_index=0)
    s, M, st = gpu_1d(w, 1)
    ref = oracle_1d_instance(w, 0, 1)
    p = int(w.pads[0])
    assert_close(M[:, p:p + 150], ref[:, p:p + 150], STEP_TOL, "1D Riemann, one step")
    assert st.fallback_mx == 0 and st.cells == 150 + 2 * p
    s.close()


def test_1d_periodic_random_steps():
    g = np.random.default_rng(5)
    n = 96
    x = np.arange(n) / n
    rho = 1 + 0.3 * np.sin(2 * np.pi * x) ** 2
    u = 0.8 * np.cos(2 * np.pi * x + 0.3)
    RT = 0.3 + 1.5 * g.random(n)
    w = W.Riemann1D(lengths=np.array([n]), left=np.zeros((1, 3)), right=np.zeros((1, 3)), scale=np.ones(1),
                    steps=np.ones(1, int), pads=np.zeros(1, int), t_end=0.0)
    w.primitives = lambda b: (rho, u, RT)
    for nsteps in (1, 3):
        s, M, _ = gpu_1d(w, nsteps, periodic=True)
        gg = O.grid(1, n, periodic=(True, False))
        p = O.params(1, w.K, nu_s=w.nu, Pr=w.Pr)
        ref = O.run(gg, p, O.state_from_primitives(gg, p, rho, u[None], RT), nsteps)
        assert_close(M, ref, STEP_TOL * nsteps, f"1D periodic, {nsteps} steps")
        s.close()


def test_1d_full_run_400_cells():
    """The 400-cell seeded Riemann problem to t = 0.2 (80 steps): <= 1e-9 after the run."""
    w = W.riemann_1d(n=400, seed_index=0)
    nsteps = int(w.steps[0])
    s, M, st = gpu_1d(w, nsteps)
    ref = oracle_1d_instance(w, 0, nsteps)
    p = int(w.pads[0])
    assert_close(M[:, p:p + 400], ref[:, p:p + 400], RUN_TOL, "400-cell 1D Riemann problem, full run")
    assert st.fallback_mx == 0
    s.close()


def test_1d_batch_ragged():
    """A ragged batch of independent instances (per-instance pads and acoustic scaling)."""
    w = W.riemann_1d_batch(n_batch=12, seed_index=101, lmin=16, lmax=90)
    s, M, st = gpu_1d(w, 2)
    for b in range(w.n_batch):
        first, n = s.instance(b)
        assert n == w.lengths[b]
        ref = oracle_1d_instance(w, b, 2)
        p = int(w.pads[b])
        assert_close(M[:, first:first + n], ref[:, p:p + n], STEP_TOL * 2, f"instance {b}")
    assert st.fallback_mx == 0
    s.close()


def test_2d_periodic_with_refinement():
    w = W.random_smooth_2d(20, 14, seed_index=7, RT_lo=0.25, RT_hi=1.2, umag=0.8)
    s = Solver.grid2d(w)
    s.step(2)
    M = s.get_moments()
    ref = oracle_2d(w, 2)
    assert_close(M, ref, 2 * STEP_TOL, "2D periodic, 2 steps")
    st = s.stats()
    assert st.fallback_mx == 0
    s.close()


def test_2d_outflow_and_inflow():
    w = W.random_smooth_2d(16, 12, seed_index=8, RT_lo=0.5, RT_hi=1.5, umag=0.6, periodic=False)
    w.bc = (1, 0, 0, 0)
    w.inlet = (1.2, 0.9, 0.1, 0.8)
    s = Solver.grid2d(w)
    s.step(2)
    M = s.get_moments()
    ref = oracle_2d(w, 2)
    m = interior_mask_2d(w)
    assert_close(M[:, m], ref[:, m], 2 * STEP_TOL, "2D outflow/inflow, 2 steps")
    s.close()


@pytest.mark.parametrize("RT", [0.5, 2.0])
def test_2d_hot_box(RT):
    w = W.hot_box(2, 12, RT)
    s = Solver.grid2d(w)
    s.step(2)
    M = s.get_moments()
    ref = oracle_2d(w, 2)
    assert_close(M, ref, 2 * STEP_TOL, f"hot box RT={RT}")
    s.close()


def test_lax_liu_config12_small():
    w = W.lax_liu_12(n=40)
    s = Solver.grid2d(w)
    s.step(3)
    M = s.get_moments()
    ref = oracle_2d(w, 3)
    m = interior_mask_2d(w)
    assert_close(M[:, m], ref[:, m], 3 * STEP_TOL, "Lax-Liu 12, 3 steps")
    s.close()


def test_zero_steps_and_roundtrip():
    w = W.riemann_1d(n=64, seed_index=3)
    s = Solver.riemann1d(w)
    M0 = s.get_moments()
    s.step(0)
    np.testing.assert_array_equal(s.get_moments(), M0)
    s.set_moments(M0 * 1.0)
    np.testing.assert_array_equal(s.get_moments(), M0)
    rho, u, RT = s.macros()
    r_ref, u_ref, T_ref = w.primitives(0)
    p = int(w.pads[0])
    np.testing.assert_allclose(rho[p:p + 64], r_ref, rtol=1e-14)
    np.testing.assert_allclose(RT[p:p + 64], T_ref, rtol=1e-12)
    s.close()


def test_invalid_arguments_are_rejected():
    p = L.lelbm_default_params()
    p.dims = 4
    with pytest.raises(L.LelbmError) as e:
        L.lelbm_create(p)
    assert e.value.code == L.LELBM_E_INVAL
    p = L.lelbm_default_params()
    p.bc[0] = L.LELBM_BC_OUTFLOW  # periodic on one side only
    with pytest.raises(L.LelbmError):
        L.lelbm_create(p)
    w = W.riemann_1d(n=32)
    s = Solver.riemann1d(w)
    rho, u, RT = w.padded_fields()
    RT = RT.copy()
    RT[int(w.pads[0]) + 3] = -1.0
    with pytest.raises(L.LelbmError) as e:
        s.set_state(rho, u, RT)
    assert e.value.code == L.LELBM_E_STATE
    with pytest.raises(L.LelbmError):
        s.step(-1)
    s.close()
