"""The allocation-free step (lelbm_step_noalloc) against the handle-based step.

Some callers cannot allocate device memory: an application that owns all device memory
through its own pool or a fixed budget, or code on a latency-critical path where cudaFree
synchronises the device.  lelbm_step_noalloc serves them with caller-owned state buffers and
a static device scratch array.  This test calls it through the C ABI twice in a row, each
time on the previous output, and checks every moment against lelbm_step on the same input
within the per-step tolerance of the other parity tests (1e-12 of each moment's largest
magnitude).  It builds everything it needs, so it runs alone in a fresh process as well as
after the other tests.
"""
import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L, workloads as W
from paper_2508_06911_gb300.solver import Solver

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12


def rel_err(got, ref):
    sc = np.maximum(np.abs(ref).max(axis=1), 1e-300)
    return float((np.abs(got - ref).max(axis=1) / sc).max())


def params_like(dims, nx, ny, bc, pad, K, nu, Pr, inlet=(1.0, 0.0, 0.0, 1.0)):
    p = L.lelbm_default_params()
    p.dims, p.nx, p.ny, p.pad = dims, nx, ny, pad
    for i in range(4):
        p.bc[i] = bc[i]
        p.inlet[i] = inlet[i]
    p.K, p.nu_shear, p.prandtl = K, nu, Pr
    return p


def run_pair(solver, p, lengths=None, pads=None):
    import torch

    M0 = solver.get_moments()
    solver.step(1)
    M1 = solver.get_moments()
    solver.step(1)
    M2 = solver.get_moments()
    m_in = torch.from_numpy(M0).cuda()
    m_mid = torch.empty_like(m_in)
    m_out = torch.empty_like(m_in)
    torch.cuda.synchronize()
    st1, st2 = L.lelbm_stats(), L.lelbm_stats()
    assert L.lelbm_step_noalloc(p, m_in.data_ptr(), m_mid.data_ptr(), st1, lengths, pads) == L.LELBM_OK
    assert L.lelbm_step_noalloc(p, m_mid.data_ptr(), m_out.data_ptr(), st2, lengths, pads) == L.LELBM_OK
    torch.cuda.synchronize()
    e1 = rel_err(m_mid.cpu().numpy(), M1)
    e2 = rel_err(m_out.cpu().numpy(), M2)
    assert e1 <= STEP_TOL, e1
    assert e2 <= 2 * STEP_TOL, e2
    assert st1.cells == st2.cells > 0 and st1.fallback_mx == 0 and st2.fallback_mx == 0
    return st1


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def test_noalloc_1d_batch_two_calls():
    w = W.riemann_1d_batch(n_batch=20, seed_index=303, lmin=24, lmax=160)
    s = Solver.riemann1d(w)
    p = params_like(1, int(w.lengths[0]), 1, (0, 0, 2, 2), int(w.pads[0]), w.K, w.nu, w.Pr)
    st = run_pair(s, p, lengths=w.lengths, pads=w.pads)
    assert st.cells == s.n_cells
    s.close()


def test_noalloc_2d_outflow_inflow_two_calls():
    w = W.random_smooth_2d(18, 12, seed_index=9, RT_lo=0.4, RT_hi=1.4, umag=0.5, periodic=False)
    w.bc = (1, 0, 0, 0)
    w.inlet = (1.1, 0.7, 0.0, 0.9)
    s = Solver.grid2d(w)
    p = params_like(2, w.nx, w.ny, w.bc, w.pad, w.K, w.nu, w.Pr, w.inlet)
    run_pair(s, p)
    s.close()


def test_noalloc_1d_periodic_batch_two_calls():
    """Periodic 1D instances: populations leaving one end of an instance re-enter at the other."""
    lengths = np.array([24, 40, 31])
    n = int(lengths.sum())
    x = np.arange(n) / n
    rho = 1.0 + 0.2 * np.sin(6 * np.pi * x)
    u = 0.6 * np.cos(4 * np.pi * x)
    RT = 0.8 + 0.3 * np.sin(10 * np.pi * x)
    s = Solver(1, int(lengths[0]), 1, K=4.0, nu=1e-3, Pr=0.71, bc=(2, 2, 2, 2), pad=0, lengths=lengths)
    s.set_state(rho, u[None], RT)
    p = params_like(1, int(lengths[0]), 1, (2, 2, 2, 2), 0, 4.0, 1e-3, 0.71)
    run_pair(s, p, lengths=lengths)
    s.close()


@pytest.mark.parametrize("case", ["random", "hot"])
def test_noalloc_2d_periodic_two_calls(case):
    """Fully periodic 2D grids: a smooth random field, and the hot box (u = (10, 10), RT = 2)
    whose populations wrap around several cells."""
    w = (W.random_smooth_2d(14, 10, seed_index=19, RT_lo=0.4, RT_hi=1.5, umag=1.5) if case == "random"
         else W.hot_box(2, 10, 2.0))
    s = Solver.grid2d(w)
    p = params_like(2, w.nx, w.ny, (2, 2, 2, 2), 0, w.K, w.nu, w.Pr)
    run_pair(s, p)
    s.close()


def test_noalloc_2d_periodic_x_padded_y_two_calls():
    """x periodic (no pads, NX = nx), y with outflow pads."""
    w = W.random_smooth_2d(16, 12, seed_index=20, RT_lo=0.4, RT_hi=1.4, umag=0.8, periodic=False)
    w.bc = (2, 2, 0, 0)
    s = Solver.grid2d(w)
    p = params_like(2, w.nx, w.ny, w.bc, w.pad, w.K, w.nu, w.Pr, w.inlet)
    run_pair(s, p)
    s.close()


def test_noalloc_rejects_too_many_instances():
    import torch

    n = L.LELBM_NOALLOC_MAX_INSTANCES + 1
    p = params_like(1, 8, 1, (0, 0, 2, 2), 4, 4.0, 1e-3, 0.71)
    cells = n * (8 + 2 * 4)
    m_in = torch.zeros((6, cells), dtype=torch.float64, device="cuda")
    m_out = torch.zeros_like(m_in)
    rc = L.lelbm_step_noalloc(p, m_in.data_ptr(), m_out.data_ptr(), None, lengths=np.full(n, 8), pads=np.full(n, 4))
    assert rc == L.LELBM_E_INVAL
    assert float(m_out.abs().max()) == 0.0  # nothing was launched
