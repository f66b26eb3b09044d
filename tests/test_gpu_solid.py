"""Solid boundary (Sec. III.B, stationary slip wall) on the GPU against the CPU oracle.

The GPU traces paths past solid faces only in cells whose populations can reach a
solid cell (a wall-distance field decides); elsewhere it streams as without solids.
Per step the FP64 path must match the oracle within 1e-12 of each moment's largest
magnitude, the count of reflected populations must be equal, and solid cells stay
empty.  The mixed path is held to its own 1e-11 per step.
"""
import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L, workloads as W
from paper_2508_06911_gb300.solver import Solver

import oracle as O
from parity_util import assert_close, interior_mask_2d, oracle_2d

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-12
MIXED_TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    O.build()


def obstacle_field(nx, ny, seed_index, RT_lo, RT_hi, umag, frac):
    w = W.random_smooth_2d(nx, ny, seed_index, RT_lo, RT_hi, umag, periodic=True)
    g = np.random.default_rng(1000 + seed_index)
    solid = np.zeros((ny, nx), np.uint8)
    # a frame of walls, a few rectangles and scattered single cells (corners of every kind)
    solid[0, :] = solid[-1, :] = 1
    solid[:, 0] = 1
    for _ in range(3):
        x0, y0 = g.integers(2, nx - 5), g.integers(2, ny - 5)
        solid[y0:y0 + g.integers(1, 4), x0:x0 + g.integers(1, 4)] = 1
    solid |= (g.random((ny, nx)) < frac).astype(np.uint8)
    w.solid = solid
    return w


def run_both(w, nsteps, **numerics):
    st_o = O.Stats()
    ref = oracle_2d(w, nsteps, st_o)
    s = Solver.grid2d(w, **numerics)
    s.step(nsteps)
    M = s.get_moments()
    st = s.stats()
    s.close()
    return M, ref, st, st_o


@pytest.mark.parametrize("RT_lo,RT_hi,frac", [(0.08, 0.14, 0.04), (0.6, 2.5, 0.03), (0.25, 0.6, 0.06)])
def test_fp64_step_with_obstacles(RT_lo, RT_hi, frac):
    """Walls, blocks and single solid cells in a periodic box: one step, then three."""
    w = obstacle_field(30, 22, 7, RT_lo, RT_hi, 0.4, frac)
    mask = interior_mask_2d(w)
    for n in (1, 3):
        M, ref, st, st_o = run_both(w, n)
        assert_close(M[:, mask], ref[:, mask], STEP_TOL * n, f"solids, {n} steps")
        assert st.wall_hits == st_o.wall_hits > 0
        assert np.all(M[:, ~mask] == 0.0)
        assert st.fallback_mx == 0


def test_mixed_step_with_obstacles():
    w = obstacle_field(30, 22, 8, 0.2, 1.5, 0.4, 0.04)
    mask = interior_mask_2d(w)
    M, ref, st, st_o = run_both(w, 2, precision=L.LELBM_MIXED)
    assert_close(M[:, mask], ref[:, mask], 2 * MIXED_TOL, "mixed, solids")
    assert st.wall_hits == st_o.wall_hits > 0


def test_supersonic_cylinder_small():
    """A Mach-3 cylinder with inflow, outflow pads and an impulsive start (the shape of
    the paper's Sec. V.G case at a few hundredths of its size)."""
    w = W.cylinder_2d(nx=72, ny=48, diameter=14, steps=4)
    mask = interior_mask_2d(w)
    M, ref, st, st_o = run_both(w, 4)
    assert_close(M[:, mask], ref[:, mask], 4 * STEP_TOL, "cylinder, 4 steps")
    assert st.wall_hits == st_o.wall_hits > 0
    rho = M[0, mask]
    assert rho.min() > 0


def test_closed_box_conservation_on_gpu():
    """A sealed box: mass and energy are conserved to rounding over many steps."""
    w = obstacle_field(40, 32, 9, 0.3, 1.2, 0.3, 0.0)
    w.solid[:, -1] = 1
    s = Solver.grid2d(w)
    M0 = s.get_moments()
    t0 = M0.sum(1)
    s.step(50)
    t1 = s.get_moments().sum(1)
    s.close()
    assert abs(t1[0] / t0[0] - 1) < 1e-12
    E0, E1 = t0[3] + t0[5] + t0[8], t1[3] + t1[5] + t1[8]
    assert abs(E1 / E0 - 1) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_wall_through_outflow_pads(prec):
    """A slip wall along the bottom that runs out through the outflow side (the oblique-shock
    geometry of Sec. V.F): the outflow pads behind the wall are solid.  A short oblique stream
    hits the wall; parity with the oracle after three steps, and no failed cell."""
    w = W.oblique_2d(2.0, 5.0, nx=48, ny=30)
    mask = interior_mask_2d(w)
    M, ref, st, st_o = run_both(w, 3, precision=L.LELBM_FP64 if prec == "fp64" else L.LELBM_MIXED)
    tol = 3 * (STEP_TOL if prec == "fp64" else MIXED_TOL)
    assert_close(M[:, mask], ref[:, mask], tol, f"wall through outflow pads ({prec})")
    assert st.wall_hits == st_o.wall_hits > 0
    assert st.fallback_mx == 0 and st_o.fallback_mx == 0


def noslip_field(nx, ny, seed_index, RT_lo, RT_hi, umag):
    """Slip and no-slip walls together: a no-slip frame, slip blocks and single cells."""
    w = obstacle_field(nx, ny, seed_index, RT_lo, RT_hi, umag, 0.02)
    w.solid = w.solid.copy()
    frame = np.zeros_like(w.solid)
    frame[0, :] = frame[-1, :] = frame[:, 0] = 1
    w.solid[frame == 1] = 2  # the frame is no-slip, the rest stays slip
    return w


@pytest.mark.parametrize("RT_lo,RT_hi", [(0.6, 2.0), (0.1, 0.35)])
def test_noslip_walls_match_oracle(RT_lo, RT_hi):
    """Stationary no-slip walls (Sec. III.B, Eq. IIIB8-IIIB15 with u_w = 0) beside slip
    blocks: one and three steps against the oracle, and mass conserved in the closed box."""
    w = noslip_field(30, 22, 11, RT_lo, RT_hi, 0.4)
    mask = interior_mask_2d(w)
    for n in (1, 3):
        M, ref, st, st_o = run_both(w, n)
        assert_close(M[:, mask], ref[:, mask], STEP_TOL * n, f"no-slip walls, {n} steps")
        assert st.wall_hits == st_o.wall_hits > 0
        assert st.fallback_mx == 0
    s = Solver.grid2d(w)
    m0 = s.get_moments()[0, mask].sum()
    s.step(20)
    m1 = s.get_moments()[0, mask].sum()
    s.close()
    assert abs(m1 / m0 - 1) < 1e-12


def test_noslip_channel_shear_mode_on_gpu():
    """The lowest shear mode between two no-slip walls, H = 32: the GPU's decay matches the
    oracle's step by step and the viscous rate nu (pi / H)^2 within 10 %."""
    H, nx, nu, RT, amp = 32, 4, 0.05, 0.5, 1e-3
    ny = H + 2
    solid = np.zeros((ny, nx), np.uint8)
    solid[0] = solid[-1] = 2
    yc = np.arange(ny) + 0.5
    mode = np.sin(np.pi * (yc - 1.0) / H)
    mode[0] = mode[-1] = 0.0
    u = np.zeros((2, ny, nx))
    u[0] = amp * mode[:, None]
    w = W.Grid2D(nx=nx, ny=ny, rho=np.ones((ny, nx)), u=u, RT=np.full((ny, nx), RT), bc=(2, 2, 2, 2), pad=0,
                 K=3.0, nu=nu, Pr=1.0, steps=400, solid=solid)
    s = Solver.grid2d(w, limiter=0)
    fl = (solid == 0).reshape(-1)
    a = []
    for _ in range(400):
        s.step(1)
        M = s.get_moments()
        ux = np.zeros(ny * nx)
        ux[fl] = M[1, fl] / M[0, fl]
        a.append((ux.reshape(ny, nx).mean(1) * mode).sum() / (mode * mode).sum())
    s.close()
    t = np.arange(1, 401)
    rate = -np.polyfit(t[66:], np.log(np.array(a)[66:]), 1)[0]
    ratio = rate / (nu * (np.pi / H) ** 2)
    print(f"no-slip channel H = {H}: decay rate / nu (pi/H)^2 = {ratio:.4f}")
    assert abs(ratio - 1) < 0.10
    ref = oracle_2d(w, 3, limiter=0)
    s = Solver.grid2d(w, limiter=0)
    s.step(3)
    got = s.get_moments()
    s.close()
    # the transverse moments vanish by symmetry (rounding noise on both sides), so the
    # bound is relative to the largest moment of the state
    err = np.abs(got[:, fl] - ref[:, fl]).max() / np.abs(ref[:, fl]).max()
    assert err <= 3 * STEP_TOL, f"no-slip channel, 3 steps: {err:.2e}"


def test_noslip_walls_need_the_fp64_path():
    w = noslip_field(16, 12, 12, 0.5, 1.0, 0.2)
    with pytest.raises(L.LelbmError):
        Solver.grid2d(w, precision=L.LELBM_MIXED)


def run_walls(w, nsteps, wall_u, **numerics):
    """GPU and oracle after nsteps on a grid whose solid bytes include moving walls (3)."""
    st_o = O.Stats()
    g = O.grid(2, w.nx, w.ny, periodic=(w.bc[0] == 2, w.bc[2] == 2), pad=0 if w.bc[0] == 2 and w.bc[2] == 2 else w.pad,
               bc=tuple(1 if b == 1 else 0 for b in w.bc), inlet=w.inlet, solid=w.padded()[3], wall_u=wall_u)
    p = O.params(2, w.K, nu_s=w.nu, Pr=w.Pr, limiter=numerics.get("limiter", 1))
    ref = O.run(g, p, O.state_from_primitives(g, p, w.rho, w.u, w.RT), nsteps, st_o)
    s = Solver.grid2d(w, wall_u=wall_u, **numerics)
    s.step(nsteps)
    M = s.get_moments()
    st = s.stats()
    s.close()
    return M, ref, st, st_o


@pytest.mark.parametrize("RT_lo,RT_hi", [(0.6, 2.0), (0.15, 0.4)])
def test_moving_lid_box_matches_oracle(RT_lo, RT_hi):
    """A box with a lid moving at u_w (solid byte 3; Eq. IIIB2-IIIB4, IIIB10-IIIB15: the image
    populations are the EPR of the cell's constraints at u - 2 u_w) and no-slip walls at rest
    elsewhere: one and three steps against the oracle, mass conserved."""
    w = obstacle_field(30, 22, 13, RT_lo, RT_hi, 0.3, 0.0)
    w.solid = np.zeros_like(w.solid)
    w.solid[0, :] = w.solid[:, 0] = w.solid[:, -1] = 2
    w.solid[-1, :] = 3
    mask = interior_mask_2d(w)
    for n in (1, 3):
        M, ref, st, st_o = run_walls(w, n, (0.4, 0.0))
        assert_close(M[:, mask], ref[:, mask], STEP_TOL * n, f"moving lid, {n} steps")
        assert st.wall_hits == st_o.wall_hits > 0 and st.fallback_mx == 0
        assert abs(M[0, mask].sum() / ref[0, mask].sum() - 1) < 1e-13


def test_couette_profile_on_gpu():
    """Plane Couette flow between a wall at rest and one moving at U: linear steady profile,
    0 and U at the two wall faces within a fifth of a cell (the oracle's pin, on the GPU)."""
    U, H, nx = 0.05, 16, 4
    ny = H + 2
    solid = np.zeros((ny, nx), np.uint8)
    solid[0], solid[-1] = 2, 3
    w = W.Grid2D(nx=nx, ny=ny, rho=np.ones((ny, nx)), u=np.zeros((2, ny, nx)), RT=np.full((ny, nx), 0.5),
                 bc=(2, 2, 2, 2), pad=0, K=3.0, nu=0.2, Pr=0.71, steps=1500, solid=solid)
    s = Solver.grid2d(w, wall_u=(U, 0.0), limiter=0)
    s.step(1500)
    M = s.get_moments()
    s.close()
    fl = (solid == 0).reshape(-1)
    ux = (M[1, fl] / M[0, fl]).reshape(H, nx).mean(1)
    y = np.arange(1, H + 1) + 0.5
    a, b = np.polyfit(y, ux, 1)
    print(f"Couette: u = 0 at y = {-b / a:.3f} (face 1), u = U at y = {(U - b) / a:.3f} (face {H + 1})")
    assert abs(-b / a - 1.0) < 0.2 and abs((U - b) / a - (H + 1.0)) < 0.2
    assert np.abs(ux - (a * y + b)).max() < 1e-3 * U
