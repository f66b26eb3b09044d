"""Pins of the oracle's solid boundary (Sec. III.B, extended bounce-back for a
stationary adiabatic slip wall).

The pins do not retype the oracle:
  * the path tracer is checked against an event-driven simulation of the
    reflected path in exact rational arithmetic, and against the closed-form
    fold of a path between two parallel walls;
  * a full step next to flat walls is checked against the method of images it
    stands for: a periodic domain holding the mirrored state, where no wall
    exists, must give the same moments in the real half;
  * conservation of mass and energy in a closed box with an obstacle, and the
    mirror symmetry of a symmetric flow around a symmetric obstacle.
"""
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(3111)


def _sign(v):
    return (v > 0) - (v < 0)


def trace_events(solid, periodic, ix, iy, c):
    """Reflected path from the centre of cell (ix, iy), advanced face event by
    face event in continuous time with exact rationals (positions, not the
    unfolded integer counters of the oracle).  A path through a cell corner
    into a solid diagonal cell reflects only the normal of a flat wall when
    exactly one side cell is solid, and both components otherwise."""
    NY, NX = solid.shape

    def is_solid(i, j):
        if periodic[0]:
            i %= NX
        if periodic[1]:
            j %= NY
        return 0 <= i < NX and 0 <= j < NY and bool(solid[j, i])

    x, y = Fr(ix), Fr(iy)
    vx, vy = Fr(float(c[0])), Fr(float(c[1]))
    i, j, t, touched = ix, iy, Fr(0), False
    half = Fr(1, 2)
    while True:
        tx = ((i + half * _sign(vx)) - x) / vx if vx != 0 else None
        ty = ((j + half * _sign(vy)) - y) / vy if vy != 0 else None
        cands = [v for v in (tx, ty) if v is not None]
        if not cands:
            break
        tn = min(cands)
        if t + tn >= 1:
            break
        x += vx * tn
        y += vy * tn
        t += tn
        cx, cy = tx == tn, ty == tn
        di, dj = (_sign(vx) if cx else 0), (_sign(vy) if cy else 0)
        if not is_solid(i + di, j + dj):
            i, j = i + di, j + dj
            continue
        touched = True
        if cx and cy:
            # corner: a flat wall (one side cell solid) reflects its normal only
            side_x, side_y = is_solid(i + di, j), is_solid(i, j + dj)
            if side_x != side_y:
                if side_x:
                    vx, j = -vx, j + dj
                else:
                    vy, i = -vy, i + di
                continue
        if cx:
            vx = -vx
        if cy:
            vy = -vy
    x += vx * (1 - t)
    y += vy * (1 - t)
    return touched, (i, j), (float(x - i), float(y - j)), (float(vx), float(vy))


def random_mask(NY, NX, frac):
    return (RNG.random((NY, NX)) < frac).astype(np.uint8)


@pytest.mark.parametrize("periodic", [(True, True), (False, False)])
def test_trace_matches_event_simulation(periodic):
    """Final cell, offset and reflected velocity agree with the rational event
    simulation on random solid masks, velocities on the 1/32 lattice of refined
    points and integer diagonals that pass exactly through cell corners."""
    NY, NX = 11, 13
    n = 0
    for trial in range(12):
        solid = random_mask(NY, NX, 0.25)
        g = O.grid(2, NX, NY, periodic=periodic, pad=0, solid=solid)
        fluid = np.argwhere(solid == 0)
        for _ in range(40):
            jy, ix = fluid[RNG.integers(len(fluid))]
            if trial % 3 == 0:   # exact diagonals / corner passes
                k = int(RNG.integers(1, 5))
                c = np.array([k * RNG.choice([-1, 1]), k * RNG.choice([-1, 1])], float)
            else:
                c = RNG.integers(-7 * 32, 7 * 32 + 1, size=2) / 32.0
            got = O.trace_path(g, int(ix), int(jy), c)
            ref = trace_events(solid, periodic, int(ix), int(jy), c)
            if not periodic[0]:
                # a path leaving a non-periodic array ends outside it in both
                fi, fj = ref[1]
                if not (0 <= fi < NX and 0 <= fj < NY):
                    continue
            assert got[0] == ref[0]
            assert got[1] == ref[1], (ix, jy, c)
            assert np.array_equal(got[2], np.array(ref[2])), (ix, jy, c)
            assert np.array_equal(got[3], np.array(ref[3])), (ix, jy, c)
            n += 1
    assert n > 200


def test_trace_channel_fold_closed_form():
    """Between two flat walls a specular path is the unfolded straight path
    folded into the channel: with the fluid cells 0..W-1 and the walls at -1/2
    and W-1/2, s = x + c + 1/2 taken modulo 2W lands at s or 2W - s."""
    W = 5
    solid = np.zeros((1, W + 1), np.uint8)
    solid[0, W] = 1
    g = O.grid(1, W + 1, 1, periodic=(True, False), pad=0, solid=solid)
    for ix in range(W):
        for c32 in range(-24 * 32, 24 * 32 + 1, 3):
            c = c32 / 32.0
            s = (ix + c + 0.5) % (2 * W)
            if s in (0.0, float(W)):
                continue  # ends on a wall face: the velocity sign is a convention
            pos = s - 0.5 if s < W else 2 * W - s - 0.5
            unfolded_up = s < W
            sgn = np.sign(c) if unfolded_up else -np.sign(c)
            touched, (fi, fj), off, cs = O.trace_path(g, ix, 0, [c])
            assert fj == 0 and 0 <= fi < W
            assert fi + off[0] == pos, (ix, c)
            if c != 0:
                assert cs[0] == sgn * abs(c), (ix, c)
            bounced = not (0 <= ix + c + 0.5 < W)
            assert touched == bounced, (ix, c)


def mirrored_state(p, rho, u, RT, mirror_x, mirror_y):
    """Equilibrium primitives (rho, u[2], RT) of shape (H, W) extended by their
    mirror images: across the right edge (mirror_x) and the top edge (mirror_y);
    the velocity component normal to each mirror changes sign."""
    if mirror_x:
        rho = np.concatenate([rho, rho[:, ::-1]], 1)
        RT = np.concatenate([RT, RT[:, ::-1]], 1)
        u = np.concatenate([u, u[:, :, ::-1] * np.array([-1.0, 1.0])[:, None, None]], 2)
    if mirror_y:
        rho = np.concatenate([rho, rho[::-1]], 0)
        RT = np.concatenate([RT, RT[::-1]], 0)
        u = np.concatenate([u, u[:, ::-1] * np.array([1.0, -1.0])[:, None, None]], 1)
    return rho, u, RT


@pytest.mark.parametrize("RTlo,RThi,W,H,box", [(0.8, 2.0, 7, 3, False), (0.08, 0.12, 6, 2, False),
                                               (0.8, 2.0, 3, 4, True), (0.08, 0.12, 3, 3, True)])
def test_flat_walls_equal_method_of_images(RTlo, RThi, W, H, box):
    """Slip walls on the faces of a channel (box: also on the x faces) give the
    moments of a wall-free periodic domain that holds the mirrored state.  The
    hot cases reflect several times per step; the cold ones stream refined
    points whose cloud-in-cell shares straddle the wall."""
    K = 2.0
    p = O.params(2, K, nu_s=5e-3, Pr=0.71)
    rho = 1 + 0.3 * RNG.random((H, W))
    RT = RTlo + (RThi - RTlo) * RNG.random((H, W))
    u = 0.35 * RNG.standard_normal((2, H, W))
    # walled domain: one solid row on top (and one solid column on the right)
    NXw, NYw = W + (1 if box else 0), H + 1
    solid = np.zeros((NYw, NXw), np.uint8)
    solid[H, :] = 1
    if box:
        solid[:, W] = 1
    gw = O.grid(2, NXw, NYw, periodic=(True, True), pad=0, solid=solid)
    rw, uw, Tw = (np.ones((NYw, NXw)), np.zeros((2, NYw, NXw)), np.ones((NYw, NXw)))
    rw[:H, :W], uw[:, :H, :W], Tw[:H, :W] = rho, u, RT
    Mw = O.state_from_primitives(gw, p, rw, uw, Tw)
    Mw[:, solid.reshape(-1) == 1] = 0.0
    # image domain: periodic, no solid cells
    ri, ui, Ti = mirrored_state(p, rho, u, RT, box, True)
    gi = O.grid(2, ri.shape[1], ri.shape[0], periodic=(True, True), pad=0)
    Mi = O.state_from_primitives(gi, p, ri, ui, Ti)
    st = O.Stats()
    for _ in range(3):
        Mw = O.step(gw, p, Mw, st)
        Mi = O.step(gi, p, Mi, None)
    assert st.wall_hits > 0
    a = Mw.reshape(-1, NYw, NXw)[:, :H, :W]
    b = Mi.reshape(-1, ri.shape[0], ri.shape[1])[:, :H, :W]
    scale = np.abs(b).max(axis=(1, 2), keepdims=True)
    err = (np.abs(a - b) / scale).max()
    assert err < 1e-12, err


def test_one_d_walls_equal_method_of_images():
    """The same check in 1D: a periodic row closed by one solid cell against the
    doubled, mirrored row."""
    K, W = 4.0, 9
    p = O.params(1, K, nu_s=5e-3, Pr=0.71)
    rho = 1 + 0.3 * RNG.random(W)
    RT = 0.3 + 2.5 * RNG.random(W)
    u = 0.5 * RNG.standard_normal(W)
    solid = np.zeros((1, W + 1), np.uint8)
    solid[0, W] = 1
    gw = O.grid(1, W + 1, 1, periodic=(True, False), solid=solid)
    Mw = O.state_from_primitives(gw, p, np.r_[rho, 1.0], np.r_[u, 0.0][None], np.r_[RT, 1.0])
    Mw[:, W] = 0.0
    gi = O.grid(1, 2 * W, 1, periodic=(True, False))
    Mi = O.state_from_primitives(gi, p, np.r_[rho, rho[::-1]], np.r_[u, -u[::-1]][None], np.r_[RT, RT[::-1]])
    for _ in range(4):
        Mw = O.step(gw, p, Mw)
        Mi = O.step(gi, p, Mi)
    scale = np.abs(Mi).max(1, keepdims=True)
    assert (np.abs(Mw[:, :W] - Mi[:, :W]) / scale).max() < 1e-12


def box_with_block(NX, NY):
    solid = np.zeros((NY, NX), np.uint8)
    solid[0, :] = solid[-1, :] = 1
    solid[:, 0] = solid[:, -1] = 1
    cx, cy = NX // 2, NY // 2
    solid[cy - 1:cy + 1, cx - 1:cx + 1] = 1
    return solid


@pytest.mark.parametrize("RTlo,RThi", [(0.08, 0.12), (0.6, 1.8)])
def test_closed_box_conserves_mass_and_energy(RTlo, RThi):
    """A gas enclosed by slip walls, around an obstacle with convex corners,
    keeps its mass and total energy to rounding; momentum is exchanged with the
    walls."""
    K = 3.0
    NX, NY = 12, 10
    solid = box_with_block(NX, NY)
    g = O.grid(2, NX, NY, periodic=(True, True), solid=solid)
    p = O.params(2, K, nu_s=5e-3, Pr=0.71)
    rho = 1 + 0.3 * RNG.random((NY, NX))
    RT = RTlo + (RThi - RTlo) * RNG.random((NY, NX))
    u = 0.4 * RNG.standard_normal((2, NY, NX))
    M = O.state_from_primitives(g, p, rho, u, RT)
    M[:, solid.reshape(-1) == 1] = 0.0
    st = O.Stats()
    for _ in range(3):
        t0 = M.sum(1)
        M = O.step(g, p, M, st)
        t1 = M.sum(1)
        assert abs(t1[0] / t0[0] - 1) < 1e-13
        E0, E1 = t0[3] + t0[5] + t0[8], t1[3] + t1[5] + t1[8]
        assert abs(E1 / E0 - 1) < 1e-13
        assert np.all(M[:, solid.reshape(-1) == 1] == 0.0)
    assert st.wall_hits > 0 and st.fallback_mx == 0
    assert M[0][solid.reshape(-1) == 0].min() > 0


def test_symmetric_flow_around_block_stays_symmetric():
    """A state mirror-symmetric about the vertical centre line of a centred
    obstacle stays mirror-symmetric (u_x odd, everything else even): a sign or
    index slip on one side of the tracer breaks it."""
    K = 2.0
    NX, NY = 12, 9
    solid = np.zeros((NY, NX), np.uint8)
    solid[3:6, 5:7] = 1
    g = O.grid(2, NX, NY, periodic=(True, True), solid=solid)
    p = O.params(2, K, nu_s=5e-3, Pr=0.71)
    half = NX // 2
    rho = 1 + 0.3 * RNG.random((NY, half))
    RT = 0.5 + 1.2 * RNG.random((NY, half))
    u = 0.4 * RNG.standard_normal((2, NY, half))
    rho = np.concatenate([rho, rho[:, ::-1]], 1)
    RT = np.concatenate([RT, RT[:, ::-1]], 1)
    u = np.concatenate([u, u[:, :, ::-1] * np.array([-1.0, 1.0])[:, None, None]], 2)
    M = O.state_from_primitives(g, p, rho, u, RT)
    M[:, solid.reshape(-1) == 1] = 0.0
    st = O.Stats()
    for _ in range(3):
        M = O.step(g, p, M, st)
    assert st.wall_hits > 0
    A = M.reshape(-1, NY, NX)
    B = A[:, :, ::-1]
    # 2D stored moments: M0 Mx My Mxx Mxy Myy MDx MDy G0 Gx Gy; odd in x: Mx Mxy MDx Gx
    sign = np.array([1, -1, 1, 1, -1, 1, -1, 1, 1, -1, 1.0])[:, None, None]
    scale = np.abs(A).max(axis=(1, 2), keepdims=True)
    assert (np.abs(A - sign * B) / scale).max() < 1e-12


def test_wall_through_outflow_pads_keeps_parallel_stream_uniform():
    """A flat slip wall along the bottom that runs out through the outflow side: the outflow
    pads whose nearest interior cell is solid are solid too, so a uniform stream parallel to
    the wall, fed by inflow pads of the same state, stays uniform (the flat-wall invariant of
    Sec. III.B).  A pad copying the empty state of a wall cell instead breaks it at once."""
    nx, ny, pad = 24, 10, 5
    K = 3.0
    rho0, ux, RT0 = 1.0, 0.8, 0.6
    NX, NY = nx + 2 * pad, ny + 2 * pad
    solid = np.zeros((NY, NX), dtype=np.uint8)
    solid[pad, pad:pad + nx] = 1  # interior row 0 along the whole length
    g = O.grid(2, nx, ny, pad=pad, bc=(1, 0, 1, 1), inlet=(rho0, ux, 0.0, RT0), solid=solid.reshape(-1))
    p = O.params(2, K, nu_s=1e-3)
    rho = np.full((ny, nx), rho0)
    u = np.stack([np.full((ny, nx), ux), np.zeros((ny, nx))])
    T = np.full((ny, nx), RT0)
    rho[0] = 0.0  # the wall row: never read
    M0 = O.state_from_primitives(g, p, np.where(rho > 0, rho, rho0), u, T)
    st = O.Stats()
    M = O.run(g, p, M0, 3, st)
    fluid = np.zeros((NY, NX), dtype=bool)
    fluid[pad + 1:pad + ny, pad:pad + nx] = True
    ref = M0[:, fluid.reshape(-1)]
    got = M[:, fluid.reshape(-1)]
    assert np.all(np.isfinite(M))
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
    assert st.fallback_mx == 0 and st.wall_hits > 0


# --- stationary no-slip walls (Sec. III.B, Eq. IIIB8-IIIB15 with u_w = 0) -----------------

def noslip_box(n, seed, RT_lo, RT_hi, umag, kind=2):
    """A periodic n x n grid inside a one-cell frame of wall cells of the given kind."""
    rng = np.random.default_rng(seed)
    solid = np.zeros((n, n), np.uint8)
    solid[0, :] = solid[-1, :] = solid[:, 0] = solid[:, -1] = kind
    g = O.grid(2, n, n, periodic=(True, True), solid=solid.reshape(-1))
    Y, X = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, 4)
    rho = 1.0 + 0.2 * np.cos(2 * np.pi * X / n + ph[0]) * np.cos(2 * np.pi * Y / n + ph[1])
    RT = RT_lo + (RT_hi - RT_lo) * (0.5 + 0.5 * np.sin(2 * np.pi * (X + Y) / n + ph[2]))
    u = umag * np.stack([np.sin(2 * np.pi * Y / n + ph[3]), np.cos(2 * np.pi * X / n + ph[0])])
    return g, solid, rho, u, RT


@pytest.mark.parametrize("RT_lo,RT_hi", [(0.5, 1.5), (0.2, 0.4)])
def test_noslip_closed_box_conserves_mass(RT_lo, RT_hi):
    """The wall returns, as image populations, exactly the mass it took (Eq. IIIB15): the
    total of rho over the fluid cells is conserved to rounding.  (Energy is not a step
    invariant here: images carry the cell's own energy per unit mass, not the absorbed one.)"""
    g, solid, rho, u, RT = noslip_box(18, 5, RT_lo, RT_hi, 0.4)
    p = O.params(2, 3.0, nu_s=5e-3)
    fluid = (solid == 0).reshape(-1)
    M = O.state_from_primitives(g, p, rho, u, RT)
    M[:, ~fluid] = 0.0
    st = O.Stats()
    for _ in range(3):
        M1 = O.step(g, p, M, st)
        assert abs(M1[0, fluid].sum() / M[0, fluid].sum() - 1) < 1e-13
        assert np.all(M1[:, ~fluid] == 0.0)
        M = M1
    assert st.wall_hits > 0 and st.fallback_mx == 0


def test_noslip_gas_at_rest_stays_at_rest():
    g, solid, rho, u, RT = noslip_box(14, 6, 0.6, 0.6, 0.0)
    rho[:] = 1.0
    p = O.params(2, 3.0, nu_s=5e-3)
    M = O.state_from_primitives(g, p, rho, u, RT)
    fluid = (solid == 0).reshape(-1)
    M[:, ~fluid] = 0.0
    M1 = O.run(g, p, M, 3)
    np.testing.assert_allclose(M1[:, fluid], M[:, fluid], rtol=1e-12, atol=1e-13)


def channel_decay_rate(H, steps, nu=0.05, RT=0.5, amp=1e-3, nx=4, kind=2):
    """Decay rate of the lowest shear mode u_x = a sin(pi (y - 1) / H) between two walls
    (interior rows 0 and H + 1), periodic along x."""
    ny = H + 2
    solid = np.zeros((ny, nx), np.uint8)
    solid[0] = solid[-1] = kind
    g = O.grid(2, nx, ny, periodic=(True, True), solid=solid.reshape(-1))
    p = O.params(2, 3.0, nu_s=nu, Pr=1.0, limiter=0)
    yc = np.arange(ny) + 0.5
    mode = np.sin(np.pi * (yc - 1.0) / H)
    mode[0] = mode[-1] = 0.0
    u = np.zeros((2, ny, nx))
    u[0] = amp * mode[:, None]
    M = O.state_from_primitives(g, p, np.ones((ny, nx)), u, np.full((ny, nx), RT))
    fl = (solid == 0).reshape(-1)
    M[:, ~fl] = 0.0
    a = []
    for _ in range(steps):
        M = O.step(g, p, M)
        ux = np.zeros(ny * nx)
        ux[fl] = M[1, fl] / M[0, fl]
        ux = ux.reshape(ny, nx).mean(1)
        a.append((ux * mode).sum() / (mode * mode).sum())
    t = np.arange(1, steps + 1)
    sl = slice(steps // 6, steps)
    return -np.polyfit(t[sl], np.log(np.array(a)[sl]), 1)[0]


def test_noslip_channel_shear_mode_decays_at_viscous_rate():
    """Between two stationary no-slip walls the lowest shear mode decays at nu (pi / H)^2
    (a wall-bounded Sec. IV.A): within 10 % at H = 32, and the deviation (the position of
    the no-slip plane, a fraction of a cell from the wall face) shrinks with H."""
    nu = 0.05
    r32 = channel_decay_rate(32, 400, nu) / (nu * (np.pi / 32) ** 2)
    r16 = channel_decay_rate(16, 200, nu) / (nu * (np.pi / 16) ** 2)
    assert abs(r32 - 1) < 0.10
    assert abs(r16 - 1) > 1.6 * abs(r32 - 1)


# --- moving no-slip walls (kind 3, velocity u_w; Eq. IIIB2-IIIB4, IIIB10-IIIB11) ---------

def channel_state(kbot, ktop, wall_u, u0, H=16, nx=4, RT=0.5, nu=0.1):
    ny = H + 2
    solid = np.zeros((ny, nx), np.uint8)
    solid[0], solid[-1] = kbot, ktop
    g = O.grid(2, nx, ny, periodic=(True, True), solid=solid.reshape(-1), wall_u=wall_u)
    p = O.params(2, 3.0, nu_s=nu, Pr=0.71, limiter=0)
    u = np.zeros((2, ny, nx))
    u[0] = u0
    M = O.state_from_primitives(g, p, np.ones((ny, nx)), u, np.full((ny, nx), RT))
    fl = (solid == 0).reshape(-1)
    M[:, ~fl] = 0.0
    return g, p, M, fl, ny, nx


def test_walls_moving_with_a_uniform_stream_leave_it_uniform():
    """No-slip walls moving at the stream's own velocity impose nothing: the image
    populations (bulk velocity -u + 2 u_w = u, Eq. IIIB4) replace exactly what the walls
    absorbed, so the stream stays uniform; walls at rest slow it down."""
    g, p, M0, fl, _, _ = channel_state(3, 3, (0.3, 0.0), 0.3)
    M = O.run(g, p, M0, 4)
    dev = np.abs(M[:, fl] - M0[:, fl]).max() / np.abs(M0[:, fl]).max()
    assert dev < 1e-13
    assert abs(M[0, fl].sum() / M0[0, fl].sum() - 1) < 1e-13
    g2, p2, N0, _, _, _ = channel_state(2, 2, (0.0, 0.0), 0.3)
    N = O.run(g2, p2, N0, 4)
    assert N[1, fl].sum() < 0.99 * N0[1, fl].sum()


def test_couette_flow_profile_is_linear_between_the_walls():
    """Plane Couette flow: a wall at rest below (kind 2) and a wall moving at U above (kind 3).
    The steady velocity profile is linear, 0 at the lower wall face (y = 1) and U at the upper
    one (y = H + 1), each within a fifth of a cell; residuals below 0.1 % of U."""
    U, H = 0.05, 16
    g, p, M, fl, ny, nx = channel_state(2, 3, (U, 0.0), 0.0, H=H, nu=0.2)
    M = O.run(g, p, M, 1500)
    ux = (M[1, fl] / M[0, fl]).reshape(H, nx).mean(1)
    y = np.arange(1, H + 1) + 0.5
    a, b = np.polyfit(y, ux, 1)
    assert abs(-b / a - 1.0) < 0.2
    assert abs((U - b) / a - (H + 1.0)) < 0.2
    assert np.abs(ux - (a * y + b)).max() < 1e-3 * U
