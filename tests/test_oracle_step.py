"""Pins of the oracle's full time step: moment streaming (Eq. IIE3), fluid boundaries
(Sec. III.A), conservation, Galilean invariance, hot box, exact Riemann solutions and
transport coefficients (Sec. IV)."""
import json
import os

import numpy as np
import pytest

import oracle as O
import exact_riemann as ER

RNG = np.random.default_rng(11)
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "las_examples.json")))


def totals(D, M):
    t = M.sum(1)
    E = t[2] + t[4] if D == 1 else t[3] + t[5] + t[8]
    return t[0], t[1:1 + D], E


def primitives(D, K, M):
    rho = M[0]
    u = M[1:1 + D] / rho
    tr = M[2] if D == 1 else M[3] + M[5]
    G0 = M[4] if D == 1 else M[8]
    RT = ((tr + G0) / rho - (u ** 2).sum(0)) / (D + K)
    return rho, u, RT


def random_periodic_state(D, K, n, RTlo, RThi, umag):
    shp = (n[1], n[0]) if D == 2 else (n[0],)
    g = O.grid(D, n[0], n[1] if D == 2 else 1, periodic=(True, True))
    p = O.params(D, K, nu_s=5e-3, Pr=0.71)
    rho = 1 + 0.2 * RNG.random(shp)
    RT = RTlo + (RThi - RTlo) * RNG.random(shp)
    u = umag * RNG.standard_normal((D,) + shp)
    return g, p, O.state_from_primitives(g, p, rho, u, RT)


@pytest.mark.parametrize("D,K,n,RTlo,RThi", [(1, 4.0, (40, 1), 0.3, 3.0), (2, 3.0, (10, 8), 0.25, 0.9),
                                             (2, 3.0, (8, 6), 1.5, 4.0)])
def test_periodic_conservation_per_step(D, K, n, RTlo, RThi):
    """Mass, momentum and energy are conserved to 1e-13 relative per step (Eq. B5, IIE3)."""
    g, p, M = random_periodic_state(D, K, n, RTlo, RThi, 0.6)
    st = O.Stats()
    for _ in range(2):
        m0, p0, e0 = totals(D, M)
        M = O.step(g, p, M, st)
        m1, p1, e1 = totals(D, M)
        assert abs(m1 / m0 - 1) < 1e-13
        assert np.abs(p1 - p0).max() / m0 < 1e-13
        assert abs(e1 / e0 - 1) < 1e-13
    assert st.fallback_eq == 0 and st.fallback_mx == 0
    # positivity of the reconstructed state: density and temperature stay positive
    rho, u, RT = primitives(D, K, M)
    assert rho.min() > 0 and RT.min() > 0


@pytest.mark.parametrize("D,K,RT", [(1, 4.0, 0.5), (1, 4.0, 32.0), (2, 3.0, 0.5), (2, 3.0, 2.0), (2, 3.0, 0.3)])
def test_hot_box_stays_uniform(D, K, RT):
    """Sec. IV.E hot box: a uniform equilibrium at u = (10, 10) is unchanged by any number of steps."""
    n = (6, 5) if D == 2 else (12, 1)
    g = O.grid(D, n[0], n[1], periodic=(True, True))
    p = O.params(D, K, nu_s=1e-3)
    shp = (n[1], n[0]) if D == 2 else (n[0],)
    u = np.full((D,) + shp, 10.0)
    M0 = O.state_from_primitives(g, p, np.ones(shp), u, np.full(shp, RT))
    nsteps = 3
    M = O.run(g, p, M0, nsteps)
    # Raw moments at |u| >> sqrt(RT) carry the central third moments with a relative rounding
    # of about (|u|/sqrt(RT))^3 eps per step (the cancellation Sec. II.B avoids by colliding in
    # the relative frame); the state must stay uniform to that level.
    bound = nsteps * 4 * np.finfo(float).eps * (10.0 * np.sqrt(D) / np.sqrt(RT)) ** 3 + 1e-14
    assert np.abs(M / M0 - 1).max() < bound


@pytest.mark.parametrize("D,U", [(1, (3,)), (2, (2, -1))])
def test_integer_galilean_shift(D, U):
    """state(x, t; u + U) = state(x - U t, t; u) for integer U: the stencil set and every
    landing cell translate by U (Eq. IIC6, IIC10, IIE3)."""
    K = 4.0 if D == 1 else 3.0
    n = (24, 1) if D == 1 else (9, 7)
    g, p, MA = random_periodic_state(D, K, n, 0.3, 1.2, 0.4)
    shp = (n[1], n[0]) if D == 2 else (n[0],)
    rho, u, RT = primitives(D, K, MA)
    rho, RT, u = rho.reshape(shp), RT.reshape(shp), u.reshape((D,) + shp)
    uB = u + np.array(U, dtype=float).reshape((D,) + (1,) * len(shp))
    MB = O.state_from_primitives(g, p, rho, uB, RT)
    nsteps = 2
    MA = O.run(g, p, MA, nsteps)
    MB = O.run(g, p, MB, nsteps)
    ra, ua, Ta = primitives(D, K, MA)
    rb, ub, Tb = primitives(D, K, MB)
    ra, Ta = ra.reshape(shp), Ta.reshape(shp)
    rb, Tb = rb.reshape(shp), Tb.reshape(shp)
    ua, ub = ua.reshape((D,) + shp), ub.reshape((D,) + shp)
    axes = (0,) if D == 1 else (1, 0)
    shift = tuple(U[a] * nsteps for a in range(D))
    rs = np.roll(ra, shift, axis=axes)
    np.testing.assert_allclose(rb, rs, rtol=1e-11)
    np.testing.assert_allclose(Tb, np.roll(Ta, shift, axis=axes), rtol=1e-10)
    for a in range(D):
        np.testing.assert_allclose(ub[a] - U[a], np.roll(ua[a], shift, axis=axes), atol=1e-10)


def test_boundary_fill_inflow_and_outflow():
    """Sec. III.A: inflow pads carry the prescribed equilibrium, outflow pads copy the nearest
    interior cell's full moments (non-equilibrium included)."""
    D, K = 2, 3.0
    g = O.grid(D, 5, 4, pad=2, bc=(1, 0, 0, 0), inlet=(1.4, 3.0, 0.0, 0.714))
    p = O.params(D, K)
    NY, NX = O.padded_shape(g)
    M = RNG.random((O.nmom(D), NY * NX)) + 0.5
    W = O.fill_pads(g, p, M).reshape(O.nmom(D), NY, NX)
    Mi = M.reshape(O.nmom(D), NY, NX)
    eq = O.eq_moments(D, K, 1.4, [3.0, 0.0], 0.714)
    for iy in range(NY):
        for ix in range(NX):
            inside = 2 <= ix < 7 and 2 <= iy < 6
            if inside:
                np.testing.assert_array_equal(W[:, iy, ix], Mi[:, iy, ix])
            elif ix < 2:
                np.testing.assert_allclose(W[:, iy, ix], eq)
            else:
                sx, sy = min(max(ix, 2), 6), min(max(iy, 2), 5)
                np.testing.assert_array_equal(W[:, iy, ix], Mi[:, sy, sx])


def test_exact_riemann_solver_self_consistency():
    """The test-side exact solver reproduces Sod's star state (p* = 0.30313, u* = 0.92745, the
    textbook values) and satisfies Rankine-Hugoniot across its shock."""
    g = GOLD["sod"]
    left = (1.0, 0.0, 1.0)
    right = (0.125, 0.0, 0.125 * 0.8)
    ps, us = ER.star_state(left, right, 1.4)
    assert ps == pytest.approx(0.30313, abs=1e-5) and us == pytest.approx(0.92745, abs=1e-5)
    xi = np.linspace(-2, 2, 4001)
    r, u, p = ER.sample(left, right, 1.4, xi)
    # shock: last jump of rho on the right; check mass and momentum flux continuity
    j = np.nonzero(np.abs(np.diff(r)) > 1e-3)[0][-1]
    S = 0.5 * (xi[j] + xi[j + 1])
    r1, u1, p1 = r[j], u[j], p[j]
    r2, u2, p2 = r[j + 1], u[j + 1], p[j + 1]
    assert r1 * (u1 - S) == pytest.approx(r2 * (u2 - S), rel=2e-3)
    assert r1 * (u1 - S) ** 2 + p1 == pytest.approx(r2 * (u2 - S) ** 2 + p2, rel=2e-3)
    assert g["t"] == 0.2


def sod_l1(N, steps_scale=1.0):
    D, K = 1, 4.0
    p = O.params(D, K, nu_s=1e-3, Pr=0.71)
    pad = 8
    g = O.grid(1, N, pad=pad)
    x = (np.arange(N) + 0.5) / N
    rho = np.where(x < 0.5, 1.0, 0.125)
    RT = np.where(x < 0.5, 1.0, 0.8)
    M = O.state_from_primitives(g, p, rho, np.zeros((1, N)), RT)
    st = O.Stats()
    M = O.run(g, p, M, int(round(0.2 * N)), st)
    r, u, T = primitives(D, K, M[:, pad:pad + N])
    re, ue, pe = ER.sample((1, 0, 1), (0.125, 0, 0.1), 1.4, (x - 0.5) / 0.2)
    return np.mean(np.abs(r - re)), np.mean(np.abs(u[0] - ue)), np.mean(np.abs(r * T - pe)), st


def test_sod_converges_to_exact_solution():
    """Sec. V.A: Sod's shock tube at t = 0.2 approaches the exact solution as N grows
    (N = 200, 400, 800, the paper's resolutions)."""
    errs = [sod_l1(N) for N in GOLD["sod"]["N"]]
    for a, b in zip(errs, errs[1:]):
        for k in range(3):
            assert b[k] < 0.8 * a[k]
    assert errs[-1][0] < 6e-3
    assert all(e[3].fallback_mx == 0 for e in errs)


def _decay_run(kind, nu, RT, L=32, amp=1e-3, Fo=1.0):
    D, K = 2, (3.0 if kind == "shear" else 0.0)
    p = O.params(D, K, nu_s=nu, Pr=1.0, limiter=0)
    g = O.grid(D, L, 1, periodic=(True, True))
    x = np.arange(L) + 0.5
    k = 2 * np.pi / L
    if kind == "shear":  # Eq. (VA1) with u0 = 0
        rho = np.ones((1, L))
        u = np.stack([np.zeros((1, L)), amp * np.cos(k * x)[None, :]])
        T = np.full((1, L), RT)
    else:  # Eq. (VB1) with u0 = 0
        rho = (1.0 + amp * np.cos(k * x))[None, :]
        u = np.zeros((2, 1, L))
        T = RT / rho
    M = O.state_from_primitives(g, p, rho, u, T)
    nsteps = int(round(Fo / (nu * k * k)))
    M = O.run(g, p, M, nsteps)
    if kind == "shear":
        a = np.abs(M[2] / M[0]).max()  # Eq. (VA4)
    else:
        a = np.abs(M[0] - 1.0).max()  # Eq. (VB3)
    return -np.log(a / amp) / (k * k * nsteps)


@pytest.mark.parametrize("kind", ["shear", "thermal"])
def test_transport_coefficients_from_wave_decay(kind):
    """Sec. IV.A-B: the measured shear viscosity and thermal diffusivity are within the paper's
    +-10% of the imposed nu (alpha = nu / Pr, Pr = 1) at RT = 0.5 (Eq. C7-C8, VA4, VB3)."""
    nu = 0.1
    meas = _decay_run(kind, nu, 0.5)
    assert abs(meas / nu - 1) < 0.10


@pytest.mark.parametrize("K", [0.0, 2.0, 4.0])
def test_sound_speed_from_acoustic_pulse(K):
    """Sec. IV.D, Eq. (VD1): a small density pulse travels at c_s = sqrt(gamma RT) with
    gamma = (D + K + 2)/(D + K) (App. B Eq. B22)."""
    D, N, RT = 1, 240, 1.0
    p = O.params(D, K, nu_s=1e-3, Pr=1.0)
    g = O.grid(D, N, periodic=(True, True))
    x = np.arange(N) + 0.5
    x0 = N / 2
    rho = 1.0 + 1e-6 * np.exp(-((x - x0) / 4.0) ** 2)
    M = O.state_from_primitives(g, p, rho, np.zeros((1, N)), np.full(N, RT))
    nsteps = 60
    M = O.run(g, p, M, nsteps)
    r, u, T = primitives(D, K, M)
    pr = r * T - 1.0 * RT
    half = pr[N // 2:]
    i = int(np.argmax(half))
    y0, y1, y2 = half[i - 1], half[i], half[i + 1]
    xp = x[N // 2 + i] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    cs = (xp - x0) / nsteps
    gamma = (D + K + 2) / (D + K)
    assert cs == pytest.approx(np.sqrt(gamma * RT), rel=0.02)


@pytest.mark.parametrize("D", [1, 2])
def test_refined_landing_moves_centre_of_mass_by_momentum(D):
    """Streaming moves every population to x + c (Eq. IIE3); a refined child landing between
    cells is shared so that its mass-weighted landing position is exactly x + c (cloud in
    cell, 3/4 and 1/4 per axis at level 1).  So over one step the centre of mass moves by
    the total momentum: sum(x rho)' = sum(x rho) + sum(rho u).  A cold blob (RT = 0.3 < 4/9,
    one refinement level) moving inside a resting uniform background checks it; the
    background is symmetric, so what crosses the periodic edges cancels."""
    n = 48 if D == 1 else 20
    K = 4.0 if D == 1 else 3.0
    g = O.grid(D, n, n if D == 2 else 1, periodic=(True, True))
    p = O.params(D, K, nu_s=5e-3, Pr=0.71)
    assert O.refine_levels(p, 0.3) == 1
    shp = (n, n) if D == 2 else (n,)
    rho = np.ones(shp)
    u = np.zeros((D,) + shp)
    RT = np.full(shp, 0.3)
    rng = np.random.default_rng(29)
    blob = (slice(n // 2 - 3, n // 2 + 3),) * D
    rho[blob] = 1.0 + 0.4 * rng.random(rho[blob].shape)
    for a in range(D):
        u[(a,) + blob] = 0.8 * rng.random(rho[blob].shape) - 0.2
    RT[blob] = 0.25 + 0.1 * rng.random(rho[blob].shape)
    M = O.state_from_primitives(g, p, rho, u, RT)
    c = (n - 1) / 2.0
    if D == 1:
        pos = [np.arange(n) - c]
    else:
        iy, ix = np.divmod(np.arange(n * n), n)
        pos = [ix - c, iy - c]
    st = O.Stats()
    for _ in range(2):
        M1 = O.step(g, p, M, st)
        for a in range(D):
            moved = (pos[a] * M1[0]).sum() - (pos[a] * M[0]).sum()
            assert abs(moved - M[1 + a].sum()) < 1e-11, (a, moved, M[1 + a].sum())
        M = M1
    assert st.fallback_eq == 0 and st.fallback_mx == 0


def test_failed_solve_falls_back_to_equilibrium_constraints():
    """A cell whose post-collision constraints no positive populations can meet (a negative
    normal stress deeper than the pressure, kept after a weak collision: large viscosity, no
    limiter) is solved with the equilibrium constraints of both populations instead.  Its
    emitted moments are then those of a cell holding the equilibrium state of the same
    rho, u and RT, so the whole step matches that state's step."""
    D, K, n = 2, 3.0, 8
    g = O.grid(D, n, n, periodic=(True, True))
    p = O.params(D, K, nu_s=5.0, Pr=0.71, limiter=0)
    rho = np.ones((n, n))
    u = np.zeros((D, n, n))
    u[0], u[1] = 0.2, -0.1
    RT = np.full((n, n), 0.6)
    M_eq = O.state_from_primitives(g, p, rho, u, RT)
    M_bad = M_eq.copy()
    cell = 3 * n + 4
    d, e = 2.0, 0.6  # multiples of rho RT; the energy trM2 + G0 is unchanged
    M_bad[3, cell] -= d * 0.6
    M_bad[5, cell] += (d - e) * 0.6
    M_bad[8, cell] += e * 0.6
    co = O.collide(p, M_bad[:, cell])
    assert co["cf"][3] < 0.0  # the xx constraint asks for a negative variance
    assert np.abs(co["cg"][1:3]).max() > 0.01  # and the phonon heat-flux constraints are not zero
    st_bad, st_eq = O.Stats(), O.Stats()
    out_bad = O.step(g, p, M_bad, st_bad)
    out_eq = O.step(g, p, M_eq, st_eq)
    assert st_bad.fallback_eq == 1 and st_bad.fallback_mx == 0
    assert st_eq.fallback_eq == 0
    scale = np.abs(out_eq).max(axis=1, keepdims=True)
    assert (np.abs(out_bad - out_eq) / scale).max() < 1e-13


# The last resort of the failure handling: when even the equilibrium constraints cannot be met
# (here forced by allowing a single Newton update, which cannot reach 1e-12 on a discrete
# stencil), the populations are Maxwellian weights on the cell's own stencil, normalised to carry
# the cell's mass.  Such weights are a quadrature of the Gaussian of mean u and variance RT per
# axis: on a stencil reaching about n_conf = 4 standard deviations the truncated tails and the
# lattice's aliasing (Poisson summation) leave the mean within 1e-2 sqrt(RT) and the variance
# within 3 % (cold refined stencils; about 1e-3 on the integer lattice).  A weight taken at
# c instead of c - u, a flipped exponent sign or a missing normalisation each fail these.
# Dropping the quadrature weights dC of a refined stencil moves the mean and variance by less
# than the quadrature's own error (a few parts per thousand), so they are not pinned here.
LAST_RESORT_CASES = [
    (1, 0.0, (2.5,), 1.0),
    (1, 2.0, (0.3,), 0.2),  # refined (RT < 4/9): dC of 1/2 and 1
    (2, 0.0, (2.5, -1.2), 1.0),
    (2, 2.0, (0.4, 0.7), 0.15),  # refined: dC of 1/4, 1/2 and 1
    (2, 0.0, (0.0, 0.0), 8.0),
    (3, 0.0, (1.5, 0.2, -0.7), 1.0),
]


@pytest.mark.parametrize("D,K,u,RT", LAST_RESORT_CASES)
def test_last_resort_weights_are_a_gaussian_quadrature(D, K, u, RT):
    p = O.params(D, K, max_iter=1)
    u = np.array(u)
    M = O.eq_moments(D, K, 1.3, u, RT)
    _, c, dC, pf, pg, level = O.cell_populations(p, M)
    assert level == 2  # both the solve and the equilibrium-constraint solve failed
    assert (pf > 0).all()
    assert abs(pf.sum() - 1.0) < 1e-14
    mean = pf @ c
    assert np.abs(mean - u).max() < 1e-2 * np.sqrt(RT), mean - u
    var = (pf * ((c - u) ** 2).sum(1)).sum() / D
    assert abs(var / RT - 1.0) < 0.03, var / RT
    if K > 0:
        np.testing.assert_array_equal(pg, pf)  # the phonons take the same weights


def test_last_resort_step_conserves_mass_and_stays_uniform():
    """A uniform periodic grid in which every cell takes the last resort: each cell falls back
    once, mass is conserved to rounding, the state stays uniform (every cell emits the same
    populations) and the momentum is rho times the quadrature's mean, within 1e-2 of rho u."""
    D, K, nx, ny = 2, 0.0, 8, 6
    g = O.grid(D, nx, ny, periodic=(True, True))
    p = O.params(D, K, max_iter=1)
    rho = np.full((ny, nx), 1.3)
    u = np.zeros((D, ny, nx))
    u[0], u[1] = 0.4, 0.7
    RT = np.full((ny, nx), 1.0)
    M = O.state_from_primitives(g, p, rho, u, RT)
    st = O.Stats()
    out = O.step(g, p, M, st)
    assert st.fallback_mx == nx * ny and st.fallback_eq == 0
    assert abs(out[0].sum() / M[0].sum() - 1.0) < 1e-13
    assert (np.abs(out - out[:, :1]).max(axis=1) <= 1e-13 * np.abs(out).max(axis=1)).all()
    assert np.abs(out[1:3, 0] / out[0, 0] - np.array([0.4, 0.7])).max() < 1e-2
