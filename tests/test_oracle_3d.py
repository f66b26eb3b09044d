"""Pins of the oracle in three dimensions (the paper's general-D formulation, Sec. II, with
D = 3: 17 stored moments, N_f = 19 and N_g = 10 constraints, Eq. IIB5, IIB14-IIB17), each
independent of the oracle: quadrature of the Maxwellian, brute-force moment sums, closed forms,
a convex-dual minimiser, conservation, invariance and the transport laws of Sec. IV."""
import itertools

import numpy as np
import pytest
from scipy.optimize import minimize

import oracle as O
from test_oracle_collision import brute_raw, gh_eq_moments

RNG = np.random.default_rng(3003)
D = 3


def test_sizes():
    assert (O.nmom(3), O.nf(3), O.ng(3)) == (17, 19, 10)
    assert (O.nmom(2), O.nf(2), O.ng(2)) == (11, 10, 6)
    assert (O.nmom(1), O.nf(1), O.ng(1)) == (6, 4, 3)


@pytest.mark.parametrize("K", [2.0, 0.0])
def test_equilibrium_moments_match_quadrature(K):
    rho, u, RT = 1.3, np.array([0.7, -1.9, 0.4]), 0.83
    np.testing.assert_allclose(O.eq_moments(D, K, rho, u, RT), gh_eq_moments(D, K, rho, u, RT, n=10),
                               rtol=1e-12, atol=1e-12)


def test_macros_roundtrip_and_neq_brute_force():
    K = 2.0
    for _ in range(10):
        rho, u, RT = RNG.uniform(0.1, 3), RNG.normal(0, 5, D), RNG.uniform(0.05, 50)
        r2, u2, RT2 = O.macros(D, K, O.eq_moments(D, K, rho, u, RT))
        assert r2 == pytest.approx(rho, rel=1e-14)
        np.testing.assert_allclose(u2, u, rtol=1e-13, atol=1e-13)
        assert RT2 == pytest.approx(RT, rel=1e-11)
    for _ in range(10):
        c = RNG.normal(0.3, 1.2, size=(60, D))
        f = RNG.random(60) + 0.05
        g = (RNG.random(60) + 0.05) * K
        M = brute_raw(D, c, f, g)
        rho, u, RT = O.macros(D, K, M)
        ct = c - u
        P_ref = np.array([[(ct[:, a] * ct[:, b] * f).sum() - (rho * RT if a == b else 0.0) for b in range(D)]
                          for a in range(D)])
        Q_ref = np.array([((ct ** 2).sum(1) * ct[:, k] * f).sum() for k in range(D)])
        P, Q, G0n, Gn = O.neq(D, K, M)
        sc = max(1.0, np.abs(M).max())
        np.testing.assert_allclose(P, P_ref, atol=1e-12 * sc)
        np.testing.assert_allclose(Q, Q_ref, atol=1e-12 * sc)
        assert G0n == pytest.approx(g.sum() - rho * K * RT, abs=1e-12 * sc)
        np.testing.assert_allclose(Gn, [(ct[:, a] * g).sum() for a in range(D)], atol=1e-12 * sc)
        assert np.trace(P) + G0n == pytest.approx(0.0, abs=1e-12 * sc)


def test_collision_limits_and_energy():
    """omega = 1 gives the Maxwellian constraints, omega -> 0 the pre-collision central moments,
    and the energy (D + K) rho RT is kept for any omega (Eq. IIB16-IIB18, B5c)."""
    K = 2.0
    c = RNG.normal(0.3, 1.2, size=(60, D))
    f = RNG.random(60) + 0.05
    g = (RNG.random(60) + 0.05) * K
    M = brute_raw(D, c, f, g)
    rho, u, RT = O.macros(D, K, M)
    ct = c - u
    one = O.collide(O.params(D, K, nu_s=0.5 * RT, nu_b=-1.0, Pr=1.0, limiter=0), M)
    ref_f = [1.0] + [0.0] * D + [RT if a == b else 0.0 for a in range(D) for b in range(a, D)] + [0.0] * D * D
    np.testing.assert_allclose(one["cf"], ref_f, atol=1e-12)
    ref_g = [1.0] + [0.0] * D + [RT if a == b else 0.0 for a in range(D) for b in range(a, D)]
    np.testing.assert_allclose(one["cg"], ref_g, atol=1e-12)
    ident = O.collide(O.params(D, K, nu_s=1e14, nu_b=1e14, Pr=1.0, limiter=0), M)
    j = 1 + D
    for a in range(D):
        for b in range(a, D):
            assert ident["cf"][j] == pytest.approx((ct[:, a] * ct[:, b] * f).sum() / rho, abs=1e-9)
            j += 1
    heat = ident["cf"][j:].reshape(D, D)  # [gamma][alpha]
    np.testing.assert_allclose(heat.sum(1), [((ct ** 2).sum(1) * ct[:, k] * f).sum() / rho for k in range(D)],
                               atol=1e-9)
    diag = [1 + D + sum(D - k for k in range(a)) for a in range(D)]
    for nu in (1e-300, 0.1, 0.5 * RT, 1e14):
        co = O.collide(O.params(D, K, nu_s=nu, nu_b=-1.0, Pr=0.7, limiter=0), M)
        energy = sum(co["cf"][i] for i in diag) + K * RT * co["cg"][0]
        assert energy == pytest.approx((D + K) * RT, rel=1e-12)


def test_knudsen_dimensionless_and_complete():
    """Eq. (D2) in 3D: a change of time unit and a Galilean shift leave Kn unchanged; every
    non-equilibrium part alone gives Kn > 0."""
    K = 2.0
    c = RNG.normal(0.3, 1.2, size=(60, D))
    f = RNG.random(60) + 0.05
    g = RNG.random(60) + 0.05

    def kn(M):
        rho, u, RT = O.macros(D, K, M)
        P, Q, G0n, Gn = O.neq(D, K, M)
        return O.knudsen(D, K, rho, RT, P, Q, G0n, Gn)

    k = kn(brute_raw(D, c, f, g * K))
    assert k > 1e-3
    for sc in (0.3, 2.5, 11.0):
        assert kn(brute_raw(D, c / sc, f, g * K / sc ** 2)) == pytest.approx(k, rel=1e-10)
    assert kn(brute_raw(D, c + np.array([3.7, -1.2, 0.8]), f, g * K)) == pytest.approx(k, rel=1e-9)
    M0 = O.eq_moments(D, K, 1.1, np.array([0.4, -0.7, 0.2]), 0.8)
    assert kn(M0) < 1e-14
    # stored order: M0, Mx..Mz (1-3), Mxx Mxy Mxz Myy Myz Mzz (4-9), MD (10-12), G0 (13), G (14-16)
    for name, idx, dv in [("shear xz", [6], [0.05]), ("fluon heat flux", [11], [0.07]),
                          ("phonon heat flux", [16], [0.06]), ("bulk", [4, 7, 9, 13], [0.03, 0.03, 0.03, -0.09])]:
        M = M0.copy()
        M[idx] += dv
        assert kn(M) > 1e-3, name


def test_las_ball_and_refinement():
    """Eq. (IIC6) in 3D: the level-0 points are the integer velocities within R_ac + 1/2 of u
    (counted here by brute force over a box); refinement (Eq. IIC10-11) replaces a point by 8
    children of a quarter spacing with dC / 8, keeping sum dC; the set translates with u."""
    p = O.params(D, 2.0)
    for RT, u in [(0.5, [0.3, -0.2, 0.45]), (2.0, [1.7, 0.1, -2.6]), (0.2, [0.05, 0.4, -0.3])]:
        u = np.array(u)
        R = max(int(np.floor(4 * np.sqrt(RT) + 0.5)), 2)
        box = np.arange(-R - 3, R + 4)
        X, Y, Z = np.meshgrid(box, box, box, indexing="ij")
        pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) + np.floor(u).astype(int)
        n0 = int((((pts - u) ** 2).sum(1) <= (R + 0.5) ** 2).sum())
        c, dC, lev = O.las(D, u, RT, p)
        assert dC.sum() == pytest.approx(n0, rel=1e-14)
        if RT > 0.44:
            assert len(c) == n0 and np.all(lev == 0)
        else:  # Nr = round(1 / (3 sqrt 0.2)) = 1: the points within 1.5 of u split in 8
            nsplit = int((((pts - u) ** 2).sum(1) <= 1.5 ** 2).sum())
            assert len(c) == n0 + 7 * nsplit
            assert np.all(dC[lev == 1] == 0.125)
        c2, dC2, _ = O.las(D, u + np.array([2, -1, 3]), RT, p)
        np.testing.assert_array_equal(np.sort((c2 - [2, -1, 3]).view("f8,f8,f8"), axis=0),
                                      np.sort(c.view("f8,f8,f8"), axis=0))


def monomials3(kind, ct):
    x, y, z = ct[:, 0], ct[:, 1], ct[:, 2]
    cols = [np.ones_like(x), x, y, z, x * x, x * y, x * z, y * y, y * z, z * z]
    if kind == 0:  # c_a^2 c_g, gamma-major
        cols += [x ** 3, y * y * x, z * z * x, x * x * y, y ** 3, z * z * y, x * x * z, y * y * z, z ** 3]
    return np.stack(cols, 1)


@pytest.mark.parametrize("kind,RT,u", [(0, 0.6, [0.2, -0.35, 0.1]), (1, 0.6, [0.2, -0.35, 0.1]),
                                       (0, 1.2, [-1.3, 0.45, 2.2])])
def test_epr_matches_convex_dual_and_planted_multipliers(kind, RT, u):
    p = O.params(D, 2.0)
    u = np.array(u)
    c, dC, _ = O.las(D, u, RT, p)
    T = monomials3(kind, c - u)
    b, o = O.basis(D, kind, np.array([0.3, -0.7, 1.1]))
    np.testing.assert_allclose(b, monomials3(kind, np.array([[0.3, -0.7, 1.1]]))[0], rtol=1e-15)
    lam_t = O.maxwell_lambda(D, kind, RT)
    lam_t = lam_t + 0.05 * RNG.standard_normal(len(lam_t)) / np.maximum(1, np.arange(len(lam_t)))
    con = T.T @ (dC * np.exp(-1 - T @ lam_t))
    st, lam, pop = O.epr(D, kind, c, dC, u, RT, con, p)
    assert st >= 0
    np.testing.assert_allclose(lam, lam_t, rtol=1e-8, atol=1e-8)

    def fun(l):
        w = dC * np.exp(-1.0 - T @ l)
        return w.sum() + l @ con, -(T * w[:, None]).sum(0) + con, (T.T * w) @ T

    res = minimize(lambda l: fun(l)[0], O.maxwell_lambda(D, kind, RT), jac=lambda l: fun(l)[1],
                   hess=lambda l: fun(l)[2], method="trust-exact", options=dict(gtol=1e-13, maxiter=500))
    np.testing.assert_allclose(lam, res.x, rtol=1e-7, atol=1e-7)
    assert np.all(pop > 0)


def periodic_grid(n, K, nu=5e-3, Pr=0.71):
    g = O.grid(D, n[0], n[1], nz=n[2], periodic=(True, True, True))
    return g, O.params(D, K, nu_s=nu, Pr=Pr)


def totals(M):
    t = M.sum(1)
    return t[0], t[1:4], t[4] + t[7] + t[9] + t[13]


def test_periodic_conservation_per_step():
    K, n = 2.0, (5, 4, 3)
    g, p = periodic_grid(n, K)
    shp = (n[2], n[1], n[0])
    rho = 1 + 0.2 * RNG.random(shp)
    RT = 0.3 + 1.2 * RNG.random(shp)
    u = 0.6 * RNG.standard_normal((D,) + shp)
    M = O.state_from_primitives(g, p, rho, u, RT)
    st = O.Stats()
    for _ in range(2):
        m0, p0, e0 = totals(M)
        M = O.step(g, p, M, st)
        m1, p1, e1 = totals(M)
        assert abs(m1 / m0 - 1) < 1e-13
        assert np.abs(p1 - p0).max() / m0 < 1e-13
        assert abs(e1 / e0 - 1) < 1e-13
    assert st.fallback_mx == 0 and st.q_max > 100


@pytest.mark.parametrize("RT", [0.5, 0.3])
def test_hot_box_stays_uniform(RT):
    """Sec. IV.E in 3D: a uniform equilibrium at u = (10, 10, 10) is unchanged by steps (to the
    rounding that raw moments at |u| >> sqrt(RT) carry, cf. the 1D/2D hot box test)."""
    K, n = 2.0, (3, 3, 2)
    g, p = periodic_grid(n, K, nu=1e-3)
    shp = (n[2], n[1], n[0])
    M0 = O.state_from_primitives(g, p, np.ones(shp), np.full((D,) + shp, 10.0), np.full(shp, RT))
    M = O.run(g, p, M0, 2)
    bound = 2 * 4 * np.finfo(float).eps * (10.0 * np.sqrt(D) / np.sqrt(RT)) ** 3 + 1e-14
    assert np.abs(M / M0 - 1).max() < bound


def test_integer_galilean_shift():
    K, n, U = 2.0, (5, 4, 4), (1, -2, 1)
    g, p = periodic_grid(n, K)
    shp = (n[2], n[1], n[0])
    rho = 1 + 0.2 * RNG.random(shp)
    RT = 0.3 + 0.9 * RNG.random(shp)
    u = 0.4 * RNG.standard_normal((D,) + shp)
    MA = O.state_from_primitives(g, p, rho, u, RT)
    MB = O.state_from_primitives(g, p, rho, u + np.array(U, dtype=float).reshape(3, 1, 1, 1), RT)
    MA = O.step(g, p, MA)
    MB = O.step(g, p, MB)
    ra = MA[0].reshape(shp)
    rb = MB[0].reshape(shp)
    np.testing.assert_allclose(rb, np.roll(ra, (U[2], U[1], U[0]), axis=(0, 1, 2)), rtol=1e-11)


@pytest.mark.parametrize("K", [0.0, 2.0])
def test_sound_speed_from_acoustic_pulse(K):
    """Sec. IV.D, Eq. (VD1) in 3D: a plane pulse travels at sqrt(gamma RT), gamma = (D+K+2)/(D+K)
    = 5/3 (K = 0) and 7/5 (K = 2), within 2 %."""
    N, RT = 160, 1.0
    g = O.grid(D, N, 1, nz=1, periodic=(True, True, True))
    p = O.params(D, K, nu_s=1e-3, Pr=1.0)
    x = np.arange(N) + 0.5
    x0 = N / 2
    rho = (1.0 + 1e-6 * np.exp(-((x - x0) / 4.0) ** 2)).reshape(1, 1, N)
    M = O.state_from_primitives(g, p, rho, np.zeros((D, 1, 1, N)), np.full((1, 1, N), RT))
    nsteps = 40
    M = O.run(g, p, M, nsteps)
    r, u, T = [], [], []
    for i in range(N):
        rr, uu, TT = O.macros(D, K, M[:, i])
        r.append(rr)
        T.append(TT)
    pr = np.array(r) * np.array(T) - RT
    half = pr[N // 2:]
    i = int(np.argmax(half))
    y0, y1, y2 = half[i - 1], half[i], half[i + 1]
    xp = x[N // 2 + i] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    gamma = (D + K + 2) / (D + K)
    assert (xp - x0) / nsteps == pytest.approx(np.sqrt(gamma * RT), rel=0.02)


def test_shear_wave_decay():
    """Sec. IV.A in 3D: a transverse wave u_z = a cos(k x) decays at nu k^2 within 10 %."""
    K, nu, RT, L, amp = 2.0, 0.1, 0.5, 32, 1e-3
    g = O.grid(D, L, 1, nz=1, periodic=(True, True, True))
    p = O.params(D, K, nu_s=nu, Pr=1.0, limiter=0)
    k = 2 * np.pi / L
    x = np.arange(L) + 0.5
    u = np.zeros((D, 1, 1, L))
    u[2, 0, 0] = amp * np.cos(k * x)
    M = O.state_from_primitives(g, p, np.ones((1, 1, L)), u, np.full((1, 1, L), RT))
    nsteps = int(round(1.0 / (nu * k * k)))
    M = O.run(g, p, M, nsteps)
    a = np.abs(M[3] / M[0]).max()
    meas = -np.log(a / amp) / (k * k * nsteps)
    assert abs(meas / nu - 1) < 0.10


def test_refined_landing_moves_centre_of_mass_by_momentum():
    """Moment streaming in 3D with refined children landing between cells (cloud-in-cell,
    reading of Eq. IIA10-11): the total first moment of the mass moves by the total momentum
    in one step, sum x rho' = sum x rho + sum rho u (periodic box, away from the wrap)."""
    K, n = 2.0, (12, 12, 12)
    g, p = periodic_grid(n, K)
    shp = (n[2], n[1], n[0])
    rho = np.full(shp, 1e-12)
    RT = np.full(shp, 0.2)  # Nr = 1: refined children
    u = np.zeros((D,) + shp)
    rho[5:7, 5:7, 5:7] = 1.0 + RNG.random((2, 2, 2))
    u[:, 5:7, 5:7, 5:7] = 0.3 * RNG.standard_normal((D, 2, 2, 2))
    M = O.state_from_primitives(g, p, rho, u, RT)
    M1 = O.step(g, p, M)
    Z, Y, X = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    pos = [X.ravel(), Y.ravel(), Z.ravel()]
    for a in range(D):
        before = (pos[a] * M[0]).sum() + M[1 + a].sum()
        after = (pos[a] * M1[0]).sum()
        assert after == pytest.approx(before, rel=1e-12, abs=1e-12)
