"""Pins of the oracle's collision module (Eq. IIB6-IIB18, App. C, App. D) against
closed forms, brute-force moment sums and invariants."""
import itertools

import numpy as np
import pytest

import oracle as O

RNG = np.random.default_rng(2508069110)


def gh_eq_moments(D, K, rho, u, RT, n=12):
    """Equilibrium raw moments by Gauss-Hermite quadrature of the Maxwellian (Eq. IIA3),
    with g = K RT f for the phonons (App. A Eq. A6b, A7) - independent of Eq. (IIB7)."""
    x, w = np.polynomial.hermite.hermgauss(n)
    nodes = np.sqrt(2.0 * RT) * x
    M = np.zeros(O.nmom(D))
    for idx in itertools.product(range(n), repeat=D):
        c = np.array([u[a] + nodes[idx[a]] for a in range(D)])
        wt = rho * np.prod([w[i] for i in idx]) / np.pi ** (D / 2)
        mm = brute_raw(D, c[None, :], np.array([wt]), np.array([K * RT * wt]))
        M += mm
    return M


def brute_raw(D, c, f, g):
    """Raw moments of a discrete population, Eq. (IIB4a), in stored order (Eq. IIB5)."""
    c = np.asarray(c).reshape(-1, D)
    csq = (c ** 2).sum(1)
    out = [f.sum()]
    out += [(c[:, a] * f).sum() for a in range(D)]
    out += [(c[:, a] * c[:, b] * f).sum() for a in range(D) for b in range(a, D)]
    out += [(csq * c[:, g_] * f).sum() for g_ in range(D)]
    out += [g.sum()] + [(c[:, a] * g).sum() for a in range(D)]
    return np.array(out)


def random_population(D, q=40):
    c = RNG.normal(0.3, 1.2, size=(q, D))
    f = RNG.random(q) + 0.05
    g = RNG.random(q) + 0.05
    return c, f, g


@pytest.mark.parametrize("D,K", [(1, 4.0), (2, 3.0), (2, 0.0), (1, 1e6)])
def test_equilibrium_moments_match_quadrature(D, K):
    rho, u, RT = 1.3, np.array([0.7, -1.9])[:D], 0.83
    M = O.eq_moments(D, K, rho, u, RT)
    np.testing.assert_allclose(M, gh_eq_moments(D, K, rho, u, RT), rtol=1e-12, atol=1e-12 * max(1, K))


@pytest.mark.parametrize("D,K", [(1, 4.0), (2, 3.0)])
def test_macros_roundtrip(D, K):
    for _ in range(20):
        rho, u, RT = RNG.uniform(0.1, 3), RNG.normal(0, 5, D), RNG.uniform(0.05, 50)
        r2, u2, RT2 = O.macros(D, K, O.eq_moments(D, K, rho, u, RT))
        assert r2 == pytest.approx(rho, rel=1e-14)
        np.testing.assert_allclose(u2, u, rtol=1e-13, atol=1e-13)
        assert RT2 == pytest.approx(RT, rel=1e-11)


@pytest.mark.parametrize("D,K", [(1, 4.0), (2, 3.0), (2, 1.0)])
def test_neq_central_moments_match_brute_force(D, K):
    """Eq. (IIB9) (cascaded) against the definitions Eq. (IIB4b) and (IIB7e-j) on a discrete population."""
    for _ in range(10):
        c, f, g = random_population(D)
        g = g * K  # phonon moments scale with K
        M = brute_raw(D, c, f, g)
        rho, u, RT = O.macros(D, K, M)
        ct = c - u
        P_ref = np.array([[(ct[:, a] * ct[:, b] * f).sum() - (rho * RT if a == b else 0.0)
                           for b in range(D)] for a in range(D)])
        Q_ref = np.array([((ct ** 2).sum(1) * ct[:, g_] * f).sum() for g_ in range(D)])
        G0n_ref = g.sum() - rho * K * RT
        Gn_ref = np.array([(ct[:, a] * g).sum() for a in range(D)])
        P, Q, G0n, Gn = O.neq(D, K, M)
        sc = max(1.0, np.abs(M).max())
        np.testing.assert_allclose(P, P_ref, atol=1e-12 * sc)
        np.testing.assert_allclose(Q, Q_ref, atol=1e-12 * sc)
        assert G0n == pytest.approx(G0n_ref, abs=1e-12 * sc)
        np.testing.assert_allclose(Gn, Gn_ref, atol=1e-12 * sc)
        # energy: M~neq_aa + G~neq_0 = 0 (Eq. B6c)
        assert np.trace(P) + G0n == pytest.approx(0.0, abs=1e-12 * sc)


def _brute_central(D, K, c, f, g):
    M = brute_raw(D, c, f, g)
    rho, u, RT = O.macros(D, K, M)
    ct = c - u
    Mab = np.array([[(ct[:, a] * ct[:, b] * f).sum() for b in range(D)] for a in range(D)])
    MD = np.array([((ct ** 2).sum(1) * ct[:, g_] * f).sum() for g_ in range(D)])
    return M, rho, u, RT, Mab, MD, g.sum(), np.array([(ct[:, a] * g).sum() for a in range(D)])


@pytest.mark.parametrize("D,K", [(1, 4.0), (2, 3.0)])
def test_collision_without_relaxation_is_identity(D, K):
    """omega -> 0 (infinite viscosities): the post-collision central moments are the
    pre-collision ones (Eq. IIB16 with omega = 0), checked against brute-force sums."""
    p = O.params(D, K, nu_s=1e14, nu_b=1e14, Pr=1.0, limiter=0)
    c, f, g = random_population(D)
    g = g * K
    M, rho, u, RT, Mab, MD, G0, Gg = _brute_central(D, K, c, f, g)
    co = O.collide(p, M)
    assert np.all(co["omega"] < 1e-11)
    cf, cg = co["cf"], co["cg"]
    assert cf[0] == 1.0 and np.all(cf[1:1 + D] == 0.0)
    j = 1 + D
    for a in range(D):
        for b in range(a, D):
            assert cf[j] == pytest.approx(Mab[a, b] / rho, abs=1e-9)
            j += 1
    heat = cf[j:].reshape(D, D)  # [gamma][alpha]
    np.testing.assert_allclose(heat.sum(1), MD / rho, atol=1e-9)
    assert cg[0] == pytest.approx(G0 / (rho * K * RT), abs=1e-9)
    np.testing.assert_allclose(cg[1:1 + D], Gg / (rho * K * RT), atol=1e-9)


@pytest.mark.parametrize("D,K", [(1, 4.0), (2, 3.0), (2, 0.0)])
def test_collision_to_equilibrium_and_reflection(D, K):
    """omega = 1 gives the Maxwellian central moments; omega = 2 reflects the
    non-equilibrium part; energy (D+K) rho RT is kept for any omega (Eq. B5c)."""
    c, f, g = random_population(D)
    g = g * K
    M, rho, u, RT, Mab, MD, G0, Gg = _brute_central(D, K, c, f, g)
    eq = O.collide(O.params(D, K, nu_s=0.0, nu_b=-1.0, Pr=1.0, limiter=0), M)
    p1 = O.params(D, K, nu_s=1e-300, nu_b=-1.0, Pr=1.0, limiter=0)
    # nu_s -> 0: omega_f = omega_h = 2
    assert np.allclose(eq["omega"], [2.0, 1.0, 2.0])
    one = O.collide(O.params(D, K, nu_s=0.5 * RT, nu_b=-1.0, Pr=1.0, limiter=0), M)
    assert np.allclose(one["omega"], [1.0, 1.0, 1.0])
    ref_f = [1.0] + [0.0] * D + [RT if a == b else 0.0 for a in range(D) for b in range(a, D)] + [0.0] * D * D
    np.testing.assert_allclose(one["cf"], ref_f, atol=1e-12)
    if K > 0:
        ref_g = [1.0] + [0.0] * D + [RT if a == b else 0.0 for a in range(D) for b in range(a, D)]
        np.testing.assert_allclose(one["cg"], ref_g, atol=1e-12)
    # reflection: cf - eq = -(identity - eq) with omega_b = 1 killing the bulk part
    ident = O.collide(O.params(D, K, nu_s=1e14, nu_b=-1.0, Pr=1.0, limiter=0), M)
    j0 = 1 + D
    np.testing.assert_allclose(eq["cf"][j0:] - one["cf"][j0:], -(ident["cf"][j0:] - one["cf"][j0:]), atol=1e-9)
    del p1
    for co in (eq, one, ident):
        tr = sum(co["cf"][j] for j in range(j0, j0 + D * (D + 1) // 2)
                 if (j - j0) in ([0] if D == 1 else [0, 2]))
        energy = tr + (K * RT * co["cg"][0] if K > 0 else 0.0)
        assert energy == pytest.approx((D + K) * RT, rel=1e-12)


def test_omega_mapping_limits():
    """Eq. (C7): omega in (0, 2]; nu = 0 -> 2, nu = RT/2 -> 1; Pr = 1 -> omega_h = omega_f;
    omega_b = 1 by default and from nu_b through (2/D - 2/(D+K)) (Eq. C8b)."""
    om = O.omegas(2, 3.0, 0.5, 0.0, -1.0, 0.71)
    assert om[0] == 2.0 and om[1] == 1.0 and om[2] == 2.0
    om = O.omegas(2, 3.0, 0.5, 0.25, -1.0, 1.0)
    assert om[0] == pytest.approx(1.0) and om[2] == pytest.approx(1.0)
    # nu_b = RT (2/D - 2/(D+K)) / 2 gives omega_b = 1
    D, K, RT = 2, 3.0, 0.8
    om = O.omegas(D, K, RT, 1e-3, RT * (2 / D - 2 / (D + K)) * 0.5, 1.0)
    assert om[1] == pytest.approx(1.0)
    # Pr scales (1/omega - 1/2) (Eq. C8a, C8c with C_p of Eq. B22b)
    om = O.omegas(2, 3.0, 0.5, 0.01, -1.0, 0.5)
    assert (1 / om[2] - 0.5) == pytest.approx((1 / om[0] - 0.5) / 0.5)


def test_knudsen_limiter_piecewise():
    """App. D: no change for Kn <= 0.01, equilibrium for Kn >= 0.1, linear in log10 Kn between."""
    w = 1.9
    assert O.limit_omega(0.0, w) == w
    assert O.limit_omega(1e-3, w) == w
    assert O.limit_omega(0.01, w) == pytest.approx(w)
    assert O.limit_omega(10 ** -1.5, w) == pytest.approx(w + (1 - w) * 0.5)
    assert O.limit_omega(0.1, w) == pytest.approx(1.0)
    assert O.limit_omega(3.0, w) == 1.0
    assert O.limit_omega(0.05, 0.5) == pytest.approx(0.5 + 0.5 * (np.log10(0.05) + 2))


def knudsen_of(D, K, M):
    rho, u, RT = O.macros(D, K, M)
    P, Q, G0n, Gn = O.neq(D, K, M)
    return O.knudsen(D, K, rho, RT, P, Q, G0n, Gn)


@pytest.mark.parametrize("D,K", [(1, 4.0), (2, 3.0)])
def test_knudsen_number_is_dimensionless_and_frame_independent(D, K):
    """Eq. (D2) pinned by its dimension, not by its formula.  Dividing every velocity of a
    cell's populations by s is a change of the time unit (the acoustic scaling of Eq. VIB2):
    the internal energy carried by g scales with RT as s^-2, second-order central moments
    as s^-2 and third-order ones as s^-3, and a Knudsen number must not change.  A
    denominator with the wrong power of RT (the two denominators of Eq. D2 swapped, or
    RT^(3/2) written RT) fails.  A common shift of every velocity (Galilean) leaves the
    central moments, and Kn, unchanged."""
    c, f, g = random_population(D)
    k = knudsen_of(D, K, brute_raw(D, c, f, g * K))
    assert k > 1e-3
    for sc in (0.3, 2.5, 11.0):
        assert knudsen_of(D, K, brute_raw(D, c / sc, f, g * K / sc ** 2)) == pytest.approx(k, rel=1e-10)
    U = np.array([3.7, -1.2])[:D]
    assert knudsen_of(D, K, brute_raw(D, c + U, f, g * K)) == pytest.approx(k, rel=1e-9)


@pytest.mark.parametrize("D,K", [(1, 4.0), (2, 3.0)])
def test_knudsen_number_sees_every_nonequilibrium_part(D, K):
    """Each non-equilibrium part of Eq. (D2) alone gives Kn > 0 (a term dropped from the sums
    would give 0 for it): the traceless stress, the heat flux of the fluons, the phonons'
    heat flux, and the bulk mode (energy moved between translational and internal degrees,
    trace of the stress = -G0^neq).  The weight of |G0^neq| against the stress trace in the
    same sum is fixed by reading only (nothing independent of Eq. D2 sets it)."""
    rho, u, RT = 1.1, np.array([0.4, -0.7])[:D], 0.8
    M0 = O.eq_moments(D, K, rho, u, RT)
    iM2 = [2] if D == 1 else [3, 4, 5]
    iMD = [3] if D == 1 else [6, 7]
    iG0, iG1 = (4, [5]) if D == 1 else (8, [9, 10])
    cases = []
    if D == 2:
        M = M0.copy()
        M[4] += 0.05  # xy shear stress
        cases.append(("shear", M))
    M = M0.copy()
    M[iMD[0]] += 0.07  # fluon heat flux
    cases.append(("fluon heat flux", M))
    M = M0.copy()
    M[iG1[0]] += 0.06  # phonon heat flux
    cases.append(("phonon heat flux", M))
    M = M0.copy()  # bulk mode: translational energy up, internal energy down by as much
    for i in iM2[::2] if D == 2 else iM2:
        M[i] += 0.03
    M[iG0] -= 0.03 * D
    cases.append(("bulk", M))
    for name, M in cases:
        assert knudsen_of(D, K, M) > 1e-3, name


@pytest.mark.parametrize("D,K", [(1, 4.0), (2, 3.0)])
def test_knudsen_number_properties(D, K):
    """Eq. (D2): zero at equilibrium, linear in the non-equilibrium part, invariant under rho scaling."""
    M_eq = O.eq_moments(D, K, 1.2, np.array([0.4, -0.3])[:D], 0.9)
    P, Q, G0n, Gn = O.neq(D, K, M_eq)
    assert O.knudsen(D, K, 1.2, 0.9, P, Q, G0n, Gn) < 1e-14
    c, f, g = random_population(D)
    M = brute_raw(D, c, f, g * K)
    rho, u, RT = O.macros(D, K, M)
    P, Q, G0n, Gn = O.neq(D, K, M)
    k1 = O.knudsen(D, K, rho, RT, P, Q, G0n, Gn)
    k2 = O.knudsen(D, K, rho, RT, 2 * P, 2 * Q, 2 * G0n, 2 * Gn)
    assert k2 == pytest.approx(2 * k1, rel=1e-13)
    P3, Q3, G3, Gn3 = O.neq(D, K, 3.0 * M)
    assert O.knudsen(D, K, 3 * rho, RT, P3, Q3, G3, Gn3) == pytest.approx(k1, rel=1e-12)
