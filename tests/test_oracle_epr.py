"""Pins of the oracle's entropic population reconstruction (Eq. IID7-IID13)."""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle as O

RNG = np.random.default_rng(7)


def monomials(D, kind, ct):
    """The constraint basis written out by hand: fluons 1, c, cc, c_a^2 c_g; phonons 1, c, cc."""
    ct = np.atleast_2d(ct)
    if D == 1:
        x = ct[:, 0]
        cols = [np.ones_like(x), x, x * x] + ([x ** 3] if kind == 0 else [])
    else:
        x, y = ct[:, 0], ct[:, 1]
        cols = [np.ones_like(x), x, y, x * x, x * y, y * y]
        if kind == 0:
            cols += [x ** 3, y * y * x, x * x * y, y ** 3]
    return np.stack(cols, 1)


def dual_solution(D, kind, c, dC, u, con, lam0):
    """Brute force: minimise the convex dual sum_i dC_i exp(-1 - lam.T_i) + lam.con (scipy)."""
    T = monomials(D, kind, c - u)

    def fun(l):
        w = dC * np.exp(-1.0 - T @ l)
        return w.sum() + l @ con, -(T * w[:, None]).sum(0) + con, (T.T * w) @ T

    res = minimize(lambda l: fun(l)[0], lam0, jac=lambda l: fun(l)[1], hess=lambda l: fun(l)[2],
                   method="trust-exact", options=dict(gtol=1e-13, maxiter=500))
    return res.x


CASES = [(1, 0, 0.6, [0.31]), (1, 1, 0.6, [0.31]), (1, 0, 0.3, [-1.4]), (2, 0, 0.25, [0.2, -0.35]),
         (2, 1, 0.25, [0.2, -0.35]), (2, 0, 0.9, [1.3, 0.45])]


@pytest.mark.parametrize("D,kind,RT,u", CASES)
def test_epr_matches_convex_dual_minimiser(D, kind, RT, u):
    p = O.params(D, 3.0)
    c, dC, _ = O.las(D, u, RT, p)
    u = np.array(u)
    # constraints: Maxwellian moments perturbed by a small non-equilibrium part
    lam_t = O.maxwell_lambda(D, kind, RT)
    lam_t = lam_t + 0.05 * RNG.standard_normal(len(lam_t)) / np.maximum(1, np.arange(len(lam_t)))
    T = monomials(D, kind, c - u)
    con = T.T @ (dC * np.exp(-1 - T @ lam_t))
    con[0] = 1.0 if kind == 0 else con[0]
    st, lam, pop = O.epr(D, kind, c, dC, u, RT, con, p)
    assert st >= 0
    ref = dual_solution(D, kind, c, dC, u, con, O.maxwell_lambda(D, kind, RT))
    np.testing.assert_allclose(lam, ref, rtol=1e-7, atol=1e-7)
    np.testing.assert_allclose(pop, dC * np.exp(-1 - T @ ref), rtol=1e-7)
    assert np.all(pop > 0)  # positivity (exponential form, Sec. II.D)
    assert np.all(np.abs(T.T @ pop - con) <= 1e-12 * np.maximum(1, np.abs(con)))


@pytest.mark.parametrize("D,kind,RT", [(1, 0, 2.0), (2, 0, 1.1), (2, 1, 0.4), (1, 1, 30.0)])
def test_epr_recovers_planted_multipliers(D, kind, RT):
    """Constraints generated from known multipliers are solved back to them (unique dual optimum)."""
    p = O.params(D, 3.0)
    u = RNG.normal(0, 2, D)
    c, dC, _ = O.las(D, u, RT, p)
    lam_t = O.maxwell_lambda(D, kind, RT) * (1 + 0.1 * RNG.standard_normal())
    lam_t[1:1 + D] += 0.1 * RNG.standard_normal(D) / np.sqrt(RT)
    T = monomials(D, kind, c - u)
    con = T.T @ (dC * np.exp(-1 - T @ lam_t))
    st, lam, pop = O.epr(D, kind, c, dC, u, RT, con, p)
    assert st >= 0
    np.testing.assert_allclose(lam, lam_t, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("D,RT", [(1, 20.0), (1, 100.0), (2, 8.0), (2, 32.0)])
def test_maxwellian_start_is_near_solution_on_wide_stencils(D, RT):
    """Eq. (IID12)-(IID13): on a well-resolved stencil the Maxwellian multipliers almost satisfy
    the equilibrium constraints, and Newton needs few updates (Sec. II.D: 'less than five')."""
    p = O.params(D, 3.0)
    u = np.array([0.37, -0.61])[:D]
    c, dC, _ = O.las(D, u, RT, p)
    for kind in (0, 1):
        lam0 = O.maxwell_lambda(D, kind, RT)
        T = monomials(D, kind, c - u)
        m = T.T @ (dC * np.exp(-1 - T @ lam0))
        n2 = D * (D + 1) // 2
        con = np.zeros(len(lam0))
        con[0] = 1.0
        j = 1 + D
        for a in range(D):
            for b in range(a, D):
                con[j] = RT if a == b else 0.0
                j += 1
        # n = 4 keeps 99.99% of the Gaussian mass (Sec. II.C); the truncated tail
        # costs the second moment a few 1e-4 relative
        # (in 2D the mass outside radius r is exp(-r^2 / 2RT), a few 1e-4)
        assert abs(m[0] - 1.0) < (1e-4 if D == 1 else 5e-4)
        assert np.abs(m - con)[1: 1 + D].max() < 1e-4 * np.sqrt(RT)
        assert np.abs(m - con)[1 + D: 1 + D + n2].max() < (2e-3 if D == 1 else 5e-3) * RT
        st, lam, pop = O.epr(D, kind, c, dC, u, RT, con, p)
        assert 1 <= st < 5


def test_cholesky_solve_matches_numpy():
    for n in (3, 4, 6, 10):
        B = RNG.standard_normal((n, n))
        A = B @ B.T + n * np.eye(n)
        b = RNG.standard_normal(n)
        AA, bb = A.copy(), b.copy()
        assert O.lib().orc_cholesky_solve(n, O._dp(AA), O._dp(bb)) == 0
        np.testing.assert_allclose(bb, np.linalg.solve(A, b), rtol=1e-12)
    A = -np.eye(3)
    assert O.lib().orc_cholesky_solve(3, O._dp(A), O._dp(np.ones(3))) == -1


def test_infeasible_constraints_fail():
    """A negative second moment has no positive population: the solve must report failure."""
    p = O.params(1, 4.0, max_iter=30)
    c, dC, _ = O.las(1, [0.2], 0.7, p)
    st, _, _ = O.epr(1, 0, c, dC, [0.2], 0.7, np.array([1.0, 0.0, -0.1, 0.0]), p)
    assert st < 0
