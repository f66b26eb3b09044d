"""Exact solution of the 1D Riemann problem of the Euler equations for an ideal gas.

Test-side pin for the oracle (independent of it): the classical construction
with a shock or a rarefaction on each side of a contact (Godunov's exact
solver, as presented in Toro, "Riemann Solvers and Numerical Methods for Fluid
Dynamics", ch. 4).  The star pressure solves f_L(p) + f_R(p) + u_R - u_L = 0;
the solution is then sampled on x/t.  Written from the gas-dynamics relations
(Rankine-Hugoniot across shocks, isentropic Riemann invariants across
rarefactions); the tests check those relations on its output as well.
"""
from __future__ import annotations

import numpy as np


def _fk(p, rho, pk, gamma):
    """Velocity jump across the left/right wave as a function of star pressure, and its derivative."""
    a = np.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        s = np.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (gamma - 1.0) / (2.0 * gamma)  # rarefaction
    return 2.0 * a / (gamma - 1.0) * ((p / pk) ** e - 1.0), (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho * a)


def star_state(left, right, gamma):
    """(p*, u*) for left/right states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    al, ar = np.sqrt(gamma * pl / rl), np.sqrt(gamma * pr / rr)
    if 2.0 * (al + ar) / (gamma - 1.0) <= ur - ul:
        raise ValueError("vacuum is generated")
    # two-rarefaction guess
    e = (gamma - 1.0) / (2.0 * gamma)
    p = ((al + ar - 0.5 * (gamma - 1.0) * (ur - ul)) / (al / pl ** e + ar / pr ** e)) ** (1.0 / e)
    p = max(p, 1e-12)
    for _ in range(200):
        fl, dl = _fk(p, rl, pl, gamma)
        fr, dr = _fk(p, rr, pr, gamma)
        f = fl + fr + ur - ul
        pn = p - f / (dl + dr)
        if pn <= 0:
            pn = 0.5 * p
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, gamma)
    fr, _ = _fk(p, rr, pr, gamma)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, gamma, xi):
    """Exact (rho, u, p) at similarity coordinates xi = (x - x0) / t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    g = gamma
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for i, s in enumerate(xi.flat):
        if s <= us:  # left of the contact
            a = np.sqrt(g * pl / rl)
            if ps > pl:  # left shock
                rs = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
                S = ul - a * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                st = (rl, ul, pl) if s <= S else (rs, us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1 / g)
                ast = a * (ps / pl) ** ((g - 1) / (2 * g))
                if s <= ul - a:
                    st = (rl, ul, pl)
                elif s >= us - ast:
                    st = (rs, us, ps)
                else:
                    uu = 2 / (g + 1) * (a + (g - 1) / 2 * ul + s)
                    rr_ = rl * (2 / (g + 1) + (g - 1) / ((g + 1) * a) * (ul - s)) ** (2 / (g - 1))
                    st = (rr_, uu, pl * (rr_ / rl) ** g)
        else:  # right of the contact
            a = np.sqrt(g * pr / rr)
            if ps > pr:  # right shock
                rs = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
                S = ur + a * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                st = (rr, ur, pr) if s >= S else (rs, us, ps)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1 / g)
                ast = a * (ps / pr) ** ((g - 1) / (2 * g))
                if s >= ur + a:
                    st = (rr, ur, pr)
                elif s <= us + ast:
                    st = (rs, us, ps)
                else:
                    uu = 2 / (g + 1) * (-a + (g - 1) / 2 * ur + s)
                    rr_ = rr * (2 / (g + 1) - (g - 1) / ((g + 1) * a) * (ur - s)) ** (2 / (g - 1))
                    st = (rr_, uu, pr * (rr_ / rr) ** g)
        rho.flat[i], u.flat[i], p.flat[i] = st
    return rho, u, p
