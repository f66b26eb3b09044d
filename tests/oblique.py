"""Attached oblique shock on a wedge of an ideal gas (the classical theta-beta-Mach relation).

Test-side reference for the oblique-shock measurements of Sec. V.F: the weak-shock angle beta
for a deflection theta at upstream Mach number M, and the post-shock Mach number, density
ratio and temperature ratio.  Written from the normal-shock (Rankine-Hugoniot) relations
applied to the velocity component normal to the shock; pinned by the analytical rows of the
paper's Table II.
"""
from __future__ import annotations

import math


def deflection(beta: float, M: float, gamma: float) -> float:
    """Flow deflection theta (radians) behind a shock at angle beta (radians)."""
    s2 = (M * math.sin(beta)) ** 2
    return math.atan(2.0 / math.tan(beta) * (s2 - 1.0) / (M * M * (gamma + math.cos(2.0 * beta)) + 2.0))


def weak_beta(theta: float, M: float, gamma: float) -> float:
    """The weak solution beta (radians) for deflection theta (radians), by bisection between
    the Mach angle and the angle of maximum deflection."""
    lo = math.asin(1.0 / M)
    hi = math.pi / 2
    # the angle of maximum deflection bounds the weak branch
    for _ in range(200):
        a, b = lo + (hi - lo) / 3, hi - (hi - lo) / 3
        if deflection(a, M, gamma) < deflection(b, M, gamma):
            lo = a
        else:
            hi = b
    bmax = 0.5 * (lo + hi)
    if theta > deflection(bmax, M, gamma):
        raise ValueError("detached shock")
    lo, hi = math.asin(1.0 / M), bmax
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if deflection(mid, M, gamma) < theta:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def post_shock(M: float, theta: float, gamma: float):
    """(beta, M2, rho2/rho1, T2/T1) for upstream Mach M and deflection theta (radians)."""
    beta = weak_beta(theta, M, gamma)
    mn1 = M * math.sin(beta)
    rho_r = (gamma + 1.0) * mn1 ** 2 / ((gamma - 1.0) * mn1 ** 2 + 2.0)
    p_r = 1.0 + 2.0 * gamma / (gamma + 1.0) * (mn1 ** 2 - 1.0)
    mn2 = math.sqrt((1.0 + 0.5 * (gamma - 1.0) * mn1 ** 2) / (gamma * mn1 ** 2 - 0.5 * (gamma - 1.0)))
    return beta, mn2 / math.sin(beta - theta), rho_r, p_r / rho_r
