"""Pins of the oracle's Lagrangian acoustic stencil (Eq. IIC6, IIC9-IIC11) against the
paper's worked examples (tests/golden/las_examples.json) and closed-form properties."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import exact_riemann as ER

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "las_examples.json")))


def test_fig3_stencil_count_and_courant():
    g = GOLD["fig3"]
    p = O.params(2, 3.0)
    c, dC, lev = O.las(2, g["u"], g["RT"], p)
    assert len(dC) == g["q"]
    assert np.all(lev == 0) and np.all(dC == 1.0)
    R = O.acoustic_radius(p, g["RT"])
    assert R == 9  # [4 sqrt 5] = [8.94]
    # Eq. (IIC7): Co_lat ~ |u| + R_ac
    assert round(math.hypot(*g["u"]) + R, 1) == g["Co_lat"]
    # Eq. (IIC3): the largest |c_i| is within one cell of Eq. (IIC7)'s estimate
    assert abs(np.max(np.hypot(c[:, 0], c[:, 1])) - g["Co_lat"]) < 1.0


def test_fig4_refined_stencil_count():
    g = GOLD["fig4"]
    p = O.params(2, 3.0)
    c, dC, lev = O.las(2, g["u"], g["RT"], p)
    assert len(dC) == g["q"]
    assert O.refine_levels(p, g["RT"]) == 1
    # Eq. (IIC11): each split point becomes 2^D children with dC scaled by 0.5^D,
    # so the total velocity volume equals the level-0 count
    c0, dC0, _ = O.las(2, g["u"], g["RT"], O.params(2, 3.0, max_refine=0))
    assert dC.sum() == pytest.approx(len(dC0), abs=0)
    assert np.all(dC[lev == 1] == 0.25)
    # children sit at +-1/4 around integer parents within 1.5 of u (Eq. IIC10)
    for ci in c[lev == 1]:
        parent = np.round(ci)  # quarter offsets round to the integer parent
        assert np.all(np.abs(ci - parent) == 0.25)
        assert np.hypot(*(parent - np.array(g["u"]))) <= 1.5


def test_refinement_switch_point():
    """N_r = [1/(3 sqrt RT)] switches 0 -> 1 at RT = 4/9 ('RT <~ 0.44', Sec. IV.A)."""
    p = O.params(2, 3.0)
    sw = GOLD["refinement_threshold"]["RT_switch_approx"]
    assert O.refine_levels(p, 4.0 / 9.0 + 1e-9) == 0
    assert O.refine_levels(p, 4.0 / 9.0 - 1e-9) == 1
    assert abs(4.0 / 9.0 - sw) < 0.005


def test_acoustic_radius_formula():
    """R_ac = max([4 sqrt RT], 2) with round-half-away (Eq. IIC6)."""
    p = O.params(1, 4.0)
    for RT, R in [(0.1, 2), (0.39, 2), (0.3907, 3), (1.0, 4), (5.0, 9), (32.0, 23), (100.0, 40)]:
        assert O.acoustic_radius(p, RT) == R, RT


@pytest.mark.parametrize("RT", [0.5, 1.0, 3.3, 10.0, 100.0])
def test_1d_level0_count(RT):
    p = O.params(1, 4.0)
    u = 0.37
    c, dC, lev = O.las(1, [u], RT, p)
    R = O.acoustic_radius(p, RT)
    assert len(dC) == 2 * R + 1
    assert set(c[:, 0].astype(int)) == set(range(math.floor(u - R - 0.5) + 1, math.floor(u + R + 0.5) + 1))


def test_galilean_translation_of_stencil():
    """Adding an integer U to u translates the velocity set by U (Eq. IIC6, IIC10)."""
    p = O.params(2, 3.0)
    for RT in [0.2, 0.7, 4.0]:
        c1, d1, _ = O.las(2, [0.3, -0.2], RT, p)
        c2, d2, _ = O.las(2, [5.3, 2.8], RT, p)
        a = sorted(map(tuple, c1 + np.array([5, 3])))
        b = sorted(map(tuple, c2))
        assert a == b
        assert np.array_equal(np.sort(d1), np.sort(d2))


def test_stencil_count_scales_as_eq_iic8():
    """q ~ (n sqrt RT)^D for high temperature (Eq. IIC8): disk area pi (R+1/2)^2."""
    p = O.params(2, 3.0)
    for RT in [8.0, 32.0]:
        c, dC, _ = O.las(2, [0.1, 0.2], RT, p)
        R = O.acoustic_radius(p, RT)
        assert abs(len(dC) / (math.pi * (R + 0.5) ** 2) - 1) < 0.05


def test_lax_lattice_courant_numbers():
    """Sec. V.B: maximum lattice temperature 7.93 (3.30 scaled) and Co_lat 12.5 (8 scaled)."""
    g = GOLD["lax"]
    p = O.params(1, 4.0)
    xi = np.linspace(-10, 10, 40001)
    r, u, pr = ER.sample(tuple(g["left"]), tuple(g["right"]), 1.4, xi)
    RT = pr / r
    for s, co_ref, rt_ref in [(1.0, g["Co_lat_unscaled"], g["RT_max_unscaled"]),
                              (1.0 / g["scale"], g["Co_lat_scaled"], g["RT_max_scaled"])]:
        assert round(RT.max() * s * s, 2) == pytest.approx(rt_ref, abs=0.006)
        co = max(abs(a) * s + O.acoustic_radius(p, b * s * s) for a, b in zip(u, RT))
        assert round(co, 1) == pytest.approx(co_ref, abs=0.051)
