"""Pins of the test-side oblique-shock relations (tests/oblique.py) against the analytical rows
of Table II (Sec. V.F), and against the normal-shock limit."""
import json
import math
import os

import pytest

import oblique as OB

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "oblique_table2.json")))


@pytest.mark.parametrize("case", GOLD["cases"], ids=lambda c: f"Ma{c['Ma1']}-theta{c['theta_deg']}")
def test_table2_analytical_rows(case):
    beta, M2, rr, Tr = OB.post_shock(case["Ma1"], math.radians(case["theta_deg"]), 1.4)
    assert math.degrees(beta) == pytest.approx(case["beta_deg"], abs=6e-4)
    assert M2 == pytest.approx(case["Ma2"], abs=6e-4)
    assert rr == pytest.approx(case["rho_ratio"], abs=6e-4)
    assert Tr == pytest.approx(case["T_ratio"], abs=6e-4)


def test_limits():
    # zero deflection: a Mach wave (beta = asin(1/M)), no jump
    beta, M2, rr, Tr = OB.post_shock(3.0, 1e-9, 1.4)
    assert beta == pytest.approx(math.asin(1 / 3.0), abs=1e-6)
    assert rr == pytest.approx(1.0, abs=1e-6) and Tr == pytest.approx(1.0, abs=1e-6)
    # normal-shock density ratio at beta = 90 degrees: (gamma+1) M^2 / ((gamma-1) M^2 + 2)
    M = 2.5
    assert OB.deflection(math.pi / 2, M, 1.4) == pytest.approx(0.0, abs=1e-12)
    with pytest.raises(ValueError):
        OB.post_shock(2.0, math.radians(30.0), 1.4)  # beyond the maximum deflection at Ma 2 (about 23 degrees)
