"""The mixed path's double-float building blocks against FP64 on random inputs.

The mixed path (LELBM_MIXED) finishes each EPR solve (Eq. IID7-IID11) on the FP32 pipe
in double-float arithmetic (pairs of FP32 numbers, Dekker 1971): the populations come
from a table-driven 2^w of a fixed-point exponent (Tang 1989), and the residual and the
streamed moments are sums of products in a double-float accumulator (Knuth's TwoSum, the
FMA TwoProduct).  The stated error bounds:
  - 2^w within 2^-46 relative of the exact value;
  - a sum of n products within n 2^-47 of the exact sum, relative to the sum of the
    magnitudes of the products.
The exact references are built here in FP64 and with Python fractions, independent of the
CUDA code.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L

pytestmark = pytest.mark.gpu

FIX = 54  # fractional bits of the fixed-point exponent


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def exact_exp2(w: np.ndarray) -> np.ndarray:
    """2^(w 2^-54) in FP64: the integer part exactly, the fraction (54 bits, rounded to 53)
    through numpy's exp2, so the reference is within about 2^-52 relative."""
    n = w >> FIX
    f = (w - (n << FIX)).astype(np.float64) * 2.0 ** -FIX
    return np.ldexp(np.exp2(f), n.astype(np.int64))


def test_exp2_within_bound():
    rng = np.random.default_rng(46)
    # exponents of the stencils' range: populations between 2^-100 and 2^100, plus the
    # table's breakpoints j/512 and values just below them
    w = rng.integers(-100 << FIX, 100 << FIX, size=200_000, dtype=np.int64)
    grid = (np.arange(-2048, 2048, dtype=np.int64) << (FIX - 9))
    w = np.concatenate([w, grid, grid - 1, grid + 1, np.array([0, 1, -1], dtype=np.int64)])
    got = L.lelbm_df_exp2(w)
    ref = exact_exp2(w)
    rel = np.abs(got / ref - 1.0)
    print(f"double-float 2^w: max rel error {rel.max():.3e} (bound {2.0 ** -46:.3e})")
    assert np.all(np.isfinite(got))
    assert rel.max() <= 2.0 ** -46


def test_exp2_matches_fp64_exp_of_lattice_exponents():
    """The same values the passes produce: 2^(-(1 + lambda . T) log2 e) at the point of a
    Maxwellian-like exponent, against numpy's FP64 exp."""
    rng = np.random.default_rng(7)
    e = rng.uniform(-40.0, 40.0, size=50_000)  # natural-log exponents
    w = np.round(-e * np.log2(np.e) * 2.0 ** FIX).astype(np.int64)
    got = L.lelbm_df_exp2(w)
    ref = exact_exp2(w)
    assert np.abs(got / ref - 1.0).max() <= 2.0 ** -46
    # and the fixed-point rounding of the exponent itself stays far below the 1e-12 judge
    assert np.abs(got / np.exp(-e) - 1.0).max() < 1e-13


@pytest.mark.parametrize("n_terms", [64, 2000])
def test_dot_within_bound(n_terms):
    rng = np.random.default_rng(n_terms)
    rows = 8
    k = rng.uniform(-1, 1, size=(rows, n_terms)).astype(np.float32)
    # populations over many orders of magnitude, signed moment weights (x^a in lattice units)
    v = np.exp(rng.uniform(-30, 5, size=(rows, n_terms))) * rng.choice([-1.0, 1.0], size=(rows, n_terms))
    got = L.lelbm_df_dot(k, v)
    for r in range(rows):
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(k[r], v[r]))
        mag = float(sum(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(k[r], v[r])))
        err = abs(float(Fraction(got[r]) - exact)) / mag
        assert err <= n_terms * 2.0 ** -47, (r, err)


def test_dot_beats_fp32_and_fp64_naive_bound():
    """A cancelling sum (the residual near convergence): the double-float result keeps
    about 2^-47 of the magnitudes, far below what FP32 keeps."""
    rng = np.random.default_rng(3)
    n = 1000
    k = rng.uniform(0.5, 1.5, size=(1, n)).astype(np.float32)
    v = rng.uniform(0.1, 1.0, size=(1, n))
    v[0, n // 2:] = -v[0, : n // 2] * k[0, : n // 2].astype(np.float64) / k[0, n // 2:].astype(np.float64)
    got = L.lelbm_df_dot(k, v)[0]
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(k[0], v[0]))
    mag = float(sum(abs(Fraction(float(a)) * Fraction(float(b))) for a, b in zip(k[0], v[0])))
    assert abs(float(Fraction(got) - exact)) <= n * 2.0 ** -47 * mag
