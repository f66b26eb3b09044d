"""The 3D LELBM step through the C ABI (the paper's general-D formulation, Sec. II with D = 3:
17 stored moments, 19 fluon and 10 phonon constraints) against the CPU oracle, FP64.

Parity: every moment of every cell within 1e-12 of that moment's largest magnitude after
one and two steps (the FP64 path's per-step bound), on
  - periodic boxes with random smooth states, with and without phonons (K = 2, 0);
  - cold states with one and two refinement levels (RT below 4/9 and below 0.05,
    Eq. IIC9-IIC11: children landing between cells, cloud in cell);
  - padded boxes with outflow and inflow sides (Sec. III.A);
  - the hot box of Sec. IV.E, u = (10, 10, 10), which stays uniform.
Plus the invariants that hold at any size: periodic conservation of mass, momentum and
energy per step, and the integer Galilean shift.
"""
import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L
from paper_2508_06911_gb300.solver import Solver

import oracle as O
from parity_util import assert_close

pytestmark = pytest.mark.gpu
D = 3
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    O.build()


def random_state(shape, seed, RT_lo, RT_hi, umag):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, size=6)
    smooth = lambda k: np.cos(2 * np.pi * x / nx + ph[k]) * np.cos(2 * np.pi * y / ny + ph[k + 1]) * \
        np.cos(2 * np.pi * z / nz + ph[(k + 2) % 6])
    rho = 1.0 + 0.2 * smooth(0) + 0.05 * rng.random(shape)
    RT = RT_lo + (RT_hi - RT_lo) * (0.5 + 0.5 * smooth(1)) * (0.9 + 0.1 * rng.random(shape))
    u = umag * np.stack([smooth(2), smooth(3), smooth(4)]) + 0.1 * umag * rng.standard_normal((3,) + shape)
    return rho, u, RT


def gpu_run(shape, rho, u, RT, K, nsteps, bc=(2, 2, 2, 2, 2, 2), pad=0, inlet=(1.0, 0.0, 0.0, 1.0), nu=5e-3,
            Pr=0.71, padded=None):
    nz, ny, nx = shape
    s = Solver(3, nx, ny, nz=nz, K=K, nu=nu, Pr=Pr, bc=bc, pad=pad, inlet=inlet)
    if padded is None:
        s.set_state(rho.ravel(), u.reshape(3, -1), RT.ravel())
    else:
        s.set_moments(padded)
    out = []
    for _ in range(nsteps):
        s.step(1)
        out.append(s.get_moments())
    st = s.stats()
    status = s.synchronize()
    s.close()
    return out, st, status


def oracle_run(shape, rho, u, RT, K, nsteps, periodic=(True, True, True), pad=0, bc=(0,) * 6,
               inlet=(1.0, 0.0, 0.0, 0.0, 1.0), nu=5e-3, Pr=0.71):
    nz, ny, nx = shape
    g = O.grid(D, nx, ny, nz=nz, periodic=periodic, pad=pad, bc=bc, inlet=inlet)
    p = O.params(D, K, nu_s=nu, Pr=Pr)
    M = O.state_from_primitives(g, p, rho, u, RT)
    st = O.Stats()
    out = []
    for _ in range(nsteps):
        M = O.step(g, p, M, st)
        out.append(M)
    return O.state_from_primitives(g, p, rho, u, RT), out, st


@pytest.mark.parametrize("K", [2.0, 0.0])
def test_periodic_random_state(K):
    shape = (4, 5, 6)
    rho, u, RT = random_state(shape, 31, 0.5, 1.6, 0.6)
    M0, ref, ost = oracle_run(shape, rho, u, RT, K, 2)
    got, st, status = gpu_run(shape, rho, u, RT, K, 2)
    for k in range(2):
        e = assert_close(got[k], ref[k], TOL, f"3D periodic K={K}, step {k + 1}")
        print(f"3D periodic K = {K}, step {k + 1}: max rel {e:.2e}")
    assert status == L.LELBM_OK and st.fallback_mx == 0
    assert st.q_max == ost.q_max and st.q_max > 300


@pytest.mark.parametrize("RT_lo,RT_hi,levels", [(0.2, 0.4, 1), (0.035, 0.045, 2)])
def test_refined_cold_state(RT_lo, RT_hi, levels):
    shape = (4, 4, 5)
    p = O.params(D, 2.0)
    assert O.refine_levels(p, RT_hi) == levels
    rho, u, RT = random_state(shape, 47 + levels, RT_lo, RT_hi, 0.15 if levels == 2 else 0.4)
    _, ref, _ = oracle_run(shape, rho, u, RT, 2.0, 2)
    got, st, status = gpu_run(shape, rho, u, RT, 2.0, 2)
    for k in range(2):
        e = assert_close(got[k], ref[k], TOL, f"3D refined ({levels} levels), step {k + 1}")
        print(f"3D refined, {levels} level(s), step {k + 1}: max rel {e:.2e}")
    assert status == L.LELBM_OK


def test_padded_outflow_and_inflow():
    shape = (4, 5, 6)
    pad = 5
    rho, u, RT = random_state(shape, 53, 0.35, 0.7, 0.3)
    inlet5 = (1.1, 0.3, -0.1, 0.2, 0.5)
    bc = (1, 0, 0, 0, 0, 1)  # inflow at x- and z+, outflow elsewhere
    M0, ref, _ = oracle_run(shape, rho, u, RT, 2.0, 2, periodic=(False, False, False), pad=pad,
                            bc=tuple(1 if b == 1 else 0 for b in bc), inlet=inlet5)
    got, st, status = gpu_run(shape, rho, u, RT, 2.0, 2, bc=bc, pad=pad, inlet=inlet5, padded=M0)
    for k in range(2):
        e = assert_close(got[k], ref[k], TOL, f"3D padded, step {k + 1}")
        print(f"3D padded, step {k + 1}: max rel {e:.2e}")
    assert status == L.LELBM_OK


@pytest.mark.parametrize("RT", [0.5, 2.0])
def test_hot_box_stays_uniform(RT):
    shape = (2, 3, 3)
    rho = np.ones(shape)
    u = np.full((3,) + shape, 10.0)
    T = np.full(shape, RT)
    M0, ref, _ = oracle_run(shape, rho, u, T, 2.0, 2, nu=1e-3)
    got, st, status = gpu_run(shape, rho, u, T, 2.0, 2, nu=1e-3)
    # raw moments at |u| >> sqrt(RT) carry rounding of order eps (|u| / sqrt(RT))^3 relative
    # (the heat-flux moments are differences of terms that large), on both sides alike
    bound = 2 * 4 * np.finfo(float).eps * (10.0 * np.sqrt(D) / np.sqrt(RT)) ** 3 + 1e-14
    assert np.abs(got[1] / M0 - 1).max() < bound
    e = assert_close(got[1], ref[1], max(TOL, bound), f"3D hot box RT={RT}")
    print(f"3D hot box RT = {RT}: max rel vs oracle {e:.2e} (rounding bound {bound:.1e})")
    assert status == L.LELBM_OK


def test_periodic_conservation_and_galilean_shift():
    shape = (6, 6, 6)
    rho, u, RT = random_state(shape, 61, 0.3, 1.0, 0.5)
    got, st, status = gpu_run(shape, rho, u, RT, 2.0, 3)
    M = [O.state_from_primitives(O.grid(D, 6, 6, nz=6, periodic=(True,) * 3), O.params(D, 2.0), rho, u, RT)] + got

    def totals(X):
        t = X.sum(1)
        return t[0], t[1:4], t[4] + t[7] + t[9] + t[13]

    for a, b in zip(M, M[1:]):
        m0, p0, e0 = totals(a)
        m1, p1, e1 = totals(b)
        assert abs(m1 / m0 - 1) < 1e-13
        assert np.abs(p1 - p0).max() / m0 < 1e-13
        assert abs(e1 / e0 - 1) < 1e-13
    U = np.array([1, -2, 1], dtype=float).reshape(3, 1, 1, 1)
    ga, _, _ = gpu_run(shape, rho, u, RT, 2.0, 1)
    gb, _, _ = gpu_run(shape, rho, u + U, RT, 2.0, 1)
    ra = ga[0][0].reshape(shape)
    rb = gb[0][0].reshape(shape)
    np.testing.assert_allclose(rb, np.roll(ra, (1, -2, 1), axis=(0, 1, 2)), rtol=1e-11)
