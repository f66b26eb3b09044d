"""Transport laws of Sec. IV through the CUDA path (C ABI), on the FP64 and mixed paths.

- Shear-wave decay (Sec. IV.A, Eq. VA1-VA4): a transverse velocity wave decays at nu k^2,
  within the paper's +-10 % of the imposed shear viscosity (App. C, Eq. C7-C8).
- Thermal-wave decay (Sec. IV.B, Eq. VB1-VB3): a density wave at constant pressure decays
  at alpha k^2 with alpha = nu / Pr, within +-10 %.
- Acoustic pulse (Sec. IV.D, Eq. VD1): a small density pulse travels at sqrt(gamma RT),
  gamma = (D + K + 2) / (D + K) (App. B, Eq. B22), within 2 %, for K = 0, 2, 4.
Each measured coefficient is also compared with the CPU oracle's on the same set-up.
"""
import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L
from paper_2508_06911_gb300.solver import Solver

import oracle as O

pytestmark = pytest.mark.gpu

PATHS = {"fp64": L.LELBM_FP64, "mixed": L.LELBM_MIXED}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    O.build()


def wave_setup(kind, RT, L_, amp):
    x = np.arange(L_) + 0.5
    k = 2 * np.pi / L_
    if kind == "shear":  # Eq. (VA1), u0 = 0
        rho = np.ones(L_)
        u = np.stack([np.zeros(L_), amp * np.cos(k * x)])
        T = np.full(L_, RT)
    else:  # Eq. (VB1), u0 = 0: constant pressure rho RT
        rho = 1.0 + amp * np.cos(k * x)
        u = np.zeros((2, L_))
        T = RT / rho
    return rho, u, T, k


def decay_rate(kind, M, amp, k, nsteps):
    if kind == "shear":
        a = np.abs(M[2] / M[0]).max()  # Eq. (VA4)
    else:
        a = np.abs(M[0] - 1.0).max()  # Eq. (VB3)
    return -np.log(a / amp) / (k * k * nsteps)


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("kind", ["shear", "thermal"])
def test_wave_decay(kind, path):
    nu, RT, L_, amp = 0.1, 0.5, 32, 1e-3
    K = 3.0 if kind == "shear" else 0.0
    rho, u, T, k = wave_setup(kind, RT, L_, amp)
    nsteps = int(round(1.0 / (nu * k * k)))
    s = Solver(2, L_, 1, K=K, nu=nu, Pr=1.0, bc=(2, 2, 2, 2), limiter=0, precision=PATHS[path])
    s.set_state(rho, u, T)
    s.step(nsteps)
    M = s.get_moments()
    st = s.stats()
    s.close()
    meas = decay_rate(kind, M, amp, k, nsteps)
    g = O.grid(2, L_, 1, periodic=(True, True))
    p = O.params(2, K, nu_s=nu, Pr=1.0, limiter=0)
    ref = O.run(g, p, O.state_from_primitives(g, p, rho[None], u[:, None], T[None]), nsteps)
    meas_o = decay_rate(kind, ref, amp, k, nsteps)
    print(f"{kind} wave, {path}: nu_meas/nu = {meas / nu:.4f} (oracle {meas_o / nu:.4f})")
    assert abs(meas / nu - 1) < 0.10
    assert meas == pytest.approx(meas_o, rel=1e-6)
    assert st.fallback_mx == 0


def pulse_position(D, K, M, RT, N):
    rho = M[0]
    x = np.arange(N) + 0.5
    ux = M[1] / rho
    # RT from Eq. (IIB6): ((trace M2 + G0)/rho - |u|^2) / (D + K)
    if D == 1:
        tr, g0 = M[2], M[4]
    else:
        tr, g0 = M[3] + M[5], M[8]
    T = ((tr + g0) / rho - ux * ux) / (D + K)
    pr = rho * T - RT
    half = pr[N // 2:]
    i = int(np.argmax(half))
    y0, y1, y2 = half[i - 1], half[i], half[i + 1]
    return x[N // 2 + i] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)


@pytest.mark.parametrize("path", sorted(PATHS))
@pytest.mark.parametrize("K", [0.0, 2.0, 4.0])
def test_sound_speed_from_acoustic_pulse(K, path):
    D, N, RT, nsteps = 1, 240, 1.0, 60
    x = np.arange(N) + 0.5
    x0 = N / 2
    rho = 1.0 + 1e-6 * np.exp(-((x - x0) / 4.0) ** 2)
    s = Solver(1, N, 1, K=K, nu=1e-3, Pr=1.0, bc=(2, 2, 2, 2), precision=PATHS[path])
    s.set_state(rho, np.zeros((1, N)), np.full(N, RT))
    s.step(nsteps)
    M = s.get_moments()
    s.close()
    cs = (pulse_position(D, K, M, RT, N) - x0) / nsteps
    gamma = (D + K + 2) / (D + K)
    g = O.grid(D, N, periodic=(True, True))
    p = O.params(D, K, nu_s=1e-3, Pr=1.0)
    ref = O.run(g, p, O.state_from_primitives(g, p, rho, np.zeros((1, N)), np.full(N, RT)), nsteps)
    cs_o = (pulse_position(D, K, ref, RT, N) - x0) / nsteps
    print(f"K = {K}, {path}: c_s = {cs:.5f}, sqrt(gamma RT) = {np.sqrt(gamma * RT):.5f}, oracle {cs_o:.5f}")
    assert cs == pytest.approx(np.sqrt(gamma * RT), rel=0.02)
    assert cs == pytest.approx(cs_o, rel=1e-6)
