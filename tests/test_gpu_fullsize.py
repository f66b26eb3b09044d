"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

- The 4096^2 four-quadrant problem (the default bench workload): the mixed path with the
  learned warm start, gated as in the bench.  One step from the seeded state; sampled target
  cells are recomputed one by one from the CPU oracle's single-cell operation
  (oracle.cell_populations: collision, LAS, EPR of each source cell within reach) and the
  moment-streaming rule (Eq. IIE3: a level-0 point lands at x + c, a refined child is shared by
  cloud-in-cell weights).  Within 1e-11 of each moment's largest magnitude over the samples,
  the mixed path's per-step bound.
- The 4096-instance 1D batch: the persistent kernel in its CUDA graph with the autotuned
  launch shape and the learned start, three steps; sampled instances against the oracle run
  instance by instance.
"""
import os

import numpy as np
import pytest

from paper_2508_06911_gb300 import build, lelbm as L, workloads as W
from paper_2508_06911_gb300.solver import Solver

import oracle as O
from parity_util import assert_close, oracle_1d_instance

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MIXED_TOL = 1e-11


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    O.build()


def raw_contribution(c, mf, mg):
    """The 11 stored moments (2D) carried by a population of velocity c (Eq. IIE3)."""
    cx, cy = c
    csq = cx * cx + cy * cy
    return np.array([mf, cx * mf, cy * mf, cx * cx * mf, cx * cy * mf, cy * cy * mf, csq * cx * mf, csq * cy * mf,
                     mg, cx * mg, cy * mg])


def oracle_target(w, p, tx, ty, reach):
    """Moments at interior cell (tx, ty) after one step, summed over every source cell within
    reach, each source's populations from the oracle's single-cell operation."""
    out = np.zeros(11)
    for sy in range(ty - reach, ty + reach + 1):
        for sx in range(tx - reach, tx + reach + 1):
            M = O.eq_moments(2, w.K, w.rho[sy, sx], w.u[:, sy, sx], w.RT[sy, sx])
            co, c, dC, pf, pg, status = O.cell_populations(p, M)
            assert status == 0
            mscale, gscale = co["rho"], co["rho"] * w.K * co["RT"]
            for k in range(len(dC)):
                pos = np.array([sx + c[k, 0], sy + c[k, 1]])
                fl = np.floor(pos)
                w1 = pos - fl
                if abs(pos[0] - tx) >= 1.0 or abs(pos[1] - ty) >= 1.0:
                    continue
                wx = 1.0 - w1[0] if fl[0] == tx else (w1[0] if fl[0] + 1 == tx else 0.0)
                wy = 1.0 - w1[1] if fl[1] == ty else (w1[1] if fl[1] + 1 == ty else 0.0)
                if wx * wy > 0.0:
                    out += wx * wy * raw_contribution(c[k], mscale * pf[k], gscale * pg[k])
    return out


def test_four_quadrant_4096_bench_launch_sampled_against_oracle():
    w = W.riemann_2d(n=4096, seed_index=2)
    weights = np.load(os.path.join(ROOT, "paper_2508_06911_gb300", "weights", "warmstart_2d_quadrants.npy"))
    s = Solver.grid2d(w, precision=L.LELBM_MIXED)
    L.lelbm_set_mlp(s.h, weights)
    L.lelbm_set_mlp_gate(s.h, 1e-3)
    s.step(1)
    M = s.get_moments()
    st = s.stats()
    status = s.synchronize()
    s.close()
    assert status == L.LELBM_OK and st.fallback_mx == 0
    NX = w.nx + 2 * w.pad
    p = O.params(2, w.K, nu_s=w.nu, Pr=w.Pr)
    umax = float(np.abs(w.u).max())
    reach = int(np.ceil(umax + O.acoustic_radius(p, float(w.RT.max())) + 0.5)) + 1
    rng = np.random.default_rng(4096)
    n = w.nx
    # targets across the quadrant interfaces (x, y = n/2), at the centre, and at random
    picks = [(n // 2 + d, n // 3) for d in (-3, -1, 0, 1, 2)] + [(n // 3, n // 2 + d) for d in (-2, 0, 1)]
    picks += [(n // 2 + d, n // 2 + e) for d, e in ((0, 0), (-1, 0), (0, -1), (-1, -1), (2, -3))]
    picks += [tuple(int(v) for v in rng.integers(reach + 1, n - reach - 1, 2)) for _ in range(5)]
    got, ref = [], []
    for tx, ty in picks:
        ref.append(oracle_target(w, p, tx, ty, reach))
        got.append(M[:, (ty + w.pad) * NX + (tx + w.pad)])
    got, ref = np.array(got).T, np.array(ref).T
    e = assert_close(got, ref, MIXED_TOL, "4096^2 four-quadrant, sampled cells, 1 step")
    print(f"4096^2 bench launch, {len(picks)} sampled cells (reach {reach}): max rel {e:.2e}")


def test_batch_4096_bench_launch_sampled_against_oracle():
    w = W.riemann_1d_batch(n_batch=4096, seed_index=1)
    weights = np.load(os.path.join(ROOT, "paper_2508_06911_gb300", "weights", "warmstart_1d.npy"))
    s = Solver.riemann1d(w, precision=L.LELBM_MIXED)
    L.lelbm_set_mlp(s.h, weights)
    s.autotune(1)  # as the bench: tune, then the persistent graph-captured launch
    M0 = s.get_moments()
    s.set_moments(M0)  # the tuner restores the state; start from it explicitly
    s.run_batch(3)
    M = s.get_moments()
    status = s.synchronize()
    rng = np.random.default_rng(11)
    picks = sorted(set(int(b) for b in rng.integers(0, 4096, 16)) | {0, 4095})
    for b in picks:
        first, n = s.instance(b)
        ref = oracle_1d_instance(w, b, 3)
        pad = int(w.pads[b])
        assert_close(M[:, first:first + n], ref[:, pad:pad + n], 3 * MIXED_TOL, f"batch instance {b}, 3 steps")
    s.close()
    assert status == L.LELBM_OK
