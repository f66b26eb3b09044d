"""The acoustic scaling of the seeded 1D batch (Eq. VIB2: dt = s dx, so lattice u = s u_phys,
RT = s^2 RT_phys, and t_phys needs t_phys N / s steps) pinned by the exact Riemann solution.

workloads.py applies the scaling before the fields reach either the oracle or the library, so a
mistake in it could not show as a parity failure.  Here instances of the batch generator (each
with its own s, from 1.2 to 3.1) are run by the oracle to their step count, mapped back to
physical units and compared with the exact solution of their physical states at the physical
time reached: the relative L1 density error is a few parts per thousand to 3 %.  Leaving u
unscaled, scaling RT by s instead of s^2, or taking N / s steps with s multiplied instead of
divided raises the mean error four- to fifteen-fold.
"""
import numpy as np

import exact_riemann as ER
import oracle as O
from paper_2508_06911_gb300 import workloads as W
from parity_util import oracle_1d_instance


def test_scaled_instances_reach_the_exact_physical_solution():
    w = W.riemann_1d_batch(n_batch=4, seed_index=77, lmin=900, lmax=1000)
    assert w.scale.min() > 1.1 and w.scale.max() > 3.0  # genuinely scaled instances
    errs = []
    for b in range(w.n_batch):
        n, p, s = int(w.lengths[b]), int(w.pads[b]), float(w.scale[b])
        rho = oracle_1d_instance(w, b, int(w.steps[b]))[0, p:p + n]
        t = int(w.steps[b]) * s / n  # physical time reached: steps x dt, dt = s / n
        x = (np.arange(n) + 0.5) / n
        exact = ER.sample(tuple(w.left[b]), tuple(w.right[b]), W.GAMMA, (x - 0.5) / t)[0]
        errs.append(np.abs(rho - exact).sum() / np.abs(exact).sum())
    print("relative L1 density error per instance:", ", ".join(f"{e:.4f}" for e in errs))
    assert max(errs) < 0.04
    assert np.mean(errs) < 0.02
