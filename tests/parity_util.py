"""Helpers shared by the parity tests: run the CPU oracle on a workload and compare states."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2508_06911_gb300.workloads import Grid2D, Riemann1D


def oracle_params(D, K, nu, Pr, **kw):
    return O.params(D, K, nu_s=nu, Pr=Pr, **kw)


def oracle_1d_instance(w: Riemann1D, b: int, nsteps: int, periodic: bool = False, stats=None, **kw):
    """Oracle state [nmom, n + 2 pad] of instance b after nsteps (same padded layout as the library)."""
    n, pad = int(w.lengths[b]), (0 if periodic else int(w.pads[b]))
    g = O.grid(1, n, periodic=(periodic, False), pad=pad)
    p = oracle_params(1, w.K, w.nu, w.Pr, **kw)
    rho, u, RT = w.primitives(b)
    M = O.state_from_primitives(g, p, rho, u[None, :], RT)
    return O.run(g, p, M, nsteps, stats)


def oracle_2d(w: Grid2D, nsteps: int, stats=None, **kw):
    """Oracle padded state [nmom, NY*NX] after nsteps."""
    g = O.grid(2, w.nx, w.ny, periodic=(w.bc[0] == 2, w.bc[2] == 2), pad=w.pad if (w.bc[0] != 2 or w.bc[2] != 2) else 0,
               bc=tuple(1 if b == 1 else 0 for b in w.bc), inlet=w.inlet,
               solid=w.padded()[3] if w.solid is not None else None)
    p = oracle_params(2, w.K, w.nu, w.Pr, **kw)
    M = O.state_from_primitives(g, p, w.rho, w.u, w.RT)
    return O.run(g, p, M, nsteps, stats)


def oracle_3d(w, nsteps: int, stats=None, **kw):
    """Oracle padded state [nmom, NZ*NY*NX] of a Grid3D after nsteps."""
    periodic = tuple(w.bc[2 * a] == 2 for a in range(3))
    g = O.grid(3, w.nx, w.ny, nz=w.nz, periodic=periodic, pad=0 if all(periodic) else w.pad,
               bc=tuple(1 if b == 1 else 0 for b in w.bc), inlet=w.inlet)
    p = oracle_params(3, w.K, w.nu, w.Pr, **kw)
    M = O.state_from_primitives(g, p, w.rho, w.u, w.RT)
    return O.run(g, p, M, nsteps, stats)


def interior_mask_2d(w: Grid2D):
    px = 0 if w.bc[0] == 2 else w.pad
    py = 0 if w.bc[2] == 2 else w.pad
    NY, NX = w.ny + 2 * py, w.nx + 2 * px
    m = np.zeros((NY, NX), dtype=bool)
    m[py:py + w.ny, px:px + w.nx] = True
    if w.solid is not None:
        m[py:py + w.ny, px:px + w.nx] &= w.solid == 0
    return m.reshape(-1)


def max_rel_err(got: np.ndarray, ref: np.ndarray) -> float:
    """Largest |got - ref| of each moment divided by that moment's largest |ref| (cells = columns)."""
    scale = np.maximum(np.abs(ref).max(axis=1), 1e-300)
    return float((np.abs(got - ref).max(axis=1) / scale).max())


def assert_close(got: np.ndarray, ref: np.ndarray, tol: float, what: str = "") -> float:
    assert np.all(np.isfinite(got)), f"{what}: non-finite values"
    e = max_rel_err(got, ref)
    assert e <= tol, f"{what}: max relative error {e:.3e} > {tol:.1e}"
    return e
