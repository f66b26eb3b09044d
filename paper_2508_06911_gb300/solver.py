"""A small object wrapper over the C ABI (marshalling only; the work runs in liblelbm.so)."""
from __future__ import annotations

import numpy as np

from . import lelbm as L
from .workloads import Grid2D, Grid3D, Riemann1D


class Solver:
    """One LELBM handle.  Fields use the padded layout documented in include/lelbm.h."""

    def __init__(self, dims: int, nx: int, ny: int = 1, *, K: float, nu: float, Pr: float = 0.71,
                 nu_bulk: float = -1.0, bc=(2, 2, 2, 2), pad: int = 0, lengths=None, pads=None, solid=None,
                 inlet=(1.0, 0.0, 0.0, 1.0), limiter: int = 1, stream: int | None = None, nz: int = 1,
                 **numerics):
        """bc: per side (x-, x+, y-, y+[, z-, z+]); inlet: (rho, ux, uy, RT) or, in 3D,
        (rho, ux, uy, uz, RT)."""
        p = L.lelbm_default_params()
        p.dims, p.nx, p.ny, p.nz = dims, nx, ny, nz
        for i in range(4):
            p.bc[i] = bc[i]
        if len(bc) == 6:
            p.bc_z[0], p.bc_z[1] = bc[4], bc[5]
        if len(inlet) == 5:
            p.inlet[0], p.inlet[1], p.inlet[2], p.inlet_uz, p.inlet[3] = inlet
        else:
            for i in range(4):
                p.inlet[i] = inlet[i]
        p.pad = pad
        p.K, p.nu_shear, p.nu_bulk, p.prandtl, p.limiter = K, nu, nu_bulk, Pr, limiter
        for k, v in numerics.items():
            setattr(p, k, v)
        p.stream = stream
        self.dims = dims
        self.h = L.lelbm_create(p, lengths=lengths, pads=pads, solid=solid)
        self.n_cells, self.n_mom, self.NX, self.NY = L.lelbm_layout(self.h)

    @classmethod
    def riemann1d(cls, w: Riemann1D, stream=None, **numerics) -> "Solver":
        s = cls(1, int(w.lengths[0]), 1, K=w.K, nu=w.nu, Pr=w.Pr, bc=(0, 0, 2, 2), pad=int(w.pads[0]),
                lengths=w.lengths if w.n_batch > 1 else None, pads=w.pads if w.n_batch > 1 else None,
                stream=stream, **numerics)
        rho, u, RT = w.padded_fields()
        s.set_state(rho, u, RT)
        return s

    @classmethod
    def grid2d(cls, w: Grid2D, stream=None, **numerics) -> "Solver":
        rho, u, RT, solid = w.padded()
        s = cls(2, w.nx, w.ny, K=w.K, nu=w.nu, Pr=w.Pr, bc=w.bc, pad=w.pad if w.bc[0] != 2 or w.bc[2] != 2 else 0,
                solid=solid if w.solid is not None else None, inlet=w.inlet, stream=stream, **numerics)
        s.set_state(rho, u, RT)
        return s

    @classmethod
    def grid3d(cls, w: Grid3D, stream=None, **numerics) -> "Solver":
        rho, u, RT = w.padded()
        periodic = all(b == 2 for b in w.bc)
        s = cls(3, w.nx, w.ny, nz=w.nz, K=w.K, nu=w.nu, Pr=w.Pr, bc=w.bc, pad=0 if periodic else w.pad,
                inlet=w.inlet, stream=stream, **numerics)
        s.set_state(rho, u, RT)
        return s

    def set_state(self, rho, u, RT) -> None:
        L.lelbm_set_state(self.h, np.ascontiguousarray(rho, dtype=np.float64),
                          np.ascontiguousarray(u, dtype=np.float64).reshape(self.dims, -1),
                          np.ascontiguousarray(RT, dtype=np.float64))

    def set_moments(self, M) -> None:
        L.lelbm_set_moments(self.h, np.ascontiguousarray(M, dtype=np.float64).reshape(self.n_mom, self.n_cells))

    def get_moments(self) -> np.ndarray:
        out = np.empty((self.n_mom, self.n_cells))
        return L.lelbm_get_moments(self.h, out)

    def macros(self):
        rho, u, RT = np.empty(self.n_cells), np.empty((self.dims, self.n_cells)), np.empty(self.n_cells)
        L.lelbm_get_macros(self.h, rho, u, RT)
        return rho, u, RT

    def step(self, n: int = 1) -> None:
        L.lelbm_step(self.h, n)

    def run_batch(self, n: int) -> None:
        """n steps of every 1D instance in one persistent launch (CUDA graph)."""
        L.lelbm_run_batch(self.h, n)

    def set_steps(self, steps) -> None:
        L.lelbm_set_steps(self.h, steps)

    def set_warmstart(self, stored: bool) -> None:
        """Start each EPR solve from the multipliers the cell kept from its last step."""
        L.lelbm_set_warmstart(self.h, stored)

    def autotune(self, trial_steps: int = 1):
        return L.lelbm_autotune(self.h, trial_steps)

    def synchronize(self) -> int:
        return L.lelbm_synchronize(self.h)

    def stats(self) -> L.lelbm_stats:
        return L.lelbm_get_stats(self.h)

    def instance(self, b: int):
        return L.lelbm_instance(self.h, b)

    def close(self) -> None:
        if self.h:
            L.lelbm_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
