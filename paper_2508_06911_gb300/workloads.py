"""Seeded synthetic workloads (primitive fields in lattice units).

This module holds no arithmetic of the LELBM method: it draws initial conditions
(density, velocity, temperature RT), the layout (pads, instance lengths) and the
step counts of the paper's problem classes.  Both the CUDA path and the CPU
oracle convert these fields to moments on their own.  Seeds: 2508069110 + index.

Problem classes (arXiv:2508.06911):
  * 1D two-state Riemann problems (Sec. V.A-B, Sod and Lax), single and batched;
  * 2D four-quadrant Riemann problems (Sec. V.D);
  * the periodic hot box (Sec. IV.E).
Lattice units: dx = 1; an acoustic scaling s maps physical (u, RT) to (s u, s^2 RT)
and the time step to s dx (Sec. V.B, Eq. VIB2), so t_phys needs t_phys N / s steps.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2508069110
GAMMA = 1.4


def rng(index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index))


def internal_dof(gamma: float, dims: int) -> float:
    """K from gamma = (D + K + 2) / (D + K) (App. B, Eq. B22)."""
    return 2.0 / (gamma - 1.0) - dims


# ---------------------------------------------------------------------------
# Exact star state of a 1D Riemann problem (used only to condition the draws:
# reject near-vacuum draws and pick the acoustic scaling from the coldest state).
# ---------------------------------------------------------------------------
def _wave(p, rho, pk, g):
    a = math.sqrt(g * pk / rho)
    if p > pk:
        A, B = 2.0 / ((g + 1) * rho), (g - 1) / (g + 1) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1 - 0.5 * (p - pk) / (p + B))
    e = (g - 1) / (2 * g)
    return 2 * a / (g - 1) * ((p / pk) ** e - 1), (p / pk) ** (-(g + 1) / (2 * g)) / (rho * a)


def star_state(left, right, g=GAMMA):
    """(p*, u*, rho*_L, rho*_R) of the exact solution, or None when vacuum forms."""
    rl, ul, pl = left
    rr, ur, pr = right
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    if 2 * (al + ar) / (g - 1) <= ur - ul:
        return None
    e = (g - 1) / (2 * g)
    p = max(((al + ar - 0.5 * (g - 1) * (ur - ul)) / (al / pl ** e + ar / pr ** e)) ** (1 / e), 1e-14)
    for _ in range(100):
        fl, dl = _wave(p, rl, pl, g)
        fr, dr = _wave(p, rr, pr, g)
        pn = p - (fl + fr + ur - ul) / (dl + dr)
        pn = pn if pn > 0 else 0.5 * p
        if abs(pn - p) < 1e-14 * p:
            p = pn
            break
        p = pn
    fl, _ = _wave(p, rl, pl, g)
    fr, _ = _wave(p, rr, pr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)

    def rho_star(rk, pk):
        if p > pk:
            q = (g - 1) / (g + 1)
            return rk * (p / pk + q) / (q * p / pk + 1)
        return rk * (p / pk) ** (1 / g)

    return p, u, rho_star(rl, pl), rho_star(rr, pr)


def temperature_range(left, right, g=GAMMA):
    """(min, max) of RT = p / rho over the exact solution, and max |u|."""
    st = star_state(left, right, g)
    if st is None:
        return None
    p, u, rsl, rsr = st
    T = [left[2] / left[0], right[2] / right[0], p / rsl, p / rsr]
    return min(T), max(T), max(abs(left[1]), abs(right[1]), abs(u))


def pad_for(umax: float, RTmax: float, n_conf: float = 4.0) -> int:
    """Pad layers wide enough for the longest streaming distance, with margin."""
    return int(math.ceil(umax + n_conf * math.sqrt(RTmax) + 0.5)) + 3


@dataclass
class Riemann1D:
    """A batch of 1D two-state Riemann problems on [0, 1), interface at 0.5."""
    lengths: np.ndarray     # interior cells per instance
    left: np.ndarray        # (n, 3) physical rho, u, p
    right: np.ndarray       # (n, 3)
    scale: np.ndarray       # acoustic scaling s per instance
    steps: np.ndarray       # steps to t_end per instance
    pads: np.ndarray        # pad layers per instance
    t_end: float
    K: float = 4.0
    nu: float = 1e-3
    Pr: float = 0.71
    name: str = ""

    @property
    def n_batch(self) -> int:
        return len(self.lengths)

    def primitives(self, b: int):
        """Lattice-unit (rho, u, RT) of instance b on its interior cells."""
        n = int(self.lengths[b])
        x = (np.arange(n) + 0.5) / n
        s = float(self.scale[b])
        L, R = self.left[b], self.right[b]
        left = x < 0.5
        rho = np.where(left, L[0], R[0])
        u = np.where(left, L[1], R[1]) * s
        RT = np.where(left, L[2] / L[0], R[2] / R[0]) * s * s
        return rho, u, RT

    def padded_fields(self):
        """Concatenated padded fields (rho, u[1][n], RT) in the layout of the C ABI (pads zero)."""
        tot = int(np.sum(self.lengths + 2 * self.pads))
        rho = np.zeros(tot)
        u = np.zeros((1, tot))
        RT = np.zeros(tot)
        off = 0
        for b in range(self.n_batch):
            n, p = int(self.lengths[b]), int(self.pads[b])
            r, uu, T = self.primitives(b)
            rho[off + p: off + p + n] = r
            u[0, off + p: off + p + n] = uu
            RT[off + p: off + p + n] = T
            off += n + 2 * p
        return rho, u, RT


def riemann_1d(n: int = 400, seed_index: int = 0, t_end: float = 0.2) -> Riemann1D:
    """Seeded Sod-like problem: left (rho, p) ~ U[0.5, 1.5], right scaled by 1/8 and 1/10, u = 0."""
    g = rng(seed_index)
    rl, pl = g.uniform(0.5, 1.5, 2)
    left = np.array([[rl, 0.0, pl]])
    right = np.array([[rl / 8.0, 0.0, pl / 10.0]])
    Tmin, Tmax, umax = temperature_range(left[0], right[0])
    pad = pad_for(umax, Tmax * 1.5)
    return Riemann1D(lengths=np.array([n]), left=left, right=right, scale=np.array([1.0]),
                     steps=np.array([int(round(t_end * n))]), pads=np.array([pad]), t_end=t_end,
                     name=f"riemann1d_{n}")


def riemann_1d_batch(n_batch: int = 4096, seed_index: int = 1, t_end: float = 0.15, lmin: int = 256,
                     lmax: int = 4096, RT_floor: float = 0.25) -> Riemann1D:
    """Seeded batch of uneven 1D Riemann problems.

    Lengths log-uniform in [lmin, lmax]; left (rho, p) ~ U[0.5, 1.5]; pressure ratio log-uniform
    in [10, 1000]; density ratio U[1, 10]; u_L, u_R ~ U[-3, 3] times the local sound speed;
    sides swapped at random.  Draws whose exact solution comes near vacuum (minimum temperature
    below a quarter of the colder initial state) are redrawn.  Each instance is scaled
    acoustically so that its coldest exact state sits at lattice RT = RT_floor.
    """
    g = rng(seed_index)
    lengths = np.rint(np.exp(g.uniform(math.log(lmin), math.log(lmax), n_batch))).astype(np.int64)
    left = np.zeros((n_batch, 3))
    right = np.zeros((n_batch, 3))
    scale = np.zeros(n_batch)
    pads = np.zeros(n_batch, dtype=np.int64)
    for b in range(n_batch):
        while True:
            rl, pl = g.uniform(0.5, 1.5, 2)
            ratio = math.exp(g.uniform(math.log(10.0), math.log(1000.0)))
            dratio = g.uniform(1.0, 10.0)
            rr, pr = rl / dratio, pl / ratio
            cl, cr = math.sqrt(GAMMA * pl / rl), math.sqrt(GAMMA * pr / rr)
            ul, ur = g.uniform(-3, 3) * cl, g.uniform(-3, 3) * cr
            L, R = (rl, ul, pl), (rr, ur, pr)
            if g.random() < 0.5:
                L, R = (rr, -ur, pr), (rl, -ul, pl)
            tr = temperature_range(L, R)
            if tr is None:
                continue
            Tmin, Tmax, umax = tr
            if Tmin < 0.25 * min(L[2] / L[0], R[2] / R[0]):
                continue
            break
        left[b], right[b] = L, R
        s = math.sqrt(RT_floor / Tmin)
        scale[b] = s
        pads[b] = pad_for(s * umax, s * s * Tmax * 1.5)
    steps = np.ceil(t_end * lengths / scale).astype(np.int64)
    return Riemann1D(lengths=lengths, left=left, right=right, scale=scale, steps=steps, pads=pads,
                     t_end=t_end, name=f"riemann1d_batch_{n_batch}")


@dataclass
class Grid2D:
    """A 2D problem: interior fields (ny, nx) in lattice units and boundary kinds."""
    nx: int
    ny: int
    rho: np.ndarray
    u: np.ndarray  # (2, ny, nx)
    RT: np.ndarray
    bc: tuple      # x-, x+, y-, y+ : 0 outflow, 1 inflow, 2 periodic
    pad: int
    K: float
    nu: float
    Pr: float
    steps: int
    inlet: tuple = (1.0, 0.0, 0.0, 1.0)
    solid: np.ndarray | None = None  # (ny, nx) uint8 over the interior
    name: str = ""

    def padded(self):
        """Padded (rho, u[2], RT, solid) in the layout of the C ABI."""
        px = 0 if self.bc[0] == 2 else self.pad
        py = 0 if self.bc[2] == 2 else self.pad
        NY, NX = self.ny + 2 * py, self.nx + 2 * px
        rho = np.zeros((NY, NX))
        u = np.zeros((2, NY, NX))
        RT = np.zeros((NY, NX))
        sol = np.zeros((NY, NX), dtype=np.uint8)
        rho[py:py + self.ny, px:px + self.nx] = self.rho
        u[:, py:py + self.ny, px:px + self.nx] = self.u
        RT[py:py + self.ny, px:px + self.nx] = self.RT
        if self.solid is not None:
            sol[py:py + self.ny, px:px + self.nx] = self.solid
        return rho.reshape(-1), u.reshape(2, -1), RT.reshape(-1), sol.reshape(-1)


def riemann_2d(n: int = 1024, seed_index: int = 2, steps: int = 2000, nu: float = 1e-3,
               max_ratio: float = 64.0, RT_floor: float = 0.25) -> Grid2D:
    """Seeded four-quadrant Riemann problem (Sec. V.D generalised): per quadrant rho ~ U[0.1, 1.5],
    (u, v) uniform in the disk of radius 1.5, p ~ U[0.03, 1.5]; draws with RT_max / RT_min above
    max_ratio are redrawn; acoustic scaling puts the coldest quadrant at lattice RT = RT_floor."""
    g = rng(seed_index)
    while True:
        rho_q = g.uniform(0.1, 1.5, 4)
        r = 1.5 * np.sqrt(g.random(4))
        th = g.uniform(0, 2 * np.pi, 4)
        uq, vq = r * np.cos(th), r * np.sin(th)
        p_q = g.uniform(0.03, 1.5, 4)
        T = p_q / rho_q
        if T.max() / T.min() <= max_ratio:
            break
    s = math.sqrt(RT_floor / T.min())
    return _quadrants(n, rho_q, uq * s, vq * s, T * s * s, steps, nu, f"riemann2d_{n}")


def lax_liu_12(n: int = 256, steps: int | None = None, nu: float = 1e-3, scale: float = 1.0) -> Grid2D:
    """Configuration 12 of the 2D Riemann problem (Sec. V.D, Eq. VID1), outflow on all sides."""
    # quadrant order: (x<.5,y<.5), (x>=.5,y<.5), (x<.5,y>=.5), (x>=.5,y>=.5)
    rho = np.array([0.8, 1.0, 1.0, 0.5313])
    u = np.array([0.0, 0.0, 0.7276, 0.0]) * scale
    v = np.array([0.0, 0.7276, 0.0, 0.0]) * scale
    T = np.array([1.0, 1.0, 1.0, 0.4]) / rho * scale * scale
    if steps is None:
        steps = int(round(0.25 * n / scale))
    return _quadrants(n, rho, u, v, T, steps, nu, f"laxliu12_{n}")


def _quadrants(n, rho_q, u_q, v_q, T_q, steps, nu, name) -> Grid2D:
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x)
    q = (X >= 0.5).astype(int) + 2 * (Y >= 0.5).astype(int)
    umax = float(np.max(np.hypot(u_q, v_q)))
    pad = pad_for(umax * 1.3, float(T_q.max()) * 2.0)
    return Grid2D(nx=n, ny=n, rho=rho_q[q], u=np.stack([u_q[q], v_q[q]]), RT=T_q[q], bc=(0, 0, 0, 0),
                  pad=pad, K=internal_dof(GAMMA, 2), nu=nu, Pr=0.71, steps=steps, name=name)


def hot_box(dims: int, n: int, RT: float, u: float = 10.0) -> Grid2D | Riemann1D:
    """Sec. IV.E: periodic, uniform rho = 1, u = (10, 10) (1D: 10), temperature RT."""
    if dims == 1:
        return Riemann1D(lengths=np.array([n]), left=np.array([[1.0, u, RT]]), right=np.array([[1.0, u, RT]]),
                         scale=np.array([1.0]), steps=np.array([1]), pads=np.array([0]), t_end=0.0,
                         K=internal_dof(GAMMA, 1), name=f"hotbox1d_{n}_RT{RT}")
    return Grid2D(nx=n, ny=n, rho=np.ones((n, n)), u=np.full((2, n, n), u), RT=np.full((n, n), RT),
                  bc=(2, 2, 2, 2), pad=0, K=internal_dof(GAMMA, 2), nu=1e-3, Pr=0.71, steps=1,
                  name=f"hotbox2d_{n}_RT{RT}")


@dataclass
class Grid3D:
    """A 3D problem: interior fields (nz, ny, nx) in lattice units and boundary kinds."""
    nx: int
    ny: int
    nz: int
    rho: np.ndarray
    u: np.ndarray  # (3, nz, ny, nx)
    RT: np.ndarray
    bc: tuple      # x-, x+, y-, y+, z-, z+ : 0 outflow, 1 inflow, 2 periodic
    pad: int
    K: float
    nu: float
    Pr: float
    steps: int
    inlet: tuple = (1.0, 0.0, 0.0, 0.0, 1.0)
    name: str = ""

    def padded(self):
        """Padded (rho, u[3], RT) in the layout of the C ABI: cell = (iz NY + iy) NX + ix."""
        px = 0 if self.bc[0] == 2 else self.pad
        py = 0 if self.bc[2] == 2 else self.pad
        pz = 0 if self.bc[4] == 2 else self.pad
        NZ, NY, NX = self.nz + 2 * pz, self.ny + 2 * py, self.nx + 2 * px
        rho = np.zeros((NZ, NY, NX))
        u = np.zeros((3, NZ, NY, NX))
        RT = np.zeros((NZ, NY, NX))
        sl = (slice(pz, pz + self.nz), slice(py, py + self.ny), slice(px, px + self.nx))
        rho[sl] = self.rho
        u[(slice(None),) + sl] = self.u
        RT[sl] = self.RT
        return rho.reshape(-1), u.reshape(3, -1), RT.reshape(-1)


def hot_box_3d(n: int, RT: float, u: float = 10.0) -> Grid3D:
    """Sec. IV.E in three dimensions: periodic n^3 box, rho = 1, u = (10, 10, 10), temperature RT."""
    return Grid3D(nx=n, ny=n, nz=n, rho=np.ones((n, n, n)), u=np.full((3, n, n, n), u), RT=np.full((n, n, n), RT),
                  bc=(2,) * 6, pad=0, K=internal_dof(GAMMA, 3), nu=1e-3, Pr=0.71, steps=1,
                  name=f"hotbox3d_{n}_RT{RT}")


def riemann_3d(n: int = 128, seed_index: int = 6, steps: int = 200, nu: float = 1e-3, max_ratio: float = 8.0,
               RT_floor: float = 0.25, periodic: bool = False) -> Grid3D:
    """Seeded eight-octant Riemann problem, the 3D analogue of riemann_2d: per octant
    rho ~ U[0.1, 1.5], velocity uniform in the ball of radius 1.5, p ~ U[0.03, 1.5]; draws with
    RT_max / RT_min above max_ratio are redrawn (3D velocity sets grow as (4 sqrt RT)^3);
    acoustic scaling puts the coldest octant at lattice RT = RT_floor; outflow on every side
    (periodic: wrap-around instead, no pads)."""
    g = rng(seed_index)
    while True:
        rho_q = g.uniform(0.1, 1.5, 8)
        d = g.standard_normal((8, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        vel = d * (1.5 * g.random(8) ** (1.0 / 3.0))[:, None]
        p_q = g.uniform(0.03, 1.5, 8)
        T = p_q / rho_q
        if T.max() / T.min() <= max_ratio:
            break
    s = math.sqrt(RT_floor / T.min())
    x = (np.arange(n) + 0.5) / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    q = (X >= 0.5).astype(int) + 2 * (Y >= 0.5).astype(int) + 4 * (Z >= 0.5).astype(int)
    vel = vel * s
    T = T * s * s
    umax = float(np.linalg.norm(vel, axis=1).max())
    pad = 0 if periodic else pad_for(umax * 1.3, float(T.max()) * 2.0)
    return Grid3D(nx=n, ny=n, nz=n, rho=rho_q[q], u=np.stack([vel[q, 0], vel[q, 1], vel[q, 2]]), RT=T[q],
                  bc=(2 if periodic else 0,) * 6, pad=pad, K=internal_dof(GAMMA, 3), nu=nu, Pr=0.71, steps=steps,
                  name=f"riemann3d_{n}")


def random_smooth_2d(nx: int, ny: int, seed_index: int, RT_lo: float, RT_hi: float, umag: float,
                     periodic: bool = True, pad: int = 0) -> Grid2D:
    """Random smooth fields for parity tests (a few Fourier modes)."""
    g = rng(seed_index)
    X, Y = np.meshgrid(np.arange(nx) / nx, np.arange(ny) / ny)

    def field():
        f = np.zeros_like(X)
        for _ in range(3):
            kx, ky = g.integers(0, 3, 2)
            f += g.standard_normal() * np.cos(2 * np.pi * (kx * X + ky * Y) + g.uniform(0, 2 * np.pi))
        return f / 3.0

    rho = 1.0 + 0.2 * np.tanh(field())
    RT = RT_lo + (RT_hi - RT_lo) * 0.5 * (1 + np.tanh(field()))
    u = umag * np.stack([field(), field()])
    bc = (2, 2, 2, 2) if periodic else (0, 0, 0, 0)
    umax = float(np.abs(u).max()) * 1.5
    p = 0 if periodic else max(pad, pad_for(umax, RT_hi * 1.5))
    return Grid2D(nx=nx, ny=ny, rho=rho, u=u, RT=RT, bc=bc, pad=p, K=internal_dof(GAMMA, 2), nu=5e-3,
                  Pr=0.71, steps=1, name=f"smooth2d_{nx}x{ny}")


def cylinder_2d(nx: int = 2048, ny: int = 1024, diameter: int = 128, mach: float = 3.0, rho: float = 1.4,
                p: float = 1.0, RT_lattice: float = 0.5, steps: int = 20000) -> Grid2D:
    """Supersonic flow past a circular cylinder with a slip wall (Sec. V.G): inviscid
    (nu = kappa = 0), uniform inflow (rho, p) at the given Mach number on the x- side,
    outflow on the other three, impulsive start (the inflow state everywhere).  The
    cylinder is the set of cells whose centres lie within diameter / 2 of (nx / 4, ny / 2)
    (a legoland mask).  Acoustic scaling puts the free stream at lattice RT_lattice."""
    RT = p / rho
    s = math.sqrt(RT_lattice / RT)
    u_lat = mach * math.sqrt(GAMMA * RT) * s
    xc, yc = (np.arange(nx) + 0.5), (np.arange(ny) + 0.5)
    X, Y = np.meshgrid(xc, yc)
    solid = ((X - nx / 4) ** 2 + (Y - ny / 2) ** 2 <= (diameter / 2) ** 2).astype(np.uint8)
    # stagnation temperature bounds the post-shock temperature
    RT_max = RT_lattice * (1.0 + 0.5 * (GAMMA - 1.0) * mach * mach)
    pad = pad_for(u_lat * 1.3, RT_max * 1.5)
    rho_f = np.full((ny, nx), rho)
    u = np.zeros((2, ny, nx))
    u[0] = u_lat
    RT_f = np.full((ny, nx), RT_lattice)
    return Grid2D(nx=nx, ny=ny, rho=rho_f, u=u, RT=RT_f, bc=(1, 0, 0, 0), pad=pad, K=internal_dof(GAMMA, 2),
                  nu=0.0, Pr=0.71, steps=steps, inlet=(rho, u_lat, 0.0, RT_lattice), solid=solid,
                  name=f"cylinder2d_{nx}x{ny}_D{diameter}_Ma{mach:g}")


def oblique_2d(mach: float, theta_deg: float, nx: int = 512, ny: int = 320, RT: float = 0.5, rho: float = 1.0,
               nu: float = 1e-3, lead: float = 0.1, flow_throughs: float = 2.5) -> Grid2D:
    """Oblique shock (Sec. V.F, Fig. VIF1) in the frame of the deflecting slip wall: a flat
    wall along the bottom of the domain from x = lead * nx on (solid interior row 0), and the
    supersonic stream (rho, RT, Mach number mach) arriving at the angle theta towards it, so
    the wall turns the flow by theta.  Inflow of the stream at x-, y- and y+ (the pads
    below the wall's leading part act as the non-reflective lower boundary), outflow at x+;
    impulsive start; run for flow_throughs passages of the domain length."""
    c_s = math.sqrt(GAMMA * RT)
    V = mach * c_s
    th = math.radians(theta_deg)
    ux, uy = V * math.cos(th), -V * math.sin(th)
    solid = np.zeros((ny, nx), dtype=np.uint8)
    solid[0, int(round(lead * nx)):] = 1
    pad = pad_for(V * 1.3, RT * 1.5)
    steps = int(math.ceil(flow_throughs * nx / ux))
    return Grid2D(nx=nx, ny=ny, rho=np.full((ny, nx), rho), u=np.stack([np.full((ny, nx), ux), np.full((ny, nx), uy)]),
                  RT=np.full((ny, nx), RT), bc=(1, 0, 1, 1), pad=pad, K=internal_dof(GAMMA, 2), nu=nu, Pr=0.71,
                  steps=steps, inlet=(rho, ux, uy, RT), solid=solid,
                  name=f"oblique2d_Ma{mach:g}_theta{theta_deg:g}_{nx}x{ny}")
