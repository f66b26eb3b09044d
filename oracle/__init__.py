"""Plain FP64 CPU oracle of the LELBM per-timestep cell update (arXiv:2508.06911).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the timed
CPU baseline of ``bench.py`` import this package.  It shares no code with the
CUDA library: the arithmetic lives in ``lelbm_oracle.c`` (plain C, FP64,
compiled without FMA contraction); this module only builds that file with gcc
and marshals numpy arrays through ctypes.

Every C function cites the equation of the paper it follows; see the header
comment of ``lelbm_oracle.c``, which lists the parts without an independent pin
("parity unpinned"; each is marked again at its function).  ``mlp.py`` (the
FP64 network of the learned warm start) is pinned by calculus only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lelbm_oracle.c")
_SO = os.path.join(_HERE, "liblelbm_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liblelbm_oracle.so`` (gcc, no FMA contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [
        ("D", ctypes.c_int),
        ("K", ctypes.c_double),
        ("nu_s", ctypes.c_double),
        ("nu_b", ctypes.c_double),
        ("Pr", ctypes.c_double),
        ("limiter", ctypes.c_int),
        ("n_conf", ctypes.c_double),
        ("r_min", ctypes.c_double),
        ("refine_div", ctypes.c_double),
        ("refine_rad", ctypes.c_double),
        ("max_refine", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
    ]


class Collision(ctypes.Structure):
    _fields_ = [
        ("rho", ctypes.c_double),
        ("u", ctypes.c_double * 3),
        ("RT", ctypes.c_double),
        ("cf", ctypes.c_double * 19),
        ("cg", ctypes.c_double * 10),
        ("omega", ctypes.c_double * 3),
        ("Kn", ctypes.c_double),
    ]


class Point(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double * 3), ("dC", ctypes.c_double), ("level", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [
        ("cells", ctypes.c_longlong),
        ("newton_hist", ctypes.c_longlong * 64),
        ("fallback_eq", ctypes.c_longlong),
        ("fallback_mx", ctypes.c_longlong),
        ("q_max", ctypes.c_longlong),
        ("disp_max", ctypes.c_double),
        ("wall_hits", ctypes.c_longlong),
    ]


class Grid(ctypes.Structure):
    _fields_ = [
        ("D", ctypes.c_int),
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("pad", ctypes.c_int),
        ("bc", ctypes.c_int * 6),
        ("inlet", ctypes.c_double * 5),
        ("solid", ctypes.POINTER(ctypes.c_ubyte)),
        ("wall_u", ctypes.c_double * 2),
    ]


_DP = ctypes.POINTER(ctypes.c_double)


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.orc_eq_moments.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _DP, ctypes.c_double, _DP]
            L.orc_macros.argtypes = [ctypes.c_int, ctypes.c_double, _DP, _DP, _DP, _DP]
            L.orc_neq.argtypes = [ctypes.c_int, ctypes.c_double, _DP, ctypes.c_double, _DP, ctypes.c_double,
                                  _DP, _DP, _DP, _DP]
            L.orc_omegas.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, _DP]
            L.orc_knudsen.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      _DP, _DP, ctypes.c_double, _DP]
            L.orc_knudsen.restype = ctypes.c_double
            L.orc_limit_omega.argtypes = [ctypes.c_double, ctypes.c_double]
            L.orc_limit_omega.restype = ctypes.c_double
            L.orc_collide.argtypes = [ctypes.POINTER(Params), _DP, ctypes.POINTER(Collision)]
            L.orc_acoustic_radius.argtypes = [ctypes.POINTER(Params), ctypes.c_double]
            L.orc_refine_levels.argtypes = [ctypes.POINTER(Params), ctypes.c_double]
            L.orc_las.argtypes = [ctypes.c_int, _DP, ctypes.c_double, ctypes.POINTER(Params),
                                  ctypes.POINTER(Point), ctypes.c_int]
            L.orc_basis_f.argtypes = [ctypes.c_int, _DP, _DP, ctypes.POINTER(ctypes.c_int)]
            L.orc_basis_g.argtypes = [ctypes.c_int, _DP, _DP, ctypes.POINTER(ctypes.c_int)]
            L.orc_cholesky_solve.argtypes = [ctypes.c_int, _DP, _DP]
            L.orc_maxwell_lambda.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _DP]
            L.orc_epr.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Point), _DP,
                                  ctypes.c_double, _DP, ctypes.POINTER(Params), _DP, _DP]
            L.orc_cell_populations.argtypes = [ctypes.POINTER(Params), _DP, ctypes.POINTER(Collision),
                                               ctypes.POINTER(Point), _DP, _DP, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int)]
            L.orc_fill_pads.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Params), _DP]
            L.orc_trace_path.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, _DP, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), _DP, _DP]
            L.orc_step.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Params), _DP, _DP,
                                   ctypes.POINTER(Stats)]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def nmom(D: int) -> int:
    return 2 + 3 * D + D * (D + 1) // 2


def nf(D: int) -> int:
    return 1 + D + D * (D + 1) // 2 + D * D


def ng(D: int) -> int:
    return 1 + D + D * (D + 1) // 2


def params(D: int, K: float, nu_s: float = 1e-3, nu_b: float = -1.0, Pr: float = 0.71,
           limiter: int = 1, n_conf: float = 4.0, r_min: float = 2.0, refine_div: float = 3.0,
           refine_rad: float = 3.0, max_refine: int = 4, tol: float = 1e-12, max_iter: int = 50) -> Params:
    """Physical and numerical parameters (defaults: the paper's constants, Sec. II.C-D, App. D)."""
    return Params(D, K, nu_s, nu_b, Pr, limiter, n_conf, r_min, refine_div, refine_rad, max_refine,
                  tol, max_iter)


def eq_moments(D, K, rho, u, RT) -> np.ndarray:
    """Equilibrium raw moments, Eq. (IIB7) with App. A Eq. (A3), (A7)."""
    out = np.zeros(nmom(D))
    uu = np.zeros(3)
    uu[:D] = np.asarray(u, dtype=np.float64).reshape(-1)[:D]
    lib().orc_eq_moments(D, K, rho, _dp(uu), RT, _dp(out))
    return out


def macros(D, K, M):
    """Density, velocity, temperature, Eq. (IIB6)."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    rho, RT = ctypes.c_double(), ctypes.c_double()
    u = np.zeros(3)
    lib().orc_macros(D, K, _dp(M), ctypes.byref(rho), _dp(u), ctypes.byref(RT))
    return rho.value, u[:D].copy(), RT.value


def neq(D, K, M):
    """Non-equilibrium central moments, Eq. (IIB9): (P[D,D], Q[D], G0n, Gn[D])."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    rho, u, RT = macros(D, K, M)
    uu = np.zeros(3)
    uu[:D] = u
    P, Q, Gn = np.zeros(9), np.zeros(3), np.zeros(3)
    G0n = ctypes.c_double()
    lib().orc_neq(D, K, _dp(M), rho, _dp(uu), RT, _dp(P), _dp(Q), ctypes.byref(G0n), _dp(Gn))
    return P.reshape(3, 3)[:D, :D].copy(), Q[:D].copy(), G0n.value, Gn[:D].copy()


def omegas(D, K, RT, nu_s, nu_b, Pr) -> np.ndarray:
    """(omega_f, omega_b, omega_h) from App. C Eq. (C7)-(C8)."""
    om = np.zeros(3)
    lib().orc_omegas(D, K, RT, nu_s, nu_b, Pr, _dp(om))
    return om


def knudsen(D, K, rho, RT, P, Q, G0n, Gn) -> float:
    """Local Knudsen number, App. D Eq. (D2)."""
    PP = np.zeros(9)
    PP.reshape(3, 3)[:D, :D] = P
    QQ, GG = np.zeros(3), np.zeros(3)
    QQ[:D] = Q
    GG[:D] = Gn
    return lib().orc_knudsen(D, K, rho, RT, _dp(PP), _dp(QQ), G0n, _dp(GG))


def limit_omega(Kn, omega) -> float:
    """Knudsen limiter, App. D Eq. (D3)."""
    return lib().orc_limit_omega(Kn, omega)


def collide(p: Params, M) -> dict:
    """Collision module: macros, limited omegas and normalised post-collision constraints."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    co = Collision()
    lib().orc_collide(ctypes.byref(p), _dp(M), ctypes.byref(co))
    D = p.D
    return dict(rho=co.rho, u=np.array(co.u[:D]), RT=co.RT, cf=np.array(co.cf[:nf(D)]),
                cg=np.array(co.cg[:ng(D)]), omega=np.array(co.omega[:]), Kn=co.Kn)


def acoustic_radius(p: Params, RT: float) -> int:
    """R_ac of Eq. (IIC6)."""
    return lib().orc_acoustic_radius(ctypes.byref(p), RT)


def refine_levels(p: Params, RT: float) -> int:
    """N_r of Eq. (IIC9)."""
    return lib().orc_refine_levels(ctypes.byref(p), RT)


def las(D, u, RT, p: Params):
    """LAS velocity set: (c[q,D], dC[q], level[q]), Eq. (IIC6), (IIC9)-(IIC11)."""
    uu = np.zeros(3)
    uu[:D] = np.asarray(u, dtype=np.float64).reshape(-1)[:D]
    cap = 256
    while True:
        buf = (Point * cap)()
        q = lib().orc_las(D, _dp(uu), RT, ctypes.byref(p), buf, cap)
        if q >= 0:
            break
        cap = -q
    c = np.array([[buf[i].c[a] for a in range(D)] for i in range(q)]).reshape(q, D)
    dC = np.array([buf[i].dC for i in range(q)])
    lev = np.array([buf[i].level for i in range(q)], dtype=np.int64)
    return c, dC, lev


def basis(D, kind, ct):
    """Moment basis T_j(c~) of the EPR constraints and the order of each entry."""
    T = np.zeros(19)
    o = (ctypes.c_int * 19)()
    cc = np.zeros(3)
    cc[:D] = ct
    n = nf(D) if kind == 0 else ng(D)
    (lib().orc_basis_f if kind == 0 else lib().orc_basis_g)(D, _dp(cc), _dp(T), o)
    return T[:n].copy(), np.array(o[:n])


def maxwell_lambda(D, kind, RT) -> np.ndarray:
    """Maxwellian start of the Lagrange multipliers, Eq. (IID13)."""
    lam = np.zeros(19)
    lib().orc_maxwell_lambda(D, kind, RT, _dp(lam))
    return lam[: (nf(D) if kind == 0 else ng(D))].copy()


def epr(D, kind, c, dC, u, RT, con, p: Params, lam0=None):
    """EPR Newton solve, Eq. (IID7)-(IID11).  Returns (status, lambda, populations)."""
    q = len(dC)
    buf = (Point * max(q, 1))()
    for i in range(q):
        for a in range(3):
            buf[i].c[a] = c[i][a] if a < D else 0.0
        buf[i].dC = dC[i]
    uu = np.zeros(3)
    uu[:D] = np.asarray(u, dtype=np.float64).reshape(-1)[:D]
    n = nf(D) if kind == 0 else ng(D)
    lam = np.zeros(19)
    lam[:n] = maxwell_lambda(D, kind, RT) if lam0 is None else lam0
    cc = np.zeros(19)
    cc[:n] = con
    pop = np.zeros(max(q, 1))
    st = lib().orc_epr(D, kind, q, buf, _dp(uu), RT, _dp(cc), ctypes.byref(p), _dp(lam), _dp(pop))
    return st, lam[:n].copy(), pop[:q].copy()


def cell_populations(p: Params, M):
    """Collision + LAS + EPR of one cell: (collision dict, c, dC, f', g', fallback level)."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    co = Collision()
    cap = 256
    while True:
        pts = (Point * cap)()
        pf, pg = np.zeros(cap), np.zeros(cap)
        status = ctypes.c_int()
        q = lib().orc_cell_populations(ctypes.byref(p), _dp(M), ctypes.byref(co), pts, _dp(pf), _dp(pg),
                                       cap, ctypes.byref(status))
        if q >= 0:
            break
        cap = -q
    D = p.D
    c = np.array([[pts[i].c[a] for a in range(D)] for i in range(q)]).reshape(q, D)
    dC = np.array([pts[i].dC for i in range(q)])
    cod = dict(rho=co.rho, u=np.array(co.u[:D]), RT=co.RT, cf=np.array(co.cf[:nf(D)]),
               cg=np.array(co.cg[:ng(D)]), omega=np.array(co.omega[:]), Kn=co.Kn)
    return cod, c, dC, pf[:q].copy(), pg[:q].copy(), status.value


def grid(D, nx, ny=1, periodic=(False, False), pad=0, bc=(0, 0, 0, 0), inlet=(1.0, 0.0, 0.0, 1.0),
         solid=None, nz=1, wall_u=(0.0, 0.0)):
    """Grid description; ``solid`` is a uint8 array over the padded grid (kept alive on the Grid).
    bc: per side (x-, x+, y-, y+[, z-, z+]); inlet: (rho, ux, uy, RT) or (rho, ux, uy, uz, RT);
    periodic: per axis (2 or 3 entries); solid: wall kinds (0 fluid, 1 slip, 2 no-slip at rest,
    3 no-slip moving at wall_u)."""
    g = Grid()
    g.D, g.nx, g.ny, g.nz = D, nx, (ny if D >= 2 else 1), (nz if D == 3 else 1)
    per = tuple(periodic) + (False,) * (3 - len(periodic))
    for a in range(3):
        g.periodic[a] = int(per[a]) if a < D else 0
    g.pad = pad
    bcs = tuple(bc) + (0,) * (6 - len(bc))
    for i in range(6):
        g.bc[i] = bcs[i]
    inl = tuple(inlet) if len(inlet) == 5 else (inlet[0], inlet[1], inlet[2], 0.0, inlet[3])
    for i in range(5):
        g.inlet[i] = inl[i]
    if solid is not None:
        s = np.ascontiguousarray(solid, dtype=np.uint8)
        g._solid_keep = s
        g.solid = s.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
    else:
        g.solid = ctypes.POINTER(ctypes.c_ubyte)()
    g.wall_u[0], g.wall_u[1] = float(wall_u[0]), float(wall_u[1])
    return g


def padded_shape(g: Grid):
    NX = g.nx + (0 if g.periodic[0] else 2 * g.pad)
    NY = 1 if g.D == 1 else g.ny + (0 if g.periodic[1] else 2 * g.pad)
    return NY, NX


def padded_shape3(g: Grid):
    """(NZ, NY, NX) of the padded grid (NZ = 1 below 3D)."""
    NY, NX = padded_shape(g)
    NZ = 1 if g.D < 3 else g.nz + (0 if g.periodic[2] else 2 * g.pad)
    return NZ, NY, NX


def fill_pads(g: Grid, p: Params, M: np.ndarray) -> np.ndarray:
    """Fluid boundary fill of the pad cells, Sec. III.A (returns a filled copy)."""
    W = np.ascontiguousarray(M, dtype=np.float64).copy()
    lib().orc_fill_pads(ctypes.byref(g), ctypes.byref(p), _dp(W))
    return W


def trace_path(g: Grid, ix: int, iy: int, c):
    """Path of one population from padded cell (ix, iy) with velocity c past the
    solid cells of ``g``, Sec. III.B (specular reflection at slip walls).

    Returns (touched, (fi, fj), offset[2], c_star[2]): the final cell, the landing
    point's offset from that cell's centre and the reflected velocity.
    """
    NY, NX = padded_shape(g)
    cc = np.zeros(2)
    cc[:g.D] = np.asarray(c, dtype=np.float64).reshape(-1)[:g.D]
    fi, fj = ctypes.c_int(), ctypes.c_int()
    off, cs = np.zeros(2), np.zeros(2)
    t = lib().orc_trace_path(ctypes.byref(g), NX, NY, ix, iy, _dp(cc), ctypes.byref(fi), ctypes.byref(fj),
                             _dp(off), _dp(cs))
    return bool(t), (fi.value, fj.value), off, cs


def step(g: Grid, p: Params, M: np.ndarray, stats: Stats | None = None) -> np.ndarray:
    """One LELBM time step on a padded SoA state M[nmom, NY*NX] (Sec. II.F, Eq. IIE3)."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    out = np.zeros_like(M)
    st = stats if stats is not None else Stats()
    rc = lib().orc_step(ctypes.byref(g), ctypes.byref(p), _dp(M), _dp(out), ctypes.byref(st))
    if rc != 0:
        raise MemoryError("oracle step failed to allocate")
    return out


def run(g: Grid, p: Params, M: np.ndarray, nsteps: int, stats: Stats | None = None) -> np.ndarray:
    """nsteps time steps."""
    for _ in range(nsteps):
        M = step(g, p, M, stats)
    return M


def state_from_primitives(g: Grid, p: Params, rho, u, RT) -> np.ndarray:
    """Equilibrium moments (Eq. IIB7) of interior primitive fields; pads left zero.

    rho, RT: arrays of the interior shape (ny, nx) (1D: (nx,); 3D: (nz, ny, nx)); u: (D, ...)
    components.
    """
    D = g.D
    if D == 3:
        return _state_from_primitives_3d(g, p, rho, u, RT)
    NY, NX = padded_shape(g)
    px = 0 if g.periodic[0] else g.pad
    py = 0 if (D == 1 or g.periodic[1]) else g.pad
    M = np.zeros((nmom(D), NY, NX))
    rho = np.asarray(rho, dtype=np.float64).reshape(g.ny if D == 2 else 1, g.nx)
    RT = np.asarray(RT, dtype=np.float64).reshape(rho.shape)
    u = np.asarray(u, dtype=np.float64).reshape(D, *rho.shape)
    for j in range(rho.shape[0]):
        for i in range(rho.shape[1]):
            M[:, py + j, px + i] = eq_moments(D, p.K, rho[j, i], u[:, j, i], RT[j, i])
    return M.reshape(nmom(D), NY * NX)


def _state_from_primitives_3d(g: Grid, p: Params, rho, u, RT) -> np.ndarray:
    NZ, NY, NX = padded_shape3(g)
    px = 0 if g.periodic[0] else g.pad
    py = 0 if g.periodic[1] else g.pad
    pz = 0 if g.periodic[2] else g.pad
    M = np.zeros((nmom(3), NZ, NY, NX))
    rho = np.asarray(rho, dtype=np.float64).reshape(g.nz, g.ny, g.nx)
    RT = np.asarray(RT, dtype=np.float64).reshape(rho.shape)
    u = np.asarray(u, dtype=np.float64).reshape(3, *rho.shape)
    for k in range(rho.shape[0]):
        for j in range(rho.shape[1]):
            for i in range(rho.shape[2]):
                M[:, pz + k, py + j, px + i] = eq_moments(3, p.K, rho[k, j, i], u[:, k, j, i], RT[k, j, i])
    return M.reshape(nmom(3), NZ * NY * NX)
