// Landing of streamed populations (Sec. II.E, Sec. III): the target cell of a lattice
// displacement (periodic wrap, discarded outside the interior) and the exact path
// tracing past solid cells of the stationary adiabatic slip wall (Sec. III.B).  Shared
// by the streaming passes of every precision.
#pragma once

#include <cstdint>

#include "lelbm_device.cuh"
#include "lelbm_internal.h"

namespace lbm {

struct LocalStats {
    unsigned long long q_max;
    double disp_max2;
    unsigned long long points;
    long long walls;  // populations reflected at solid faces (an undone deposit counts -1)
};

// Landing cell of an integer displacement (dx, dy) from the emitting cell, or -1
// when the population leaves the interior of its instance (Sec. III: discarded).
template <int D>
__device__ __forceinline__ long long land(const Geometry& g, long long cell, long long lo, int n, int ix, int iy,
                                          int dx, int dy) {
    if constexpr (D == 1) {
        int r = (int)(cell - lo) + dx;  // instances are shorter than 2^31 cells
        if (g.periodic[0]) {
            r %= n;
            if (r < 0) r += n;
            return lo + r;
        }
        return (unsigned int)r < (unsigned int)n ? lo + r : -1;
    } else {
        int tx = ix + dx, ty = iy + dy;
        if (g.periodic[0]) {
            tx %= g.nx;
            if (tx < 0) tx += g.nx;
        } else if (tx < g.pad || tx >= g.pad + g.nx) {
            return -1;
        }
        if (g.periodic[1]) {
            ty %= g.ny;
            if (ty < 0) ty += g.ny;
        } else if (ty < g.pad || ty >= g.pad + g.ny) {
            return -1;
        }
        return (long long)ty * g.NX + tx;
    }
}

// Is interior cell tgt (a result of land) fluid?  Only 2D grids with solid cells have
// interior cells that are not, so the others need no load of the cell type.
template <int D>
__device__ __forceinline__ bool lands_on_fluid(const Geometry& g, const uint8_t* type, long long tgt) {
    if constexpr (D == 1) return true;
    return g.wall_dist == nullptr || type[tgt] == CELL_FLUID;
}

// ---------------------------------------------------------------------------
// Solid boundary, Sec. III.B (stationary adiabatic slip wall, 2D).
// ---------------------------------------------------------------------------
// Is padded cell (i, j) solid?  Periodic axes wrap; cells off the array are not.
__device__ __forceinline__ bool solid_at(const Geometry& g, const uint8_t* type, int i, int j) {
    if (g.periodic[0]) {
        i %= g.NX;
        if (i < 0) i += g.NX;
    }
    if (g.periodic[1]) {
        j %= g.NY;
        if (j < 0) j += g.NY;
    }
    if (i < 0 || i >= g.NX || j < 0 || j >= g.NY) return false;
    return type[(long long)j * g.NX + i] == CELL_SOLID;
}

// Contact bit of padded cell (i, j) for a path that reflects off it: 1 for a slip wall, 2
// for a no-slip wall at rest, 4 for a moving no-slip wall, 0 for a cell that is not solid.
__device__ __forceinline__ int wall_bit(const Geometry& g, const uint8_t* type, int i, int j) {
    if (g.periodic[0]) {
        i %= g.NX;
        if (i < 0) i += g.NX;
    }
    if (g.periodic[1]) {
        j %= g.NY;
        if (j < 0) j += g.NY;
    }
    if (i < 0 || i >= g.NX || j < 0 || j >= g.NY) return 0;
    const long long k = (long long)j * g.NX + i;
    if (type[k] != CELL_SOLID) return 0;
    return g.noslip ? (g.noslip[k] == 1 ? 2 : (g.noslip[k] == 2 ? 4 : 1)) : 1;
}
// The no-slip boundary of a contact bit: 1 at rest, 2 moving, 0 none.
__device__ __forceinline__ int noslip_of_bit(int b) { return b == 2 ? 1 : (b == 4 ? 2 : 0); }

// End of the path x -> x + c past solid cells: the path is walked face by face and at
// a face of a solid cell the velocity component normal to it is reversed (specular
// reflection), until the displacement |c| is used up.  Positions are exact integers in
// units of 1/64 cell: along each axis the faces lie at unfolded distances 32 + 64 k,
// and which of two faces comes first is decided by cross-multiplication, so ties (a
// path through a cell corner) are exact.  Through a corner whose diagonal cell is
// solid, only the normal of a flat wall (exactly one side cell solid) is reversed,
// otherwise both.  The walk ends after at most |c_x| + |c_y| + 2 face events.
struct WallLanding {
    int i, j;        // final (fluid) cell, unwrapped padded coordinates
    double off[2];   // landing point relative to its centre, each in (-1/2, 1/2]
    double cs[2];    // reflected velocity c*
    int touched;     // walls the path reflected off: bit 1 slip, bit 2 no-slip at rest, bit 4
                     // moving no-slip (0: none)
    int last_ns;     // the last no-slip boundary it touched: 1 at rest, 2 moving, 0 none
};

__device__ __forceinline__ WallLanding trace_path(const Geometry& g, const uint8_t* type, int ix, int iy,
                                                  const double* c) {
    constexpr long long S = 64;
    const long long qx = llround((double)S * c[0]), qy = llround((double)S * c[1]);
    int sx = (qx > 0) - (qx < 0), sy = (qy > 0) - (qy < 0);
    const long long ax = qx < 0 ? -qx : qx, ay = qy < 0 ? -qy : qy;
    int i = ix, j = iy;
    int touched = 0, last_ns = 0;
    long long kx = 0, ky = 0;
    while (true) {
        const long long Xn = S / 2 + S * kx, Yn = S / 2 + S * ky;
        const bool hx = ax > 0 && Xn < ax, hy = ay > 0 && Yn < ay;
        if (!hx && !hy) break;
        bool stx = hx, sty = hy;
        if (hx && hy) {
            const long long l = Xn * ay, r = Yn * ax;
            stx = l <= r;
            sty = r <= l;
        }
        if (stx && sty) {
            const int bd = wall_bit(g, type, i + sx, j + sy);
            if (!bd) {
                i += sx;
                j += sy;
            } else {
                const int ba = wall_bit(g, type, i + sx, j), bb = wall_bit(g, type, i, j + sy);
                if (ba && !bb) {
                    touched |= ba;
                    if (noslip_of_bit(ba)) last_ns = noslip_of_bit(ba);
                    sx = -sx;
                    j += sy;
                } else if (bb && !ba) {
                    touched |= bb;
                    if (noslip_of_bit(bb)) last_ns = noslip_of_bit(bb);
                    sy = -sy;
                    i += sx;
                } else {
                    touched |= bd | ba | bb;
                    // a corner: the diagonal cell, else a side cell, names the boundary
                    const int k = noslip_of_bit(bd) ? bd : (noslip_of_bit(ba) ? ba : bb);
                    if (noslip_of_bit(k)) last_ns = noslip_of_bit(k);
                    sx = -sx;
                    sy = -sy;
                }
            }
        } else {
            const int ti = i + (stx ? sx : 0), tj = j + (sty ? sy : 0);
            const int bt = wall_bit(g, type, ti, tj);
            if (bt) {
                if (stx) sx = -sx;
                if (sty) sy = -sy;
                touched |= bt;
                if (noslip_of_bit(bt)) last_ns = noslip_of_bit(bt);
            } else {
                i = ti;
                j = tj;
            }
        }
        kx += stx;
        ky += sty;
    }
    WallLanding L;
    L.i = i;
    L.j = j;
    L.off[0] = (double)sx * (double)(ax - S * kx) * (1.0 / S);
    L.off[1] = (double)sy * (double)(ay - S * ky) * (1.0 / S);
    L.cs[0] = (double)sx * fabs(c[0]);
    L.cs[1] = (double)sy * fabs(c[1]);
    L.touched = touched;
    L.last_ns = last_ns;
    return L;
}

// Adds the raw moments T_N(cp) mf and T_N(cp) mg (2D) to cell tgt of Mout.
__device__ __forceinline__ void add_moments_2d(double* Mout, long long ncell, long long tgt, const double* cp,
                                               double mf, double mg) {
    const double csq = cp[0] * cp[0] + cp[1] * cp[1];
    const double dM[11] = {mf,           cp[0] * mf,          cp[1] * mf,          cp[0] * cp[0] * mf,
                           cp[0] * cp[1] * mf, cp[1] * cp[1] * mf, csq * cp[0] * mf, csq * cp[1] * mf,
                           mg,           cp[0] * mg,          cp[1] * mg};
#pragma unroll
    for (int mm = 0; mm < 11; mm++) atomicAdd(Mout + mm * ncell + tgt, dM[mm]);
}

// How stream_traced treats a population (Sec. III.B, Eq. IIIB8-IIIB15):
//   kStreamReal: a population of the cell.  Its path reflects specularly at slip walls; a
//     path that touches a no-slip wall is absorbed by the last no-slip boundary n it
//     touched (acc[2(n-1)] += mf, acc[2(n-1)+1] += mg: the Delta m of Eq. IIIB8; n = 1 at
//     rest, 2 moving), as is a cloud-in-cell share that would fall on a no-slip cell; a
//     share that would fall on a slip cell is mirrored back across the wall.
//   kStreamImageSum / kStreamImagePut: an image population of no-slip boundary sel (cp is
//     the reversed velocity -c_i, Eq. IIIB13).  Only a path whose last no-slip contact is
//     sel enters the domain, and shares that would fall on a solid cell are dropped; _Sum
//     adds the mass that enters to acc[0..1] (Eq. IIIB14), _Put deposits it scaled by sf
//     and sg (Eq. IIIB15).
enum : int { kStreamReal = 0, kStreamImageSum = 1, kStreamImagePut = 2 };

// Streams one population of cell (ix, iy) with velocity cp past the solid cells (2D):
// its path is traced, the landing point is shared between cells by cloud-in-cell
// weights, and a share that would fall on a slip-wall cell is mirrored back across the
// wall with the normal component of its velocity reversed (into the side cell behind a
// flat wall, into the final cell behind a corner of solid cells).  acc == null: every wall
// is treated as a slip wall (the paths without no-slip walls).  Returns the walls the path
// touched (bit 1 slip, bit 2 no-slip).  Kept out of line: only cells near a solid cell take
// this path.
static __device__ __noinline__ int stream_traced(const Geometry& g, const uint8_t* type, double* Mout, int ix, int iy,
                                                 const double* cp, double mf, double mg, int mode = kStreamReal,
                                                 double* acc = nullptr, double sf = 1.0, double sg = 1.0,
                                                 int sel = 0) {
    const WallLanding L = trace_path(g, type, ix, iy, cp);
    const bool noslip = acc != nullptr;
    if (noslip) {
        if (mode == kStreamReal && L.last_ns) {
            acc[2 * (L.last_ns - 1)] += mf;
            acc[2 * (L.last_ns - 1) + 1] += mg;
            return L.touched;
        }
        if (mode != kStreamReal && L.last_ns != sel) return L.touched;
    }
    const double pos[2] = {(double)L.i + L.off[0], (double)L.j + L.off[1]};
    int base[2];
    double w1[2];
#pragma unroll
    for (int a = 0; a < 2; a++) {
        const double fl = floor(pos[a]);
        base[a] = (int)fl;
        w1[a] = pos[a] - fl;
    }
    const int ncx = w1[0] > 0.0 ? 2 : 1, ncy = w1[1] > 0.0 ? 2 : 1;
    for (int sy = 0; sy < ncy; sy++)
        for (int sx = 0; sx < ncx; sx++) {
            const double w = (sx ? w1[0] : 1.0 - w1[0]) * (sy ? w1[1] : 1.0 - w1[1]);
            int tx = base[0] + sx, ty = base[1] + sy;
            double cw[2] = {L.cs[0], L.cs[1]};
            const int kind = wall_bit(g, type, tx, ty);
            if (kind && noslip) {
                if (mode != kStreamReal) continue;
                const int n = noslip_of_bit(kind);
                if (n) {
                    acc[2 * (n - 1)] += w * mf;
                    acc[2 * (n - 1) + 1] += w * mg;
                    continue;
                }
            }
            if (kind) {
                bool ox = tx != L.i, oy = ty != L.j;
                if (ox && oy) {
                    const bool sa = solid_at(g, type, tx, L.j), sb = solid_at(g, type, L.i, ty);
                    if (!sa && sb) ox = false;
                    else if (sa && !sb) oy = false;
                }
                if (ox) {
                    cw[0] = -cw[0];
                    tx = L.i;
                }
                if (oy) {
                    cw[1] = -cw[1];
                    ty = L.j;
                }
            }
            if (mode == kStreamImageSum) {
                acc[0] += w * mf;
                acc[1] += w * mg;
                continue;
            }
            const long long tgt = land<2>(g, 0, 0, 0, ix, iy, tx - ix, ty - iy);
            const double kf = mode == kStreamImagePut ? sf : 1.0, kg = mode == kStreamImagePut ? sg : 1.0;
            if (tgt >= 0 && type[tgt] == CELL_FLUID) add_moments_2d(Mout, g.ncell, tgt, cw, w * kf * mf, w * kg * mg);
        }
    return L.touched;
}

}  // namespace lbm
