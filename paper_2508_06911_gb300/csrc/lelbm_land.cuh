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
    bool touched;    // reflected at least once
};

__device__ __forceinline__ WallLanding trace_path(const Geometry& g, const uint8_t* type, int ix, int iy,
                                                  const double* c) {
    constexpr long long S = 64;
    const long long qx = llround((double)S * c[0]), qy = llround((double)S * c[1]);
    int sx = (qx > 0) - (qx < 0), sy = (qy > 0) - (qy < 0);
    const long long ax = qx < 0 ? -qx : qx, ay = qy < 0 ? -qy : qy;
    int i = ix, j = iy;
    bool touched = false;
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
            if (!solid_at(g, type, i + sx, j + sy)) {
                i += sx;
                j += sy;
            } else {
                const bool sa = solid_at(g, type, i + sx, j), sb = solid_at(g, type, i, j + sy);
                touched = true;
                if (sa && !sb) {
                    sx = -sx;
                    j += sy;
                } else if (sb && !sa) {
                    sy = -sy;
                    i += sx;
                } else {
                    sx = -sx;
                    sy = -sy;
                }
            }
        } else {
            const int ti = i + (stx ? sx : 0), tj = j + (sty ? sy : 0);
            if (solid_at(g, type, ti, tj)) {
                if (stx) sx = -sx;
                if (sty) sy = -sy;
                touched = true;
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

// Streams one population of cell (ix, iy) with velocity cp past the solid cells (2D):
// its path is traced, the landing point is shared between cells by cloud-in-cell
// weights, and a share that would fall on a solid cell is mirrored back across the wall
// with the normal component of its velocity reversed (into the side cell behind a flat
// wall, into the final cell behind a corner of solid cells).  Returns whether the path
// was reflected.  Kept out of line: only cells near a solid cell take this path.
static __device__ __noinline__ bool stream_traced(const Geometry& g, const uint8_t* type, double* Mout, int ix, int iy,
                                           const double* cp, double mf, double mg) {
    const WallLanding L = trace_path(g, type, ix, iy, cp);
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
            if (solid_at(g, type, tx, ty)) {
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
            const long long tgt = land<2>(g, 0, 0, 0, ix, iy, tx - ix, ty - iy);
            if (tgt >= 0 && type[tgt] == CELL_FLUID) add_moments_2d(Mout, g.ncell, tgt, cw, w * mf, w * mg);
        }
    return L.touched;
}

}  // namespace lbm
