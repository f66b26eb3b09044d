// Device code of the LELBM time step (arXiv:2508.06911) for sm_103a: the fused
// single-cell kernel templates.  Each (dimension, precision) variant of the
// cell-update kernel and each precision of the persistent 1D batch kernel is
// instantiated in its own object (lelbm_cell.cu, lelbm_batch.cu) so that the
// variants compile in parallel.
//
// One thread owns one cell for the whole single-cell operation (Fig. 5):
// collision module -> LAS module -> EPR module -> MS module.  The velocity set
// is never stored: it is re-enumerated row by row for every Newton pass and for
// the streaming pass, so a cell needs registers only, whatever its temperature
// (the memory-constant property of moment streaming, Sec. II.E).
//
// The EPR Newton works in thermal units t = (c - u) / sqrt(RT): the monomials
// T_j(t) are O(1) at any temperature, the Jacobian is well scaled, and the
// residual tested against the tolerance is the paper's residual divided by
// sqrt(RT)^order.  Rounding-sensitive decisions (macroscopic variables,
// acoustic radius, refinement levels, stencil membership) use explicitly
// rounded operations so they do not depend on FMA contraction.

#pragma once

#include <cfloat>
#include <cstdint>

#include "lelbm_device.cuh"
#include "lelbm_df.cuh"
#include "lelbm_internal.h"
#include "lelbm_land.cuh"
#include "lelbm_mlp.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// FP32 streaming (the FP32 path).  Populations and their moment fractions are
// computed in FP32; every fraction is widened to FP64 for the FP64 atomic
// accumulation, with integer operations (GB300 runs FP64 at 1/64 of the FP32 rate).
// The emitted mass, momentum and energy are summed exactly (compensated FP32 sums of
// the deposited values), and what they miss of the cell's conserved moments (the FP32
// Newton leaves a residual of about 1e-6) is added at the emitting cell, so the
// totals are conserved to FP64 rounding.
// ---------------------------------------------------------------------------
// Compensated FP32 sum: hi + lo carries the exact sum to about 1e-14 relative
// (Knuth's two-sum on every addition).  The explicitly rounded operations keep the
// compiler from fusing a product that produced v into these additions: the sum must be
// of v as rounded, the value that is deposited.
struct Acc32 {
    float hi, lo;
    __device__ __forceinline__ void add(float v) {
        const float s = __fadd_rn(hi, v);
        const float bp = __fsub_rn(s, hi);
        lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(v, bp)));
        hi = s;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Splits v into (1 - w) v and w v with the two parts summing to v exactly: the larger
// part is rounded, the smaller is the exact difference (Sterbenz).
__device__ __forceinline__ void split_exact(float v, float w, float& lo_part, float& hi_part) {
    if (w <= 0.5f) {
        lo_part = flush_sub(v * (1.f - w));
        hi_part = v - lo_part;
    } else {
        hi_part = flush_sub(v * w);
        lo_part = v - hi_part;
    }
}

// Moment fractions T_N(c) mf and T_N(c) mg (stored-moment order) in FP32.
template <int D>
__device__ __forceinline__ void fractions32(const float* cp, float mf, float mg, float* v) {
    float csq = 0.f;
#pragma unroll
    for (int a = 0; a < D; a++) csq += cp[a] * cp[a];
    v[0] = mf;
#pragma unroll
    for (int a = 0; a < D; a++) v[1 + a] = cp[a] * mf;
#pragma unroll
    for (int a = 0; a < D; a++)
#pragma unroll
        for (int b = a; b < D; b++) v[iM2<D>(a, b)] = cp[a] * cp[b] * mf;
#pragma unroll
    for (int gg = 0; gg < D; gg++) v[iMD<D>(gg)] = csq * cp[gg] * mf;
    v[iG0<D>()] = mg;
#pragma unroll
    for (int gg = 0; gg < D; gg++) v[iG1<D>(gg)] = cp[gg] * mg;
}

// Sign of each 2D stored moment under x -> -x (ox) and y -> -y (oy).
__device__ __forceinline__ float reflect_sign_2d(int i, bool ox, bool oy) {
    // M0 Mx My Mxx Mxy Myy MDx MDy G0 Gx Gy
    const bool odd_x = i == 1 || i == 4 || i == 6 || i == 9;
    const bool odd_y = i == 2 || i == 4 || i == 7 || i == 10;
    return ((odd_x && ox) != (odd_y && oy)) ? -1.f : 1.f;
}

// stream_traced for FP32 fractions v (of the unreflected velocity cp): the landing
// point is shared by exact splits, and reflections and mirrored shares reverse the
// odd moments.  Returns whether the path was reflected.
static __device__ __noinline__ bool stream_traced32(const Geometry& g, const uint8_t* type, double* Mout, int ix,
                                                    int iy, const double* cp, const float* v) {
    const WallLanding L = trace_path(g, type, ix, iy, cp);
    const bool rx = (L.cs[0] < 0.0) != (cp[0] < 0.0), ry = (L.cs[1] < 0.0) != (cp[1] < 0.0);
    const double pos[2] = {(double)L.i + L.off[0], (double)L.j + L.off[1]};
    int base[2];
    float w1[2];
#pragma unroll
    for (int a = 0; a < 2; a++) {
        const double fl = floor(pos[a]);
        base[a] = (int)fl;
        w1[a] = (float)(pos[a] - fl);
    }
    for (int sy = 0; sy < 2; sy++)
        for (int sx = 0; sx < 2; sx++) {
            if ((sx && w1[0] == 0.f) || (sy && w1[1] == 0.f)) continue;
            int tx = base[0] + sx, ty = base[1] + sy;
            bool ox = false, oy = false;
            if (solid_at(g, type, tx, ty)) {
                ox = tx != L.i;
                oy = ty != L.j;
                if (ox && oy) {
                    const bool sa = solid_at(g, type, tx, L.j), sb = solid_at(g, type, L.i, ty);
                    if (!sa && sb) ox = false;
                    else if (sa && !sb) oy = false;
                }
                if (ox) tx = L.i;
                if (oy) ty = L.j;
            }
            const long long tgt = land<2>(g, 0, 0, 0, ix, iy, tx - ix, ty - iy);
            if (tgt < 0 || type[tgt] != CELL_FLUID) continue;
#pragma unroll
            for (int mm = 0; mm < 11; mm++) {
                float x0, x1, part = v[mm];
                split_exact(part, w1[0], x0, x1);
                part = sx ? x1 : x0;
                split_exact(part, w1[1], x0, x1);
                part = sy ? x1 : x0;
                part *= reflect_sign_2d(mm, rx != ox, ry != oy);
                if (part != 0.f) atomicAdd(Mout + mm * g.ncell + tgt, widen(part));
            }
        }
    return L.touched;
}

template <int D>
__device__ __forceinline__ void scatter_cell32(const Model& m, const Geometry& g, const uint8_t* type, double* Mout,
                                               long long cell, const CellState<D>& c, const Stencil<D>& st,
                                               const RowTable<D>& tab, const float* lf, const float* lg,
                                               LocalStats& ls) {
    constexpr int NM = Dim<D>::NM;
    const bool has_g = m.K > 0.0;
    const float mfs = (float)c.rho;                              // rho dV f'
    const float mgs = has_g ? (float)(c.rho * m.K * c.RT) : 0.f;  // rho K RT dV g'
    long long lo = 0;
    int n = 0, ix = 0, iy = 0;
    if constexpr (D == 1) {
        const int b = g.inst_of_cell[cell];
        lo = g.inst_lo[b];
        n = g.inst_n[b];
    } else {
        iy = (int)(cell / g.NX);
        ix = (int)(cell - (long long)iy * g.NX);
    }
    bool near_wall = false;
    if constexpr (D == 2) {
        if (g.wall_dist)
            near_wall = (double)g.wall_dist[cell] <= fmax(fabs(c.u[0]), fabs(c.u[1])) + (double)st.R + 1.5;
    }
    Acc32 em{0.f, 0.f}, ee{0.f, 0.f}, ep[D];
#pragma unroll
    for (int a = 0; a < D; a++) ep[a] = Acc32{0.f, 0.f};
    unsigned long long q = 0;
    long long walls = 0;
    int dmax = 0;
    auto account = [&](const float* v) {
        em.add(v[0]);
#pragma unroll
        for (int a = 0; a < D; a++) ep[a].add(v[1 + a]);
#pragma unroll
        for (int a = 0; a < D; a++) ee.add(v[iM2<D>(a, a)]);
        ee.add(v[iG0<D>()]);
    };
    auto put = [&](long long tgt, const float* v) {
        if (tgt < 0 || !lands_on_fluid<D>(g, type, tgt)) return;
        double* p = Mout + tgt;
#pragma unroll
        for (int mm = 0; mm < NM; mm++) atomicAdd(p + mm * g.ncell, widen(v[mm]));
    };
    const float s32 = tab.s32;
    auto row = [&](int cy, int xa, int xb) {
        const float y = D == 2 ? tab.ty(cy) : 0.f;
        float cf[4], cg[3];
        row_coeffs32<D>(lf, lg, y, cf, cg);
        const float x0 = tab.tx(xa);
        float kf = 0.f, cxf = (float)xa;  // point index and c_x as floats (exact)
        for (int k = 0; k <= xb - xa; k++, kf += 1.f, cxf += 1.f) {
            const float x = fmaf(kf, s32, x0);
            const float f = __expf(-fmaf(fmaf(fmaf(cf[3], x, cf[2]), x, cf[1]), x, cf[0]));
            const float gp = has_g ? __expf(-fmaf(fmaf(cg[2], x, cg[1]), x, cg[0])) : 0.f;
            const int cx = xa + k;
            float cpf[D];
            cpf[0] = cxf;
            if constexpr (D == 2) cpf[1] = (float)cy;
            float v[NM];
            fractions32<D>(cpf, mfs * f, mgs * gp, v);
            account(v);
            if constexpr (D == 2) {
                if (near_wall) {
                    const double cpd[2] = {(double)cx, (double)cy};
                    walls += stream_traced32(g, type, Mout, ix, iy, cpd, v) ? 1 : 0;
                    continue;
                }
            }
            put(land<D>(g, cell, lo, n, ix, iy, cx, cy), v);
        }
        q += (unsigned long long)(xb - xa + 1);
        const int ex = max(abs(xa), abs(xb));
        dmax = max(dmax, ex * ex + cy * cy);
    };
    // a refined point at cp (weight w), FP32 thermal coordinates (x, y); the landing
    // cell's cloud-in-cell split along each axis is base + {0, 1} with weight w1
    auto refined = [&](const float* cpf, float x, float y, float w, const int* base, const float* w1,
                       const double* cpd) {
        float cf[4], cg[3];
        row_coeffs32<D>(lf, lg, y, cf, cg);
        const float f = w * __expf(-fmaf(fmaf(fmaf(cf[3], x, cf[2]), x, cf[1]), x, cf[0]));
        const float gp = has_g ? w * __expf(-fmaf(fmaf(cg[2], x, cg[1]), x, cg[0])) : 0.f;
        float v[NM];
        fractions32<D>(cpf, mfs * f, mgs * gp, v);
        account(v);
        q++;
        if constexpr (D == 2) {
            if (near_wall) {
                walls += stream_traced32(g, type, Mout, ix, iy, cpd, v) ? 1 : 0;
                return;
            }
        }
        const int ncx = w1[0] > 0.f ? 2 : 1;
        const int ncy = (D == 2 && w1[D - 1] > 0.f) ? 2 : 1;
        for (int sy = 0; sy < ncy; sy++)
            for (int sx = 0; sx < ncx; sx++) {
                float part[NM];
#pragma unroll
                for (int mm = 0; mm < NM; mm++) {
                    float a0, a1;
                    split_exact(v[mm], w1[0], a0, a1);
                    part[mm] = sx ? a1 : a0;
                    if constexpr (D == 2) {
                        split_exact(part[mm], w1[1], a0, a1);
                        part[mm] = sy ? a1 : a0;
                    }
                }
                put(land<D>(g, cell, lo, n, ix, iy, base[0] + sx, D == 2 ? base[D - 1] + sy : 0), part);
            }
    };
    // Split points without wall tracing: one deposit per landing cell and child row.  Along
    // x the children p -/+ 1/4 land 3/4 on p and 1/4 on p -/+ 1; their shares are summed
    // with each other and with the level-0 points a - 1 and b + 1 of the row (1D), or, in
    // 2D, per child row cy + sy/4 and then shared 3/4 : 1/4 between rows cy and cy + sy.
    // The accounting takes the deposits as they are.
    constexpr float w_child = D == 1 ? 0.5f : 0.25f;
    // fractions of the level-0 point (cx, cy), and of the child (p + sx/4, cy + sy/4) with
    // the exponent polynomials cf, cg of its row
    auto point_v = [&](int cx, int cy, float* v) {
        float cf[4], cg[3];
        row_coeffs32<D>(lf, lg, D == 2 ? tab.ty(cy) : 0.f, cf, cg);
        const float x = tab.tx(cx);
        const float f = __expf(-fmaf(fmaf(fmaf(cf[3], x, cf[2]), x, cf[1]), x, cf[0]));
        const float gp = has_g ? __expf(-fmaf(fmaf(cg[2], x, cg[1]), x, cg[0])) : 0.f;
        float cpf[D];
        cpf[0] = (float)cx;
        if constexpr (D == 2) cpf[1] = (float)cy;
        fractions32<D>(cpf, mfs * f, mgs * gp, v);
    };
    auto child_v = [&](const float* cf, const float* cg, int p, int sx, float cyq, float* v) {
        const float x = tab.tx(p, 0.25f * (float)sx);
        const float f = w_child * __expf(-fmaf(fmaf(fmaf(cf[3], x, cf[2]), x, cf[1]), x, cf[0]));
        const float gp = has_g ? w_child * __expf(-fmaf(fmaf(cg[2], x, cg[1]), x, cg[0])) : 0.f;
        float cpf[D];
        cpf[0] = (float)p + 0.25f * (float)sx;
        if constexpr (D == 2) cpf[1] = cyq;
        fractions32<D>(cpf, mfs * f, mgs * gp, v);
    };
    auto emit = [&](int tx, int ty, const float* v) {
        account(v);
        put(land<D>(g, cell, lo, n, ix, iy, tx, ty), v);
    };
    // column t of child row sy: V (x-summed children) and, when l0, the level-0 point (t, cy).
    // 1D: one deposit V (+ the point); 2D: V/4 on row cy + sy, 3V/4 (+ the point) on row cy.
    // One call site each for emit and point_v keeps the code of this path short.
    auto emit_col = [&](int t, int cy, int sy, const float* V, bool l0) {
        float lv[NM];
        if (l0) {
            point_v(t, cy, lv);
        } else {
#pragma unroll
            for (int mm = 0; mm < NM; mm++) lv[mm] = 0.f;
        }
#pragma unroll 1
        for (int k = (D == 2 ? 0 : 1); k < 2; k++) {
            const float w = D == 1 ? 1.f : (k == 0 ? 0.25f : 0.75f);
            float o[NM];
#pragma unroll
            for (int mm = 0; mm < NM; mm++) o[mm] = k == 0 ? w * V[mm] : fmaf(w, V[mm], lv[mm]);
            emit(t, k == 0 ? cy + sy : cy, o);
        }
    };
    // child row sy (0 in 1D) of the split points a..b of row cy (level-0 points x0..x1);
    // with_l0: the level-0 points a - 1 and b + 1 join their columns' deposits.  The
    // children are taken in order p - 1/4, p + 1/4, ...; each adds w_lo of its fractions
    // to column lo (cA) and w_hi to column lo + 1 (cB): (p - 1, p) with (1/4, 3/4) for the
    // left child, (p, p + 1) with (3/4, 1/4) for the right one.  After a left child,
    // column p - 1 is complete.  Two empty left children past b emit columns b and b + 1.
    auto band_row = [&](int cy, int sy, int a, int b, int x0, int x1, bool with_l0) {
        float cf[4], cg[3];
        row_coeffs32<D>(lf, lg, D == 2 ? tab.ty(cy, 0.25f * (float)sy) : 0.f, cf, cg);
        const float cyq = (float)cy + 0.25f * (float)sy;
        float cA[NM], cB[NM], v[NM];
#pragma unroll
        for (int mm = 0; mm < NM; mm++) cA[mm] = cB[mm] = 0.f;
        const int nch = 2 * (b - a + 1);
#pragma unroll 1
        for (int h = 0; h <= nch + 2; h++) {
            const int p = a + (h >> 1);
            const bool left = (h & 1) == 0;
            if (h < nch) {
                child_v(cf, cg, p, left ? -1 : 1, cyq, v);
            } else {
#pragma unroll
                for (int mm = 0; mm < NM; mm++) v[mm] = 0.f;
            }
            const float w_lo = left ? 0.25f : 0.75f, w_hi = left ? 0.75f : 0.25f;
#pragma unroll
            for (int mm = 0; mm < NM; mm++) {
                cA[mm] = fmaf(w_lo, v[mm], cA[mm]);
                cB[mm] = fmaf(w_hi, v[mm], cB[mm]);
            }
            if (left) {
                const int t = p - 1;  // complete
                emit_col(t, cy, sy, cA, with_l0 && ((t == a - 1 && t >= x0) || (t == b + 1 && t <= x1)));
#pragma unroll
                for (int mm = 0; mm < NM; mm++) {
                    cA[mm] = cB[mm];
                    cB[mm] = 0.f;
                }
            }
        }
        q += (unsigned long long)nch + (with_l0 ? (a - 1 >= x0) + (b + 1 <= x1) : 0);
        const int ex = max(abs(x0), abs(x1));
        dmax = max(dmax, ex * ex + cy * cy);
    };
    // a row with split points a..b: its level-0 segments and its child rows
    auto split_row = [&](int cy, int x0, int x1, int a, int b) {
#pragma unroll 1
        for (int sy = (D == 2 ? -1 : 0); sy <= (D == 2 ? 1 : 0); sy += 2) band_row(cy, sy, a, b, x0, x1, sy <= 0);
    };
    // the level-0 segments of a row: x0..x1 less the split points a..b and their
    // neighbours a - 1, b + 1 (which split_row deposits)
    auto row_segments = [&](int cy, int x0, int x1, int a, int b) {
        const bool band = a <= b;
#pragma unroll 1
        for (int k = 0; k < (band ? 2 : 1); k++) {
            const int xa = band ? (k == 0 ? x0 : b + 2) : x0;
            const int xb = band ? (k == 0 ? a - 2 : x1) : x1;
            if (xa <= xb) row(cy, xa, xb);
        }
        if (band) split_row(cy, x0, x1, a, b);
    };
    if (tab.ok) {
        // children of split points at (p + sx/4, cy + sy/4): along an axis the landing
        // point p - 1/4 splits 3/4 : 1/4 over p - 1, p and p + 1/4 splits over p, p + 1
        auto child = [&](int p, int cy, int sx, int sy) {
            const float qx = 0.25f * (float)sx, qy = 0.25f * (float)sy;
            float cpf[D];
            int base[D];
            float w1[D];
            cpf[0] = (float)p + qx;
            base[0] = sx < 0 ? p - 1 : p;
            w1[0] = sx < 0 ? 0.75f : 0.25f;
            if constexpr (D == 2) {
                cpf[1] = (float)cy + qy;
                base[1] = sy < 0 ? cy - 1 : cy;
                w1[1] = sy < 0 ? 0.75f : 0.25f;
            }
            double cpd[2] = {0.0, 0.0};
            if constexpr (D == 2) {
                if (near_wall) {
                    cpd[0] = (double)cpf[0];
                    cpd[1] = (double)cpf[1];
                }
            }
            refined(cpf, tab.tx(p, qx), D == 2 ? tab.ty(cy, qy) : 0.f, D == 1 ? 0.5f : 0.25f, base, w1, cpd);
        };
        if (near_wall) {
            tab.visit(row, child);  // every share is traced on its own
        } else if constexpr (D == 1) {
            row_segments(0, tab.x0, tab.x1, tab.a, tab.b);
        } else {
            for (int r = 0; r < tab.nrows; r++) {
                int rx0, rx1, ra, rb;
                tab.row_ext(r, rx0, rx1, ra, rb);
                row_segments(tab.y_first + r, rx0, rx1, ra, rb);
            }
        }
    } else {
        auto leaf = [&](const double* cp, double dC) {
            float cpf[D];
            int base[D];
            float w1[D];
#pragma unroll
            for (int a = 0; a < D; a++) {
                cpf[a] = (float)cp[a];
                const double fl = floor(cp[a]);
                base[a] = (int)fl;
                w1[a] = (float)(cp[a] - fl);
            }
            refined(cpf, (float)((cp[0] - c.u[0]) * c.inv_sig),
                    D == 2 ? (float)((cp[D - 1] - c.u[D - 1]) * c.inv_sig) : 0.f, (float)dC, base, w1, cp);
        };
        st.for_each_row(row, leaf);
    }
    // what the emitted fractions miss of the conserved moments stays in the cell
    if (type[cell] == CELL_FLUID) {
        double usq = 0.0;
#pragma unroll
        for (int a = 0; a < D; a++) usq += c.u[a] * c.u[a];
        const double dm = c.rho - em.value();
        const double dE = c.rho * (usq + ((double)D + m.K) * c.RT) - ee.value();
        atomicAdd(Mout + cell, dm);
#pragma unroll
        for (int a = 0; a < D; a++) {
            atomicAdd(Mout + (1 + a) * g.ncell + cell, c.rho * c.u[a] - ep[a].value());
            atomicAdd(Mout + iM2<D>(a, a) * g.ncell + cell, dE / (double)D);
        }
    }
    if (q > ls.q_max) ls.q_max = q;
    ls.points += q;
    ls.walls += walls;
    ls.disp_max2 = fmax(ls.disp_max2, (double)dmax);
}

// Moment streaming, Eq. (IIE3): T_N(c_i) rho f'_i and T_N(c_i) rho K RT g'_i added at
// x + c_i.  Level-0 points land on one cell; refined points are shared between the
// cells they overlap (cloud-in-cell).
//
// With CHECK, the same pass also accumulates the moments of degree <= 3 (fluons)
// and <= 2 (phonons) of the deposited populations and returns whether their
// residual against conF / conG is within the tolerance (the FP64 judge of the
// mixed path).  sign = -1 removes a previous deposit of the same populations.
// Image populations of the no-slip walls (Sec. III.B, Eq. IIIB10-IIIB15) for a cell whose
// streaming gave no-slip boundary n (1 at rest, 2 moving at u_w) the mass absorbed[2(n-1)]
// (f) and the phonon energy absorbed[2(n-1)+1] (g).  The images of boundary n are the EPR
// populations of the cell's post-collision central constraints (conF, conG) at the bulk
// velocity u_n = u - 2 u_w (Eq. IIIB11, both components), launched with -c_i; at rest they
// are the cell's own populations.  Those whose last no-slip contact is boundary n enter the
// domain, scaled so that they carry exactly what the boundary absorbed: one pass sums what
// enters, a second deposits it.  If nothing enters (a cell boxed in by walls) the absorbed
// mass and internal energy stay in the cell, at rest.
static __device__ __noinline__ void noslip_images(const Model& m, const Geometry& g, const uint8_t* type, double* Mout,
                                                  long long cell, int ix, int iy, const CellState<2>& c,
                                                  const Stencil<2>& st, const double* lf, const double* lg,
                                                  const double* conF, const double* conG, double mfs, double mgs,
                                                  const double* absorbed) {
    const bool has_g = m.K > 0.0;
    for (int n = 1; n <= 2; n++) {
        const double* dm = absorbed + 2 * (n - 1);
        if ((dm[0] == 0.0 && dm[1] == 0.0) || (n == 2 && !conF)) continue;
        CellState<2> ci = c;
        Stencil<2> si = st;
        double li_f[10], li_g[6];
#pragma unroll
        for (int j = 0; j < 10; j++) li_f[j] = lf[j];
#pragma unroll
        for (int j = 0; j < 6; j++) li_g[j] = lg[j];
        if (n == 2) {  // the EPR at u_n, with the fallbacks of a failed solve
            ci.u[0] = c.u[0] - 2.0 * g.wall_u[0];
            ci.u[1] = c.u[1] - 2.0 * g.wall_u[1];
            si.init(ci, m);
            unsigned int pf = 0, pg = 0;
            int sf, sg;
            solve_fg<2>(ci, si, conF, conG, has_g, li_f, li_g, m, sf, sg, pf, pg);
            if (sf < 0 || sg < 0) {
                maxwell_start_fg<2, 10, 6>(ci.RT, li_f, li_g);
                solve_fg<2>(ci, si, conF, conG, has_g, li_f, li_g, m, sf, sg, pf, pg);
            }
            if (sf < 0 || sg < 0) {
                double ef[10], eg[6];
#pragma unroll
                for (int j = 0; j < 10; j++) ef[j] = (j == 0 || j == 3 || j == 5) ? 1.0 : 0.0;
#pragma unroll
                for (int j = 0; j < 6; j++) eg[j] = (j == 0 || j == 3 || j == 5) ? 1.0 : 0.0;
                maxwell_start_fg<2, 10, 6>(ci.RT, li_f, li_g);
                solve_fg<2>(ci, si, ef, eg, has_g, li_f, li_g, m, sf, sg, pf, pg);
                if (sf < 0 || sg < 0) {  // normalised Maxwellian weights, f and g alike
#pragma unroll
                    for (int j = 0; j < 10; j++) li_f[j] = (j == 3 || j == 5) ? 0.5 : 0.0;
                    double S = 0.0;
                    auto sum = [&](const double* cp, double dC) {
                        const double tx = (cp[0] - ci.u[0]) * ci.inv_sig, ty = (cp[1] - ci.u[1]) * ci.inv_sig;
                        S += dC * exp(-0.5 * (tx * tx + ty * ty));
                    };
                    si.for_each(sum);
                    li_f[0] = log(S) - 1.0;
#pragma unroll
                    for (int j = 0; j < 6; j++) li_g[j] = li_f[j];
                }
            }
        }
        double kept[2] = {0.0, 0.0}, unused[2] = {0.0, 0.0};
        for (int pass = 0; pass < 2; pass++) {
            const double sf = kept[0] > 0.0 ? dm[0] / kept[0] : 0.0;
            const double sg = kept[1] > 0.0 ? dm[1] / kept[1] : 0.0;
            auto image = [&](const double* cp, double dC) {
                const double t[2] = {(cp[0] - ci.u[0]) * ci.inv_sig, (cp[1] - ci.u[1]) * ci.inv_sig};
                double T[10];
                Basis<2, true>::eval(t, T);
                double ef = 1.0;
#pragma unroll
                for (int j = 0; j < 10; j++) ef += li_f[j] * T[j];
                double gp = 0.0;
                if (has_g) {
                    double eg = 1.0;
#pragma unroll
                    for (int j = 0; j < 6; j++) eg += li_g[j] * T[j];
                    gp = dC * exp(-eg);
                }
                const double cm[2] = {-cp[0], -cp[1]};
                stream_traced(g, type, Mout, ix, iy, cm, mfs * (dC * exp(-ef)), mgs * gp,
                              pass == 0 ? kStreamImageSum : kStreamImagePut, pass == 0 ? kept : unused, sf, sg, n);
            };
            si.for_each(image);
        }
        if (type[cell] == CELL_FLUID) {
            if (kept[0] <= 0.0 && dm[0] != 0.0) atomicAdd(Mout + cell, dm[0]);
            if (kept[1] <= 0.0 && dm[1] != 0.0) atomicAdd(Mout + (long long)iG0<2>() * g.ncell + cell, dm[1]);
        }
    }
}

template <int D, bool CHECK>
__device__ __forceinline__ bool scatter_cell(const Model& m, const Geometry& g, const uint8_t* type, double* Mout,
                                             long long cell, const CellState<D>& c, const Stencil<D>& st,
                                             const double* lf, const double* lg, LocalStats& ls, double sign = 1.0,
                                             const double* conF = nullptr, const double* conG = nullptr) {
    constexpr int NM = Dim<D>::NM;
    constexpr int RF = D == 1 ? 4 : 10, RG = D == 1 ? 3 : 6;  // monomials of degree <= 3 / <= 2
    const bool has_g = m.K > 0.0;
    const double mfs = sign * c.rho;               // rho dV f'
    const double mgs = sign * c.rho * m.K * c.RT;  // rho K RT dV g'
    double RFm[RF], RGm[RG];
    if constexpr (CHECK) {
#pragma unroll
        for (int i = 0; i < RF; i++) RFm[i] = 0.0;
#pragma unroll
        for (int i = 0; i < RG; i++) RGm[i] = 0.0;
    }
    long long lo = 0;
    int n = 0, ix = 0, iy = 0;
    if constexpr (D == 1) {
        const int b = g.inst_of_cell[cell];
        lo = g.inst_lo[b];
        n = g.inst_n[b];
    } else {
        iy = (int)(cell / g.NX);
        ix = (int)(cell - (long long)iy * g.NX);
    }
    unsigned long long q = 0;
    long long walls = 0;
    double dmax2 = 0.0;
    // Sec. III.B: paths are traced past solid faces only where a solid cell lies within
    // reach: a path or a cloud-in-cell share touches cells at Chebyshev distance at
    // most max_a |c_a| + 1, and |c_a| <= |u_a| + R_ac + 1/2.
    bool near_wall = false;
    if constexpr (D == 2) {
        if (g.wall_dist)
            near_wall = (double)g.wall_dist[cell] <= fmax(fabs(c.u[0]), fabs(c.u[1])) + (double)st.R + 1.5;
    }
    auto deposit = [&](long long tgt, const double* cp, double mf, double mg) {
        if (tgt < 0 || !lands_on_fluid<D>(g, type, tgt)) return;
        double csq = 0.0;
#pragma unroll
        for (int a = 0; a < D; a++) csq += cp[a] * cp[a];
        double dM[NM];
        dM[0] = mf;
#pragma unroll
        for (int a = 0; a < D; a++) dM[1 + a] = cp[a] * mf;
#pragma unroll
        for (int a = 0; a < D; a++)
#pragma unroll
            for (int b = a; b < D; b++) dM[iM2<D>(a, b)] = cp[a] * cp[b] * mf;
#pragma unroll
        for (int gg = 0; gg < D; gg++) dM[iMD<D>(gg)] = csq * cp[gg] * mf;
        dM[iG0<D>()] = mg;
#pragma unroll
        for (int gg = 0; gg < D; gg++) dM[iG1<D>(gg)] = cp[gg] * mg;
#pragma unroll
        for (int mm = 0; mm < NM; mm++) atomicAdd(Mout + mm * g.ncell + tgt, dM[mm]);
    };
    double absorbed[4] = {0.0, 0.0, 0.0, 0.0};  // Eq. (IIIB8): what the no-slip walls took (f, g;
                                                // at rest, moving)
    auto deposit_traced = [&](const double* cp, double mf, double mg) {
        if constexpr (D == 2)
            walls += stream_traced(g, type, Mout, ix, iy, cp, mf, mg, kStreamReal, g.noslip ? absorbed : nullptr)
                         ? (sign > 0.0 ? 1 : -1)
                         : 0;
    };
    auto row = [&](int cy, int xa, int xb) {
        double y = 0.0;
        if constexpr (D == 2) y = ((double)cy - c.u[1]) * c.inv_sig;
        double cf[4], cg[3];
        row_coeffs<D>(lf, lg, y, cf, cg);
        double SF[4] = {0.0, 0.0, 0.0, 0.0}, SG[3] = {0.0, 0.0, 0.0};
        auto point = [&](int k, double x, double f, double gp) {
            const int cx = xa + k;
            if constexpr (CHECK) {
                const double x2 = x * x;
                SF[0] += f;
                SF[1] += x * f;
                SF[2] += x2 * f;
                SF[3] += x2 * x * f;
                SG[0] += gp;
                SG[1] += x * gp;
                SG[2] += x2 * gp;
            }
            double cp[D];
            cp[0] = (double)cx;
            if constexpr (D == 2) cp[1] = (double)cy;
            if (near_wall)
                deposit_traced(cp, mfs * f, mgs * gp);
            else
                deposit(land<D>(g, cell, lo, n, ix, iy, cx, cy), cp, mfs * f, mgs * gp);
        };
        row_eval(cf, cg, true, has_g, ((double)xa - c.u[0]) * c.inv_sig, c.inv_sig, xb - xa + 1, point);
        if constexpr (CHECK) {
            // fold y^b into the moments x^a y^b (a + b <= 3 / <= 2)
            double yp[4] = {1.0, y, y * y, y * y * y};
#pragma unroll
            for (int b = 0; b <= (D == 2 ? 3 : 0); b++)
#pragma unroll
                for (int a = 0; a + b <= 3; a++) RFm[tix(a, b, 3)] += SF[a] * yp[b];
#pragma unroll
            for (int b = 0; b <= (D == 2 ? 2 : 0); b++)
#pragma unroll
                for (int a = 0; a + b <= 2; a++) RGm[tix(a, b, 2)] += SG[a] * yp[b];
        }
        q += (unsigned long long)(xb - xa + 1);
        const double ex = (double)(abs(xa) > abs(xb) ? xa : xb);
        dmax2 = fmax(dmax2, ex * ex + (double)cy * (double)cy);
    };
    auto leaf = [&](const double* cp, double dC) {
        const double x = (cp[0] - c.u[0]) * c.inv_sig;
        double y = 0.0;
        if constexpr (D == 2) y = (cp[1] - c.u[1]) * c.inv_sig;
        double cf[4], cg[3];
        row_coeffs<D>(lf, lg, y, cf, cg);
        const double f = dC * exp(-(((cf[3] * x + cf[2]) * x + cf[1]) * x + cf[0]));
        const double gp = has_g ? dC * exp(-((cg[2] * x + cg[1]) * x + cg[0])) : 0.0;
        const double mf = mfs * f, mg = mgs * gp;
        if constexpr (CHECK) {
            double px[4] = {1.0, x, x * x, x * x * x}, py[4] = {1.0, y, y * y, y * y * y};
#pragma unroll
            for (int b = 0; b <= (D == 2 ? 3 : 0); b++)
#pragma unroll
                for (int a = 0; a + b <= 3; a++) RFm[tix(a, b, 3)] += px[a] * py[b] * f;
#pragma unroll
            for (int b = 0; b <= (D == 2 ? 2 : 0); b++)
#pragma unroll
                for (int a = 0; a + b <= 2; a++) RGm[tix(a, b, 2)] += px[a] * py[b] * gp;
        }
        q++;
        double csq = 0.0;
        int base[D];
        double w1[D];
#pragma unroll
        for (int a = 0; a < D; a++) {
            csq += cp[a] * cp[a];
            const double fl = floor(cp[a]);
            base[a] = (int)fl;
            w1[a] = cp[a] - fl;
        }
        dmax2 = fmax(dmax2, csq);
        if (near_wall) {
            deposit_traced(cp, mf, mg);
            return;
        }
        const int ncx = w1[0] > 0.0 ? 2 : 1;
        const int ncy = (D == 2 && w1[D - 1] > 0.0) ? 2 : 1;
        for (int sy = 0; sy < ncy; sy++)
            for (int sx = 0; sx < ncx; sx++) {
                double w = sx ? w1[0] : 1.0 - w1[0];
                if constexpr (D == 2) w *= sy ? w1[1] : 1.0 - w1[1];
                deposit(land<D>(g, cell, lo, n, ix, iy, base[0] + sx, D == 2 ? base[D - 1] + sy : 0), cp, w * mf,
                        w * mg);
            }
    };
    st.for_each_row(row, leaf);
    if constexpr (D == 2) {
        if (absorbed[0] != 0.0 || absorbed[1] != 0.0 || absorbed[2] != 0.0 || absorbed[3] != 0.0)
            noslip_images(m, g, type, Mout, cell, ix, iy, c, st, lf, lg, conF, conG, mfs, mgs, absorbed);
    }
    if (q > ls.q_max) ls.q_max = q;
    ls.points += q;
    ls.walls += walls;
    ls.disp_max2 = fmax(ls.disp_max2, dmax2);
    if constexpr (CHECK) {
        double rmax = 0.0;
        bool finite = true;
#pragma unroll
        for (int j = 0; j < RF; j++) {
            const double r = RFm[tix(bx<D, true>(j), by<D, true>(j), 3)] - conF[j];
            finite = finite && isfinite(r);
            rmax = fmax(rmax, fabs(r));
        }
        if (has_g) {
#pragma unroll
            for (int j = 0; j < RG; j++) {
                const double r = RGm[tix(bx<D, false>(j), by<D, false>(j), 2)] - conG[j];
                finite = finite && isfinite(r);
                rmax = fmax(rmax, fabs(r));
            }
        }
        return finite && rmax <= m.tol;
    }
    return true;
}

// Per-block counters in shared memory, flushed to DevStats once per block.
struct BlockCounters {
    unsigned long long hist[64];
    unsigned long long cells, feq, fmx, q, dmax, pf, pg, pm, p32, redo, retry, walls, mlpc, pdf, pdfc;
};

// Per-thread tallies.
// Per-thread tallies (32-bit: a thread adds them to its block's counters at least once per
// time step, see counters_to_block).
struct ThreadCounters {
    unsigned int cells, pf, pg, p32, redo, retry;
    LocalStats ls;
    unsigned int mlp_cells;
    unsigned int pdf;   // stencil points of double-float streaming passes (mixed path)
    unsigned int pdfc;  // stencil points of double-float correction passes (mixed path)
};

__device__ __forceinline__ void counters_init(BlockCounters& bc) {
    for (int i = threadIdx.x; i < 64; i += blockDim.x) bc.hist[i] = 0;
    if (threadIdx.x == 0)
        bc.cells = bc.feq = bc.fmx = bc.q = bc.dmax = bc.pf = bc.pg = bc.pm = bc.p32 = bc.redo = bc.retry =
            bc.walls = bc.mlpc = bc.pdf = bc.pdfc = 0;
}

// Adds the thread tallies to the block counters, then (after a barrier) the block
// counters to the device counters.  Every thread of the block must call it.
// Adds the thread tallies to the block counters and clears them.
__device__ __forceinline__ void counters_to_block(BlockCounters& bc, ThreadCounters& tc) {
    using ull = unsigned long long;
    atomicAdd(&bc.cells, (ull)tc.cells);
    atomicAdd(&bc.p32, (ull)tc.p32);
    if (tc.redo) atomicAdd(&bc.redo, (ull)tc.redo);
    if (tc.retry) atomicAdd(&bc.retry, (ull)tc.retry);
    if (tc.pf) atomicAdd(&bc.pf, (ull)tc.pf);
    if (tc.pg) atomicAdd(&bc.pg, (ull)tc.pg);
    atomicAdd(&bc.pm, tc.ls.points);
    if (tc.ls.walls) atomicAdd(&bc.walls, (ull)tc.ls.walls);
    if (tc.mlp_cells) atomicAdd(&bc.mlpc, (ull)tc.mlp_cells);
    if (tc.pdf) atomicAdd(&bc.pdf, (ull)tc.pdf);
    if (tc.pdfc) atomicAdd(&bc.pdfc, (ull)tc.pdfc);
    atomicMax(&bc.q, tc.ls.q_max);
    atomicMax(&bc.dmax, (ull)__double_as_longlong(sqrt(tc.ls.disp_max2)));
    tc = ThreadCounters{0, 0, 0, 0, 0, 0, {0, 0.0, 0, 0}, 0, 0, 0};
}

__device__ __forceinline__ void counters_flush(BlockCounters& bc, ThreadCounters& tc, DevStats* stats) {
    counters_to_block(bc, tc);
    __syncthreads();
    for (int i = threadIdx.x; i < 64; i += blockDim.x)
        if (bc.hist[i]) atomicAdd(&stats->newton_hist[i], bc.hist[i]);
    if (threadIdx.x == 0) {
        atomicAdd(&stats->cells, bc.cells);
        atomicAdd(&stats->points_f, bc.pf);
        atomicAdd(&stats->points_g, bc.pg);
        atomicAdd(&stats->points_ms, bc.pm);
        atomicAdd(&stats->points_32, bc.p32);
        if (bc.redo) atomicAdd(&stats->judge_redo, bc.redo);
        if (bc.retry) atomicAdd(&stats->mlp_retry, bc.retry);
        if (bc.walls) atomicAdd(&stats->wall_hits, bc.walls);
        if (bc.mlpc) atomicAdd(&stats->mlp_cells, bc.mlpc);
        if (bc.pdf) atomicAdd(&stats->points_df, bc.pdf);
        if (bc.pdfc) atomicAdd(&stats->points_df_corr, bc.pdfc);
        if (bc.feq) atomicAdd(&stats->fallback_eq, bc.feq);
        if (bc.fmx) atomicAdd(&stats->fallback_mx, bc.fmx);
        atomicMax(&stats->q_max, bc.q);
        atomicMax(&stats->disp_max_bits, bc.dmax);
    }
}

// Entry j of Eq. (IID13) in thermal units: lambda_0 = l0, the second-order diagonal 1/2,
// the rest 0 (the same for the fluon and the phonon basis).
template <int D>
__device__ __forceinline__ float start_base(int j, float l0) {
    const bool diag2 = D == 1 ? j == 2 : (j == 3 || j == 5);
    return j == 0 ? l0 : (diag2 ? 0.5f : 0.f);
}

// The FP64 EPR of one cell from the multipliers lf, lg, with the fallbacks of a failed
// solve (equilibrium constraints, then normalised Maxwellian weights), and its FP64
// streaming pass.
template <int D>
__device__ __forceinline__ void fp64_tail(const Model& m, const Geometry& g, const uint8_t* type, double* Mout,
                                          DevStats* stats, long long cell, BlockCounters& bc,
                                          unsigned int& pf, unsigned int& pg, unsigned int& retry,
                                          LocalStats& ls, double* conF, double* conG, const CellState<D>& c,
                                          const Stencil<D>& st, double* lf, double* lg, bool learned) {
    constexpr int NF = Dim<D>::NF, NG = Dim<D>::NG;
    const bool has_g = m.K > 0.0;
    int sf, sg;
    solve_fg<D>(c, st, conF, conG, has_g, lf, lg, m, sf, sg, pf, pg);
    if ((sf < 0 || sg < 0) && learned) {  // the plain EPR is the fallback of the learned start
        retry++;
        maxwell_start_fg<D, NF, NG>(c.RT, lf, lg);
        solve_fg<D>(c, st, conF, conG, has_g, lf, lg, m, sf, sg, pf, pg);
    }
    if (sf >= 0 && sg >= 0) {
        atomicAdd(&bc.hist[sf < 63 ? sf : 63], 1ull);
        if (has_g) atomicAdd(&bc.hist[sg < 63 ? sg : 63], 1ull);
        if (m.lam_store) {  // the converged multipliers minus Eq. (IID13), as FP32 corrections
            const float l0 = (float)maxwell_l0<D>(c.RT);
#pragma unroll
            for (int j = 0; j < NF; j++)
                m.lam_store[(long long)j * g.ncell + cell] = (float)lf[j] - start_base<D>(j, l0);
#pragma unroll
            for (int j = 0; j < NG; j++)
                m.lam_store[(long long)(NF + j) * g.ncell + cell] = has_g ? (float)lg[j] - start_base<D>(j, l0) : 0.f;
        }
        if (m.rec_x) {  // training pairs: features and converged multipliers minus Eq. (IID13)
            float xin[MlpDims<D>::NIN];
            mlp_features<D>(c, st, xin);
            double mf[NF], mg[NG];
            maxwell_start_fg<D, NF, NG>(c.RT, mf, mg);
#pragma unroll
            for (int k = 0; k < MlpDims<D>::NIN; k++) m.rec_x[cell * MlpDims<D>::NIN + k] = xin[k];
#pragma unroll
            for (int j = 0; j < NF; j++) m.rec_y[cell * MlpDims<D>::NOUT + j] = (float)(lf[j] - mf[j]);
#pragma unroll
            for (int j = 0; j < NG; j++) m.rec_y[cell * MlpDims<D>::NOUT + NF + j] = has_g ? (float)(lg[j] - mg[j]) : 0.f;
        }
    } else {
        // equilibrium constraints (omega = 1) for both populations
#pragma unroll
        for (int j = 0; j < NF; j++) conF[j] = 0.0;
#pragma unroll
        for (int j = 0; j < NG; j++) conG[j] = 0.0;
        conF[0] = conG[0] = 1.0;
        int jj = 1 + D;
#pragma unroll
        for (int a = 0; a < D; a++)
#pragma unroll
            for (int b = a; b < D; b++) {
                conF[jj] = conG[jj] = (a == b) ? 1.0 : 0.0;
                jj++;
            }
        maxwell_start_fg<D, NF, NG>(c.RT, lf, lg);
        solve_fg<D>(c, st, conF, conG, has_g, lf, lg, m, sf, sg, pf, pg);
        if (m.lam_store) {  // a cell solved by a fallback starts from Eq. (IID13) next time
#pragma unroll
            for (int k = 0; k < NF + NG; k++) m.lam_store[(long long)k * g.ncell + cell] = 0.f;
        }
        if (sf >= 0 && sg >= 0) {
            atomicAdd(&bc.feq, 1ull);
        } else {
            // normalised Maxwellian weights: f'_i = dC_i exp(-t^2/2) / S (mass exact)
#pragma unroll
            for (int j = 0; j < NF; j++) lf[j] = 0.0;
            lf[0] = -1.0;
            jj = 1 + D;
#pragma unroll
            for (int a = 0; a < D; a++)
#pragma unroll
                for (int b = a; b < D; b++) {
                    lf[jj] = (a == b) ? 0.5 : 0.0;
                    jj++;
                }
            double MF[MomentSet<D>::NF], MG[MomentSet<D>::NG];
            moment_pass<D>(c, st, lf, lg, true, false, MF, MG);
            lf[0] = log(MF[0]) - 1.0;
#pragma unroll
            for (int j = 0; j < NG; j++) lg[j] = lf[j];
            atomicAdd(&bc.fmx, 1ull);
            atomicMin(&stats->first_fail, (unsigned long long)cell);
        }
    }
    if (m.det_lam) {  // deterministic streaming: the gather kernel deposits from these
#pragma unroll
        for (int j = 0; j < NF; j++) m.det_lam[(long long)j * g.ncell + cell] = lf[j];
#pragma unroll
        for (int j = 0; j < NG; j++) m.det_lam[(long long)(NF + j) * g.ncell + cell] = has_g ? lg[j] : 0.0;
        double umax = 0.0;
#pragma unroll
        for (int a = 0; a < D; a++) umax = fmax(umax, fabs(c.u[a]));
        atomicMax(m.det_halo, (int)ceil(umax + (double)st.R + 0.5) + 1);
        unsigned long long q = 0;  // the velocity set's size and reach, for the counters
        auto count = [&](const double* cp, double) {
            q++;
            double d2 = 0.0;
#pragma unroll
            for (int a = 0; a < D; a++) d2 += cp[a] * cp[a];
            ls.disp_max2 = fmax(ls.disp_max2, d2);
        };
        st.for_each(count);
        if (q > ls.q_max) ls.q_max = q;
        return;
    }
    scatter_cell<D, false>(m, g, type, Mout, cell, c, st, lf, lg, ls, 1.0, conF, conG);
}

struct TailCounts {
    unsigned int pf, pg, retry;
    LocalStats ls;
};

// fp64_tail from Eq. (IID13), out of line, for the FP32 path's rare failed solves; the
// FP32 constraints cf32, cg32 are widened to FP64.
template <int D>
static __device__ __noinline__ TailCounts fp64_tail_cold(const Model& m, const Geometry& g, const uint8_t* type,
                                                         double* Mout, DevStats* stats, long long cell,
                                                         BlockCounters* bc, const float* cf32, const float* cg32,
                                                         CellState<D> c, const Stencil<D> st) {
    TailCounts t{0, 0, 0, {0, 0.0, 0, 0}};
    double conF[Dim<D>::NF], conG[Dim<D>::NG];
#pragma unroll
    for (int j = 0; j < Dim<D>::NF; j++) c.cf[j] = conF[j] = (double)cf32[j];
#pragma unroll
    for (int j = 0; j < Dim<D>::NG; j++) c.cg[j] = conG[j] = (double)cg32[j];
    double lf[Dim<D>::NF], lg[Dim<D>::NG];
    maxwell_start_fg<D, Dim<D>::NF, Dim<D>::NG>(c.RT, lf, lg);
    fp64_tail<D>(m, g, type, Mout, stats, cell, *bc, t.pf, t.pg, t.retry, t.ls, conF, conG, c, st, lf, lg, false);
    return t;
}

// ---------------------------------------------------------------------------
// The mixed path's finish (LELBM_MIXED): FP32 Newton to the FP32 noise floor, then per
// population one double-float correction (residual in double-float, Jacobian in FP32 at
// the same multipliers) and a double-float streaming pass that re-checks the residual of
// exactly the populations it deposits against the FP64 path's tolerance (Sec. II.D).  A
// miss takes the deposit back and corrects again; a second miss leaves the cell to the
// FP64 EPR.
// ---------------------------------------------------------------------------
// Corrects and streams one population.  Returns the number of double-float Newton updates
// (>= 1) once its deposit passed the check, -1 when nothing of it is deposited and the
// FP64 EPR must solve the cell.
template <int D, bool FLUON>
__device__ __forceinline__ int df_population(const Model& m, const CellState<D>& c, const RowTable<D>& tab,
                                             double* lam, const double* con, const float2* etab, double xm,
                                             DFStream& ds, ThreadCounters& tc) {
    using Q = DFPop<D, FLUON>;
    double r[Q::N];
    double rmax;
#pragma unroll 1
    for (int it = 0; it < 2; it++) {
        {
            float MJ[Q::NJ];
            if (!df_pass<D, FLUON, DF_CORR>(c.u[0], c.u[D - 1], c.inv_sig, tab, lam, con, etab, xm, r, rmax, MJ, ds,
                                            tc.ls, tc.pdfc, ds.beta))
                return -1;
            // far from the FP32 solution's neighbourhood (or non-finite): the FP64 EPR decides
            if (!(rmax < 1e-3)) return -1;
            if (rmax > m.tol && !df_update<D, FLUON>(MJ, r, lam)) return -1;
        }
        if (!df_pass<D, FLUON, DF_STREAM>(c.u[0], c.u[D - 1], c.inv_sig, tab, lam, con, etab, xm, r, rmax, nullptr, ds, tc.ls, tc.pdf, ds.beta)) return -1;
        if (rmax <= m.tol) return it + 1;
        // the deposited populations miss the tolerance: take them back
        ds.mh = -ds.mh;
        ds.ml = -ds.ml;
        df_pass<D, FLUON, DF_STREAM>(c.u[0], c.u[D - 1], c.inv_sig, tab, lam, con, etab, xm, r, rmax, nullptr, ds, tc.ls, tc.pdf, ds.beta);
        ds.mh = -ds.mh;
        ds.ml = -ds.ml;
        tc.redo++;
    }
    return -1;
}

// Returns true when the cell is solved and streamed; false leaves the cell, with nothing
// of it deposited, to the FP64 EPR.  Phonons go first: their system is the smaller one, so
// less of it stays live through the fluon passes.
template <int D>
__device__ __forceinline__ bool df_finish(const Model& m, const Geometry& g, const uint8_t* type, double* Mout,
                                          long long cell, BlockCounters& bc, ThreadCounters& tc, const double* conF,
                                          const double* conG, const CellState<D>& c, const Stencil<D>& st,
                                          const RowTable<D>& tab, float* lf32, float* lg32, bool learned,
                                          const float2* etab, long long* bslot) {
    constexpr int NF = Dim<D>::NF, NG = Dim<D>::NG;
    const bool has_g = m.K > 0.0;
    {
        float cf32[NF], cg32[NG];
#pragma unroll
        for (int j = 0; j < NF; j++) cf32[j] = (float)conF[j];
#pragma unroll
        for (int j = 0; j < NG; j++) cg32[j] = (float)conG[j];
        int sf, sg;
        bool ok32 = solve_fg32<D>(c, st, tab, cf32, cg32, has_g, lf32, lg32, sf, sg, tc.p32);
        if (!ok32 && learned) {
            tc.retry++;
            maxwell_start32<D, NF, NG>((float)c.RT, lf32, lg32);
            ok32 = solve_fg32<D>(c, st, tab, cf32, cg32, has_g, lf32, lg32, sf, sg, tc.p32);
        }
        if (!ok32) return false;
    }
    DFStream ds;
    ds.g = &g;
    ds.type = type;
    ds.Mout = Mout;
    ds.cell = cell;
    ds.lo = 0;
    ds.n = 0;
    ds.ix = ds.iy = 0;
    ds.near_wall = false;
    ds.beta = bslot;
    if constexpr (D == 1) {
        const int b = g.inst_of_cell[cell];
        ds.lo = g.inst_lo[b];
        ds.n = g.inst_n[b];
    } else {
        ds.iy = (int)(cell / g.NX);
        ds.ix = (int)(cell - (long long)ds.iy * g.NX);
        // Sec. III.B: trace paths past solid faces where a solid cell lies within reach
        if (g.wall_dist)
            ds.near_wall = (double)g.wall_dist[cell] <= fmax(fabs(c.u[0]), fabs(c.u[1])) + (double)st.R + 1.5;
    }
    const double xm = (double)st.R + 2.0;  // |X|, |Y| of every stencil offset from floor(u)
    double lg[NG];
    int ug = 0;
    if (has_g) {
#pragma unroll
        for (int j = 0; j < NG; j++) lg[j] = (double)lg32[j];
        df_split(c.rho * m.K * c.RT, ds.mh, ds.ml);
        ug = df_population<D, false>(m, c, tab, lg, conG, etab, xm, ds, tc);
        if (ug < 0) return false;
    }
    double lf[NF];
#pragma unroll
    for (int j = 0; j < NF; j++) lf[j] = (double)lf32[j];
    df_split(c.rho, ds.mh, ds.ml);
    const int uf = df_population<D, true>(m, c, tab, lf, conF, etab, xm, ds, tc);
    if (uf < 0) {
        if (has_g) {  // take the phonon deposit back too: the FP64 EPR streams both
            double r[NG], rmax;
            df_split(-(c.rho * m.K * c.RT), ds.mh, ds.ml);
            df_pass<D, false, DF_STREAM>(c.u[0], c.u[D - 1], c.inv_sig, tab, lg, conG, etab, xm, r, rmax, nullptr, ds, tc.ls, tc.pdf, ds.beta);
        }
        return false;
    }
    atomicAdd(&bc.hist[uf], 1ull);
    if (has_g) atomicAdd(&bc.hist[ug], 1ull);
    if (m.lam_store) {  // the converged multipliers minus Eq. (IID13), as FP32 corrections
        const float l0 = (float)maxwell_l0<D>(c.RT);
#pragma unroll
        for (int j = 0; j < NF; j++) m.lam_store[(long long)j * g.ncell + cell] = (float)lf[j] - start_base<D>(j, l0);
#pragma unroll
        for (int j = 0; j < NG; j++)
            m.lam_store[(long long)(NF + j) * g.ncell + cell] = has_g ? (float)lg[j] - start_base<D>(j, l0) : 0.f;
    }
    return true;
}

// The FP64 EPR of one cell from Eq. (IID13), with its fallbacks and its FP64 streaming,
// out of line, for the mixed path's rare cells that the double-float finish leaves.  The
// collision and the stencil are recomputed from the cell's moments in Min (FP64, as in
// the prepare step), so no per-cell value of the hot path stays live for this call;
// conF, conG are the cell's scratch slots.
template <int D>
static __device__ __noinline__ TailCounts fp64_cell_cold(const Model& m, const Geometry& g, const uint8_t* type,
                                                         const double* __restrict__ Min, double* Mout,
                                                         DevStats* stats, long long cell, BlockCounters* bc,
                                                         double* conF, double* conG) {
    TailCounts t{0, 0, 0, {0, 0.0, 0, 0}};
    double M[Dim<D>::NM];
#pragma unroll
    for (int i = 0; i < Dim<D>::NM; i++) M[i] = Min[i * g.ncell + cell];
    CellState<D> c;
    Stencil<D> st;
    collide<D>(M, m, c);
    st.init(c, m);
#pragma unroll
    for (int j = 0; j < Dim<D>::NF; j++) conF[j] = c.cf[j];
#pragma unroll
    for (int j = 0; j < Dim<D>::NG; j++) conG[j] = c.cg[j];
    double lf[Dim<D>::NF], lg[Dim<D>::NG];
    maxwell_start_fg<D, Dim<D>::NF, Dim<D>::NG>(c.RT, lf, lg);
    fp64_tail<D>(m, g, type, Mout, stats, cell, *bc, t.pf, t.pg, t.retry, t.ls, conF, conG, c, st, lf, lg, false);
    return t;
}

// The single-cell operation of Fig. 5 in two halves around the (warp-wide) warm-start
// network: prepare_cell loads the moments, runs the collision module and sets up the
// stencil; finish_cell runs EPR (with the fallbacks) and moment streaming into Mout.
template <int D, int PREC>
__device__ __forceinline__ bool prepare_cell(const Model& m, const Geometry& g, const double* __restrict__ Min,
                                             DevStats* stats, long long cell, BlockCounters& bc, CellState<D>& c,
                                             Stencil<D>& st) {
    constexpr int NM = Dim<D>::NM;
    double M[NM];
#pragma unroll
    for (int i = 0; i < NM; i++) M[i] = Min[i * g.ncell + cell];
    if constexpr (PREC == PREC_FP32)
        collide32<D>(M, m, c);
    else
        collide<D>(M, m, c);
    if (!c.ok) {  // non-physical cell: nothing can be reconstructed
        atomicAdd(&bc.fmx, 1ull);
        atomicMin(&stats->first_fail, (unsigned long long)cell);
        return false;
    }
    if constexpr (PREC == PREC_FP32)
        st.init32(c, m);
    else
        st.init(c, m);
    return true;
}

// dl: the learned correction of the Maxwellian start (fluons then phonons), or null.
template <int D, int PREC>
__device__ __forceinline__ void finish_cell(const Model& m, const Geometry& g, const uint8_t* type,
                                            const double* __restrict__ Min, double* Mout,
                                            DevStats* stats, long long cell, BlockCounters& bc, ThreadCounters& tc,
                                            Con<PREC>* conF, Con<PREC>* conG, const CellState<D>& c, const Stencil<D>& st,
                                            const float* dl, char2* rowbuf, const float2* etab, long long* bslot) {
    constexpr int NF = Dim<D>::NF, NG = Dim<D>::NG;
    tc.cells++;
    const bool has_g = m.K > 0.0;
    float dls[MlpDims<D>::NOUT];
    if (!dl && m.mlp_start) {  // the learned start of this step, from mlp_start_kernel
        dls[0] = m.mlp_start[cell];
        if (isfinite(dls[0])) {  // a NaN first row: the kernel left the cell to Eq. (IID13)
#pragma unroll
            for (int k = 1; k < MlpDims<D>::NOUT; k++) dls[k] = m.mlp_start[(long long)k * g.ncell + cell];
            dl = dls;
            tc.mlp_cells++;
        }
    }
    double lf[NF], lg[NG];
    float lf32[NF], lg32[NG];  // the FP32 path's multipliers
    bool learned = false;
    bool dl_ok = dl != nullptr;
    if (dl) {
#pragma unroll
        for (int k = 0; k < MlpDims<D>::NOUT; k++) dl_ok = dl_ok && isfinite(dl[k]);
    }
    // the FP32 Newton's start (FP32 and mixed paths); RT in FP32 (the FP32 path has its own)
    const float rt32 = PREC == PREC_FP32 ? c.RT32 : (float)c.RT;
    if constexpr (PREC != PREC_FP64) {
        maxwell_start32<D, NF, NG>(rt32, lf32, lg32);
        if (dl_ok) {
#pragma unroll
            for (int j = 0; j < NF; j++) lf32[j] += dl[j];
            if (has_g) {
#pragma unroll
                for (int j = 0; j < NG; j++) lg32[j] += dl[NF + j];
            }
            learned = true;
        } else if (m.lam_store) {  // the correction this cell kept from its last step
            bool fin = true;
#pragma unroll
            for (int j = 0; j < NF; j++) {
                const float v = m.lam_store[(long long)j * g.ncell + cell];
                fin = fin && isfinite(v);
                lf32[j] += v;
            }
            if (has_g) {
#pragma unroll
                for (int j = 0; j < NG; j++) {
                    const float v = m.lam_store[(long long)(NF + j) * g.ncell + cell];
                    fin = fin && isfinite(v);
                    lg32[j] += v;
                }
            }
            learned = fin;
            if (!fin) maxwell_start32<D, NF, NG>(rt32, lf32, lg32);
        }
    } else {
        maxwell_start_fg<D, NF, NG>(c.RT, lf, lg);
        if (dl_ok) {
#pragma unroll
            for (int j = 0; j < NF; j++) lf[j] += (double)dl[j];
            if (has_g) {
#pragma unroll
                for (int j = 0; j < NG; j++) lg[j] += (double)dl[NF + j];
            }
            learned = true;
        } else if (m.lam_store) {
            bool fin = true;
#pragma unroll
            for (int j = 0; j < NF; j++) {
                const float v = m.lam_store[(long long)j * g.ncell + cell];
                fin = fin && isfinite(v);
                lf[j] += (double)v;
            }
            if (has_g) {
#pragma unroll
                for (int j = 0; j < NG; j++) {
                    const float v = m.lam_store[(long long)(NF + j) * g.ncell + cell];
                    fin = fin && isfinite(v);
                    lg[j] += (double)v;
                }
            }
            learned = fin;
            if (!fin) maxwell_start_fg<D, NF, NG>(c.RT, lf, lg);
        }
    }
#pragma unroll
    for (int j = 0; j < NF; j++) conF[j] = PREC == PREC_FP32 ? c.cf32[j] : c.cf[j];
#pragma unroll
    for (int j = 0; j < NG; j++) conG[j] = PREC == PREC_FP32 ? c.cg32[j] : c.cg[j];
    int sf, sg;
    RowTable<D> tab;
    if constexpr (PREC == PREC_FP32)
        tab.build32(c, st, rowbuf);
    else if constexpr (PREC == PREC_MIXED)
        tab.build(c, st, rowbuf);
    if constexpr (PREC == PREC_FP32) {
        // FP32 Newton and FP32 streaming; the plain FP64 EPR is the fallback
        bool ok32 = solve_fg32<D>(c, st, tab, conF, conG, has_g, lf32, lg32, sf, sg, tc.p32);
        if (!ok32 && learned) {
            tc.retry++;
            maxwell_start32<D, NF, NG>(c.RT32, lf32, lg32);
            learned = false;
            ok32 = solve_fg32<D>(c, st, tab, conF, conG, has_g, lf32, lg32, sf, sg, tc.p32);
        }
        if (ok32) {
            atomicAdd(&bc.hist[sf < 63 ? sf : 63], 1ull);
            if (has_g) atomicAdd(&bc.hist[sg < 63 ? sg : 63], 1ull);
            if (m.lam_store) {  // the converged multipliers minus Eq. (IID13), for the next step
                const float l0 = -1.f + 0.5f * D * logf(6.2831853071795865f * c.RT32);
#pragma unroll
                for (int j = 0; j < NF; j++)
                    m.lam_store[(long long)j * g.ncell + cell] = lf32[j] - start_base<D>(j, l0);
#pragma unroll
                for (int j = 0; j < NG; j++)
                    m.lam_store[(long long)(NF + j) * g.ncell + cell] = has_g ? lg32[j] - start_base<D>(j, l0) : 0.f;
            }
            scatter_cell32<D>(m, g, type, Mout, cell, c, st, tab, lf32, lg32, tc.ls);
            return;
        }
        // the plain FP64 EPR, out of line: it is rare, and inline it would shape the
        // register allocation of the whole FP32 path
        tc.redo++;
        const TailCounts t = fp64_tail_cold<D>(m, g, type, Mout, stats, cell, &bc, conF, conG, c, st);
        tc.pf += t.pf;
        tc.pg += t.pg;
        tc.retry += t.retry;
        if (t.ls.q_max > tc.ls.q_max) tc.ls.q_max = t.ls.q_max;
        tc.ls.points += t.ls.points;
        tc.ls.walls += t.ls.walls;
        tc.ls.disp_max2 = fmax(tc.ls.disp_max2, t.ls.disp_max2);
    } else {
        if constexpr (PREC == PREC_MIXED) {
            // FP32 Newton, double-float correction and streaming judged at the FP64
            // tolerance; the FP64 EPR (out of line) takes the cells it leaves
            if (tab.ok && df_finish<D>(m, g, type, Mout, cell, bc, tc, conF, conG, c, st, tab, lf32, lg32, learned,
                                       etab, bslot))
                return;
            tc.redo++;
            const TailCounts t = fp64_cell_cold<D>(m, g, type, Min, Mout, stats, cell, &bc, conF, conG);
            tc.pf += t.pf;
            tc.pg += t.pg;
            tc.retry += t.retry;
            if (t.ls.q_max > tc.ls.q_max) tc.ls.q_max = t.ls.q_max;
            tc.ls.points += t.ls.points;
            tc.ls.walls += t.ls.walls;
            tc.ls.disp_max2 = fmax(tc.ls.disp_max2, t.ls.disp_max2);
            return;
        }
        fp64_tail<D>(m, g, type, Mout, stats, cell, bc, tc.pf, tc.pg, tc.retry, tc.ls, conF, conG, c, st, lf, lg,
                     learned);
    }
}

// The mixed path's FP32 Newton phase (row table only), out of line: its moment
// accumulators then have the register file to themselves.  Constraints come from the
// cell's FP64 scratch slots; lf32, lg32 hold the start and receive the solution.
template <int D>
static __device__ __noinline__ bool fp32_phase(const RowTable<D>& tab_in, const double* conF, const double* conG,
                                               bool has_g, float* lf32_io, float* lg32_io, float rt32, bool learned,
                                               unsigned int& np32, unsigned int& retry) {
    constexpr int NF = Dim<D>::NF, NG = Dim<D>::NG;
    const RowTable<D> tab = tab_in;
    CellState<D> c;  // not read: the row table carries the geometry
    Stencil<D> st;
    float cf32[NF], cg32[NG], lf32[NF], lg32[NG];
#pragma unroll
    for (int j = 0; j < NF; j++) {
        cf32[j] = (float)conF[j];
        lf32[j] = lf32_io[j];
    }
#pragma unroll
    for (int j = 0; j < NG; j++) {
        cg32[j] = (float)conG[j];
        lg32[j] = lg32_io[j];
    }
    unsigned int np = 0;
    int sf, sg;
    bool ok = solve_fg32<D, true>(c, st, tab, cf32, cg32, has_g, lf32, lg32, sf, sg, np);
    if (!ok && learned) {
        retry++;
        maxwell_start32<D, NF, NG>(rt32, lf32, lg32);
        ok = solve_fg32<D, true>(c, st, tab, cf32, cg32, has_g, lf32, lg32, sf, sg, np);
    }
    np32 += np;
#pragma unroll
    for (int j = 0; j < NF; j++) lf32_io[j] = lf32[j];
#pragma unroll
    for (int j = 0; j < NG; j++) lg32_io[j] = lg32[j];
    return ok;
}

// The mixed path's cell update in block-synchronous phases.  The 128 cells a block claims go
// together through (1) the collision, stencil set-up, warm start and row table, (2) the
// FP32 Newton, (3) the phonons' and (4) the fluons' double-float correction and streaming,
// with a block barrier between phases: the warps of a block then run the same code at the
// same time, which keeps the instruction working set of an SM to a few phases.  Every
// thread of the block calls this, active or not.
// INLINE_MLP: the warm-start network runs here, warp-wide (the persistent 1D batch); the
// cell-update kernel instead reads the corrections mlp_start_kernel wrote (m.mlp_start).
// Barrier of the threads that step a chunk of cells together: the whole block
// (nthreads = blockDim.x), or one group of nthreads threads (hardware barrier 1 + group).
__device__ __forceinline__ void group_sync(int group, int nthreads) {
    if (nthreads == (int)blockDim.x)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(1 + group), "r"(nthreads) : "memory");
}

template <int D, bool INLINE_MLP>
__device__ __forceinline__ void mixed_block(const Model& m, const Geometry& g, const uint8_t* type,
                                            const double* __restrict__ Min, double* Mout, DevStats* stats,
                                            long long cell, bool active, BlockCounters& bc, ThreadCounters& tc,
                                            double* conF, double* conG, char2* rowbuf, const float2* etab,
                                            long long* bslot, unsigned char* s_mlp, bool mlp, int group,
                                            int gthreads) {
    constexpr int NF = Dim<D>::NF, NG = Dim<D>::NG;
    const bool has_g = m.K > 0.0;
    CellState<D> c;
    Stencil<D> st;
    bool ok = false;
    if (active) ok = prepare_cell<D, PREC_MIXED>(m, g, Min, stats, cell, bc, c, st);
    float lf32[NF], lg32[NG];
    bool learned = false;
    {
        float dl[MlpDims<D>::NOUT];
        if constexpr (INLINE_MLP) {
            if (mlp) {  // warp-uniform: every lane takes part in the tensor-core inference
                float xin[MlpDims<D>::NIN];
                if (ok) mlp_features<D, false>(c, st, xin);
                warp_mlp<D>(s_mlp, xin, ok, dl);
                if (ok) tc.mlp_cells++;
            }
        } else {
            mlp = m.mlp_start != nullptr && ok;
            if (mlp) {  // a NaN first row: the network's kernel left the cell to Eq. (IID13)
                dl[0] = m.mlp_start[cell];
                mlp = isfinite(dl[0]);
            }
            if (mlp) {
#pragma unroll
                for (int k = 1; k < MlpDims<D>::NOUT; k++) dl[k] = m.mlp_start[(long long)k * g.ncell + cell];
                tc.mlp_cells++;
            }
        }
        if (ok) {
            tc.cells++;
            // Eq. (IID13) in FP32, plus the learned or the stored correction
            maxwell_start32<D, NF, NG>((float)c.RT, lf32, lg32);
            bool fin = true;
            if (mlp) {
#pragma unroll
                for (int k = 0; k < MlpDims<D>::NOUT; k++) fin = fin && isfinite(dl[k]);
                if (fin) {
#pragma unroll
                    for (int j = 0; j < NF; j++) lf32[j] += dl[j];
                    if (has_g) {
#pragma unroll
                        for (int j = 0; j < NG; j++) lg32[j] += dl[NF + j];
                    }
                    learned = true;
                }
            } else if (m.lam_store) {
#pragma unroll
                for (int j = 0; j < NF; j++) {
                    const float v = m.lam_store[(long long)j * g.ncell + cell];
                    fin = fin && isfinite(v);
                    lf32[j] += v;
                }
                if (has_g) {
#pragma unroll
                    for (int j = 0; j < NG; j++) {
                        const float v = m.lam_store[(long long)(NF + j) * g.ncell + cell];
                        fin = fin && isfinite(v);
                        lg32[j] += v;
                    }
                }
                learned = fin;
                if (!fin) maxwell_start32<D, NF, NG>((float)c.RT, lf32, lg32);
            }
#pragma unroll
            for (int j = 0; j < NF; j++) conF[j] = c.cf[j];
#pragma unroll
            for (int j = 0; j < NG; j++) conG[j] = c.cg[j];
        }
    }
    RowTable<D> tab;
    if (ok) tab.build(c, st, rowbuf);
    bool alive = ok && tab.ok;
    group_sync(group, gthreads);
    // (2) FP32 Newton to the FP32 noise floor
    if (alive) alive = fp32_phase<D>(tab, conF, conG, has_g, lf32, lg32, (float)c.RT, learned, tc.p32, tc.retry);
    group_sync(group, gthreads);
    DFStream ds;
    ds.g = &g;
    ds.type = type;
    ds.Mout = Mout;
    ds.cell = cell;
    ds.lo = 0;
    ds.n = 0;
    ds.ix = ds.iy = 0;
    ds.near_wall = false;
    ds.beta = bslot;
    ds.mh = ds.ml = 0.f;
    double xm = 0.0;
    if (alive) {
        if constexpr (D == 1) {
            const int b = g.inst_of_cell[cell];
            ds.lo = g.inst_lo[b];
            ds.n = g.inst_n[b];
        } else {
            ds.iy = (int)(cell / g.NX);
            ds.ix = (int)(cell - (long long)ds.iy * g.NX);
            // Sec. III.B: trace paths past solid faces where a solid cell lies within reach
            if (g.wall_dist)
                ds.near_wall = (double)g.wall_dist[cell] <= fmax(fabs(c.u[0]), fabs(c.u[1])) + (double)st.R + 1.5;
        }
        xm = (double)st.R + 2.0;  // |X|, |Y| of every stencil offset from floor(u)
    }
    // (3) phonons
    double lg[NG];
    int ug = 0;
    if (alive && has_g) {
#pragma unroll
        for (int j = 0; j < NG; j++) lg[j] = (double)lg32[j];
        df_split(c.rho * m.K * c.RT, ds.mh, ds.ml);
        ug = df_population<D, false>(m, c, tab, lg, conG, etab, xm, ds, tc);
        alive = ug >= 0;
    }
    group_sync(group, gthreads);
    // (4) fluons
    double lf[NF];
    int uf = 0;
    if (alive) {
#pragma unroll
        for (int j = 0; j < NF; j++) lf[j] = (double)lf32[j];
        df_split(c.rho, ds.mh, ds.ml);
        uf = df_population<D, true>(m, c, tab, lf, conF, etab, xm, ds, tc);
        if (uf < 0) {
            alive = false;
            if (has_g) {  // take the phonon deposit back too: the FP64 EPR streams both
                double r[NG], rmax;
                df_split(-(c.rho * m.K * c.RT), ds.mh, ds.ml);
                df_pass<D, false, DF_STREAM>(c.u[0], c.u[D - 1], c.inv_sig, tab, lg, conG, etab, xm, r, rmax,
                                             nullptr, ds, tc.ls, tc.pdf, ds.beta);
            }
        }
    }
    if (alive) {
        atomicAdd(&bc.hist[uf], 1ull);
        if (has_g) atomicAdd(&bc.hist[ug], 1ull);
        if (m.lam_store) {  // the converged multipliers minus Eq. (IID13), as FP32 corrections
            const float l0 = (float)maxwell_l0<D>(c.RT);
#pragma unroll
            for (int j = 0; j < NF; j++)
                m.lam_store[(long long)j * g.ncell + cell] = (float)lf[j] - start_base<D>(j, l0);
#pragma unroll
            for (int j = 0; j < NG; j++)
                m.lam_store[(long long)(NF + j) * g.ncell + cell] = has_g ? (float)lg[j] - start_base<D>(j, l0) : 0.f;
        }
    } else if (ok) {
        // the FP64 EPR, out of line, for the rare cells left: no row table (more refinement
        // levels or rows than it holds), a failed FP32 phase or a missed check
        tc.redo++;
        const TailCounts t = fp64_cell_cold<D>(m, g, type, Min, Mout, stats, cell, &bc, conF, conG);
        tc.pf += t.pf;
        tc.pg += t.pg;
        tc.retry += t.retry;
        if (t.ls.q_max > tc.ls.q_max) tc.ls.q_max = t.ls.q_max;
        tc.ls.points += t.ls.points;
        tc.ls.walls += t.ls.walls;
        tc.ls.disp_max2 = fmax(tc.ls.disp_max2, t.ls.disp_max2);
    }
}

// One time step of the whole padded grid: warps claim chunks of 32 consecutive cells
// from a global counter (the cost of a cell varies with its temperature, q ~
// (n sqrt RT)^D, so a static split leaves SMs idle at the end).
// Blocks per SM the compiler must fit (registers): the FP32 variants, whose FP64 fallback
// is out of line and whose per-thread tallies live in shared memory, are light enough in
// their hot path for four 128-thread blocks (128 registers); the rest keep the full
// register file.
// Groups of the mixed path's block that claim and step their cells independently, each
// with its own phase barriers: fewer warps wait at a barrier for the slowest one, while at
// most two phases share an SM's instruction caches.  Two groups of six warps measured 4.8 %
// faster than one group of twelve on the 4096^2 four-quadrant problem; three groups of four
// were 12 % slower.
constexpr int kMixedGroups = 2;

template <int D, int PREC>
constexpr int min_blocks() { return PREC == PREC_FP32 ? 4 : (PREC == PREC_MIXED ? 1 : 1); }

template <int D, int PREC>
__global__ void __launch_bounds__(cell_threads<PREC>(), min_blocks<D, PREC>()) cell_update_kernel(const __grid_constant__ Model m, const __grid_constant__ Geometry g,
                                                          const uint8_t* __restrict__ type,
                                                          const double* __restrict__ Min, double* Mout,
                                                          DevStats* stats, unsigned long long* work) {
    constexpr int NF = Dim<D>::NF, NG = Dim<D>::NG;
    __shared__ BlockCounters bc;
    constexpr int NT = cell_threads<PREC>();
    __shared__ Con<PREC> s_con[NT][NF + NG];  // constraints of each thread's cell (out of registers)
    // 2D row tables of the FP32 passes (one per thread)
    __shared__ char2 s_rows[(D == 2 && PREC != PREC_FP64) ? NT : 1][(D == 2 && PREC != PREC_FP64) ? kRowsMax : 1];
    Con<PREC>* conF = s_con[threadIdx.x];
    Con<PREC>* conG = conF + NF;
    char2* rowbuf = (D == 2 && PREC != PREC_FP64) ? s_rows[threadIdx.x] : nullptr;
    // double-float table of 2^(j/512) (mixed path)
    __shared__ float2 s_exp[PREC == PREC_MIXED ? kExpTab : 1];
    __shared__ long long s_beta[PREC == PREC_MIXED ? NT : 1][DFPop<D, true>::NB];  // exponent coefficients
    if (PREC == PREC_MIXED) exp2_table_init(s_exp);
    counters_init(bc);
    __syncthreads();
    // per-thread tallies in shared memory: a dozen 64-bit counters kept in registers across
    // the whole cell update would cost the hot path registers or spills
    __shared__ ThreadCounters s_tc[NT];
    s_tc[threadIdx.x] = ThreadCounters{0, 0, 0, 0, 0, 0, {0, 0.0, 0, 0}, 0, 0, 0};
    ThreadCounters& tc = s_tc[threadIdx.x];
    const int lane = threadIdx.x & 31;
    if constexpr (PREC == PREC_MIXED) {  // groups claim G-cell chunks and step them in phases
        constexpr int G = NT / kMixedGroups;
        const int grp = threadIdx.x / G, gl = threadIdx.x - grp * G;
        __shared__ unsigned long long s_base[kMixedGroups];
        for (;;) {
            if (gl == 0) s_base[grp] = atomicAdd(work, (unsigned long long)G);
            group_sync(grp, G);
            const unsigned long long base = s_base[grp];
            group_sync(grp, G);
            if (base >= (unsigned long long)g.ncell) break;
            const long long cell = (long long)base + gl;
            const bool active = cell < g.ncell && type[cell] != CELL_SOLID;
            mixed_block<D, false>(m, g, type, Min, Mout, stats, cell, active, bc, tc, conF, conG, rowbuf, s_exp,
                                  s_beta[threadIdx.x], nullptr, false, grp, G);
        }
        counters_flush(bc, tc, stats);
        return;
    }
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(work, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= (unsigned long long)g.ncell) break;
        const long long cell = (long long)base + lane;
        const bool active = cell < g.ncell && type[cell] != CELL_SOLID;
        CellState<D> c;
        Stencil<D> st;
        bool ok = false;
        if (active) ok = prepare_cell<D, PREC>(m, g, Min, stats, cell, bc, c, st);
        if (ok)
            finish_cell<D, PREC>(m, g, type, Min, Mout, stats, cell, bc, tc, conF, conG, c, st, nullptr, rowbuf, s_exp,
                                 PREC == PREC_MIXED ? s_beta[threadIdx.x] : nullptr);
    }
    counters_flush(bc, tc, stats);
}

// Persistent 1D batch: a block claims a whole instance from the queue (order[]) and
// runs all of its steps with block barriers only -- instances share no cells, so no
// grid-wide barrier is needed.  Each step fills the instance's pads (Sec. III.A),
// zeroes its block of the next buffer, then lets its warps claim 32-cell chunks from
// a shared counter.  An instance that ends on an odd step copies its block back, so
// every instance finishes in buffer A.  steps_left[] (may be null: unlimited) caps
// each instance and is decremented.
// The persistent batch keeps 128-thread blocks (a block per instance); on the mixed path
// three of them per SM (168 registers), as many as the FP32 variant fits at 128.
template <int PREC>
constexpr int batch_min_blocks() { return PREC == PREC_MIXED ? 3 : min_blocks<1, PREC>(); }

template <int PREC>
__global__ void __launch_bounds__(128, batch_min_blocks<PREC>()) batch_persistent_kernel(const __grid_constant__ Model m,
                                                               const __grid_constant__ Geometry g, double in0, double in1,
                                                               double in3, int bc_left_inflow, int bc_right_inflow,
                                                               const uint8_t* __restrict__ type, double* A, double* B,
                                                               DevStats* stats, unsigned long long* work,
                                                               const int* order, const long long* inst_first,
                                                               const int* inst_pad, int* steps_left, int nsteps) {
    constexpr int D = 1, NM = Dim<1>::NM, NF = Dim<1>::NF, NG = Dim<1>::NG;
    __shared__ BlockCounters bc;
    __shared__ Con<PREC> s_con[128][NF + NG];
    __shared__ unsigned int s_next;
    __shared__ int s_inst;
    extern __shared__ __align__(16) unsigned char s_mlp[];  // warm-start network (when set)
    Con<PREC>* conF = s_con[threadIdx.x];
    Con<PREC>* conG = conF + NF;
    __shared__ float2 s_exp[PREC == PREC_MIXED ? kExpTab : 1];  // double-float 2^(j/512) (mixed path)
    __shared__ long long s_beta[PREC == PREC_MIXED ? 128 : 1][DFPop<1, true>::NB];  // exponent coefficients
    if (PREC == PREC_MIXED) exp2_table_init(s_exp);
    counters_init(bc);
    const bool mlp = m.mlp_w != nullptr;
    if (mlp) mlp_stage_mma<1>(s_mlp, m.mlp_w, m.mlp_nrm);
    // per-thread tallies in shared memory: a dozen 64-bit counters kept in registers across
    // the whole cell update would cost the hot path registers or spills
    __shared__ ThreadCounters s_tc[128];
    s_tc[threadIdx.x] = ThreadCounters{0, 0, 0, 0, 0, 0, {0, 0.0, 0, 0}, 0, 0, 0};
    ThreadCounters& tc = s_tc[threadIdx.x];
    const int lane = threadIdx.x & 31;
    double Meq[NM];
    {
        const double uin[1] = {in1};
        eq_moments<1>(m.K, in0, uin, in3, Meq);
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned long long k = atomicAdd(work, 1ull);
            s_inst = k < (unsigned long long)g.n_inst ? order[k] : -1;
        }
        __syncthreads();
        const int b = s_inst;
        if (b < 0) break;
        const int n = g.inst_n[b];
        const int pad = inst_pad[b];
        const long long lo = g.inst_lo[b];
        const long long first = inst_first[b];
        const int nblk = n + 2 * pad;
        int k = nsteps;
        if (steps_left) k = min(k, steps_left[b]);
        for (int s = 0; s < k; s++) {
            const double* Min = (s & 1) ? B : A;
            double* Mout = (s & 1) ? A : B;
            // pads, then a zeroed output block
            for (int i = threadIdx.x; i < 2 * pad; i += blockDim.x) {
                const bool left = i < pad;
                const long long cell = left ? first + i : lo + n + (i - pad);
                double* Mw = const_cast<double*>(Min);
                if (left ? bc_left_inflow : bc_right_inflow) {
#pragma unroll
                    for (int q = 0; q < NM; q++) Mw[q * g.ncell + cell] = Meq[q];
                } else {
                    const long long src = left ? lo : lo + n - 1;
#pragma unroll
                    for (int q = 0; q < NM; q++) Mw[q * g.ncell + cell] = Min[q * g.ncell + src];
                }
            }
            for (int i = threadIdx.x; i < nblk; i += blockDim.x)
#pragma unroll
                for (int q = 0; q < NM; q++) Mout[q * g.ncell + first + i] = 0.0;
            if (threadIdx.x == 0) s_next = 0;
            __syncthreads();
            if constexpr (PREC == PREC_MIXED) {  // block-wide chunks, stepped in phases
                for (;;) {
                    __shared__ unsigned int s_base;
                    if (threadIdx.x == 0) {
                        s_base = s_next;
                        s_next += blockDim.x;
                    }
                    __syncthreads();
                    const unsigned int base = s_base;
                    __syncthreads();
                    if (base >= (unsigned int)nblk) break;
                    const int i = (int)base + (int)threadIdx.x;
                    const long long cell = first + i;
                    const bool active = i < nblk && type[cell] != CELL_SOLID;
                    mixed_block<D, true>(m, g, type, Min, Mout, stats, cell, active, bc, tc, conF, conG, nullptr,
                                         s_exp, s_beta[threadIdx.x], s_mlp, mlp, 0, (int)blockDim.x);
                }
            }
            for (; PREC != PREC_MIXED;) {
                unsigned int base = 0;
                if (lane == 0) base = atomicAdd(&s_next, 32u);
                base = __shfl_sync(0xffffffffu, base, 0);
                if (base >= (unsigned int)nblk) break;
                const int i = (int)base + lane;
                const long long cell = first + i;
                const bool active = i < nblk && type[cell] != CELL_SOLID;
                CellState<D> c;
                Stencil<D> st;
                bool ok = false;
                if (active) ok = prepare_cell<D, PREC>(m, g, Min, stats, cell, bc, c, st);
                float dl[MlpDims<D>::NOUT];
                const bool use_mlp = mlp;
                if (use_mlp) {
                    float xin[MlpDims<D>::NIN];
                    if (ok) mlp_features<D, PREC == PREC_FP32>(c, st, xin);
                    warp_mlp<D>(s_mlp, xin, ok, dl);
                    if (ok) tc.mlp_cells++;
                }
                if (ok)
                    finish_cell<D, PREC>(m, g, type, Min, Mout, stats, cell, bc, tc, conF, conG, c, st,
                                         use_mlp ? dl : nullptr, nullptr, s_exp, PREC == PREC_MIXED ? s_beta[threadIdx.x] : nullptr);
            }
            counters_to_block(bc, tc);  // keeps the 32-bit tallies of a long launch small
            __syncthreads();
        }
        if (k & 1) {  // the result is in B: copy the block back to A
            for (int i = threadIdx.x; i < nblk; i += blockDim.x)
#pragma unroll
                for (int q = 0; q < NM; q++) A[q * g.ncell + first + i] = B[q * g.ncell + first + i];
        }
        if (steps_left && threadIdx.x == 0) steps_left[b] -= k;
    }
    counters_flush(bc, tc, stats);
}

}  // namespace lbm
