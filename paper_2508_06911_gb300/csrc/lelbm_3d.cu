// The LELBM time step in three dimensions (the paper's general-D formulation, Sec. II,
// with D = 3: 17 stored moments, N_f = 19 fluon and N_g = 10 phonon constraints, Eq.
// IIB5, IIB14-IIB17), FP64, fluid boundaries only (Sec. III.A).
//
// One warp per cell.  A 3D velocity set holds hundreds of points (q ~ (4/3) pi (R_ac +
// 1/2)^3, 180 at RT = 0.5, 380 at RT = 1) and its Jacobians (19 x 19 and 10 x 10) do not
// fit one thread's registers, so the 32 lanes share a cell:
//   - the LAS stencil (Eq. IIC6, IIC9-IIC11) is laid out as row items in shared memory:
//     each item is a run of points along x at fixed (y, z), level-0 runs with spacing 1
//     and the children of split points as runs with spacing 2^-L (Eq. IIC10-IIC11);
//   - a Newton pass (Eq. IID7-IID11) gives each lane one item at a time: it evaluates the
//     populations along the run (the exponent is a cubic in x on the run) and their row
//     sums sum x^a f (a <= 6 for fluons, <= 4 for phonons); the lanes then fold the row
//     sums of 32 items into the population moments x^a y^b z^c f that make up the residual
//     and the Jacobian (84 fluon and 35 phonon monomials, a few per lane);
//   - the Cholesky factorisation and solve are shared by the lanes of the warp;
//   - moment streaming (Eq. IIE3) deposits T_N(c_i) rho f'_i and T_N(c_i) rho K RT g'_i
//     at x + c_i with FP64 atomic additions (cloud-in-cell for refined children).
// Thermal units throughout the Newton (t = (c - u) / sqrt(RT)), as in 1D and 2D.
#include <cuda_runtime.h>

#include <cstdint>

#include "lelbm_device.cuh"
#include "lelbm_internal.h"

namespace lbm {

constexpr int kW3Warps = 4;           // warps (cells in flight) per block
constexpr int kW3Items = 1024;        // row items per cell (R_ac up to about 16, RT ~ 16)
constexpr int kNF3 = 19, kNG3 = 10;   // constraints
constexpr int kPF3 = 6, kPG3 = 4;     // degree of the Jacobian moments
constexpr int kMF3 = 84, kMG3 = 35;   // monomials x^a y^b z^c of degree <= 6, <= 4
constexpr int kMon3 = kMF3 + kMG3;
constexpr int kSub = 64;              // item coordinates in units of 1/64 cell

// Exponents of the fluon basis T_j (Eq. IIB14-IIB16): 1, t_a, t_a t_b (a <= b), and the
// heat-flux entries t_a^2 t_g ordered g-major; the phonon basis is the first ten.
__device__ __constant__ int8_t c_bex[kNF3] = {0, 1, 0, 0, 2, 1, 1, 0, 0, 0, 3, 1, 1, 2, 0, 0, 2, 0, 0};
__device__ __constant__ int8_t c_bey[kNF3] = {0, 0, 1, 0, 0, 1, 0, 2, 1, 0, 0, 2, 0, 1, 3, 1, 0, 2, 0};
__device__ __constant__ int8_t c_bez[kNF3] = {0, 0, 0, 1, 0, 0, 1, 0, 1, 2, 0, 0, 2, 0, 0, 2, 1, 1, 3};

// Position of x^a y^b z^c among the monomials of degree <= P, ordered by c, then b, then a.
__device__ __forceinline__ int mon_index(int a, int b, int c, int P) {
    int idx = 0;
    for (int cc = 0; cc < c; cc++) {
        const int m = P - cc;
        idx += (m + 1) * (m + 2) / 2;
    }
    const int m = P - c;
    for (int bb = 0; bb < b; bb++) idx += m - bb + 1;
    return idx + a;
}

// Position of y^b z^c (b + c <= 6) in a row's table of transverse monomials.
__device__ __forceinline__ int yz_index(int b, int c) { return c * 7 - c * (c - 1) / 2 + b; }

// One run of stencil points: c = (x + k h, y, z) for k = 0..n-1, h = 2^-level, all in
// units of 1/64 cell; dC = 2^(-3 level) (Eq. IIC11).
struct Item3 {
    short x, y, z, nl;  // nl = n | level << 12
};

struct Warp3 {
    Item3 items[kW3Items];
    double S[32][12];     // row sums of a chunk: fluon x^0..6, phonon x^0..4
    double YZ[32][28];    // y^b z^c (b + c <= 6) of the chunk's rows (thermal units), yz_index
    double MF[kMF3];      // population moments of the fluons
    double MG[kMG3];      // and of the phonons
    double A[kNF3 * kNF3];
    double Ag[kNG3 * kNG3];
    double rf[kNF3], rg[kNG3];
    double lf[kNF3], lg[kNG3];
    double cf[kNF3], cg[kNG3];
    int n_items;
    int flag;
};

// ---------------------------------------------------------------------------
// LAS stencil as row items (Eq. IIC6, IIC9-IIC11), with the membership tests of the 1D
// and 2D stencils: squared distances summed x, y, z with one rounding each.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dist2_3(double x, double y, double z, const double* u) {
    const double dx = __dsub_rn(x, u[0]), dy = __dsub_rn(y, u[1]), dz = __dsub_rn(z, u[2]);
    return __dadd_rn(__dadd_rn(__dadd_rn(0.0, __dmul_rn(dx, dx)), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// The run of points x_k = x0 + k h (k = 0..n-1) at (y, z) within r2 of u: [k0, k1]
// (empty when k0 > k1).  The test is monotone in |x - u_x| along the run, so the set is an
// interval; its ends are found from the real-valued chord and then checked exactly.
__device__ __forceinline__ void run_band(double x0, double h, int n, double y, double z, const double* u, double r2,
                                         int& k0, int& k1) {
    k0 = 1;
    k1 = 0;
    const double dy = __dsub_rn(y, u[1]), dz = __dsub_rn(z, u[2]);
    // the test at x = u_x: every point of the run has at least this squared distance
    const double yz2 = __dadd_rn(__dmul_rn(dy, dy), __dmul_rn(dz, dz));
    if (yz2 > r2) return;
    const double s = sqrt(r2 - yz2);
    k0 = (int)floor((u[0] - s - x0) / h) - 1;
    k1 = (int)ceil((u[0] + s - x0) / h) + 1;
    k0 = k0 < 0 ? 0 : k0;
    k1 = k1 > n - 1 ? n - 1 : k1;
    while (k0 <= k1 && dist2_3(x0 + k0 * h, y, z, u) > r2) k0++;
    while (k1 >= k0 && dist2_3(x0 + k1 * h, y, z, u) > r2) k1--;
}

// Emits the items of one level-0 row (cy, cz): the unsplit runs and, recursively, the
// child runs of its split points.  count_only: only counts.  Returns the item count.
template <bool WRITE>
__device__ int row_items(int cy, int cz, const double* u, const Stencil<3>& st, Item3* out, int cap) {
    int cnt = 0;
    auto emit = [&](double x, double y, double z, int n, int level) {
        if (WRITE && cnt < cap) {
            Item3 it;
            it.x = (short)rint(x * kSub);
            it.y = (short)rint(y * kSub);
            it.z = (short)rint(z * kSub);
            it.nl = (short)(n | (level << 12));
            out[cnt] = it;
        }
        cnt++;
    };
    const double y = cy, z = cz;
    const double rr = sqrt(st.rr2);
    const int xlo = (int)floor(u[0] - rr) - 1, xhi = (int)ceil(u[0] + rr) + 1;
    int a0, a1;
    run_band((double)xlo, 1.0, xhi - xlo + 1, y, z, u, st.rr2, a0, a1);
    if (a0 > a1) return 0;
    // stack of child runs still to split: (x0, y, z, n, level)
    struct Run {
        double x, y, z;
        int n, level;
    };
    Run stack[16];
    int sp = 0;
    Run top{(double)(xlo + a0), y, z, a1 - a0 + 1, 0};
    for (;;) {
        const double h = ldexp(1.0, -top.level);
        int b0 = 1, b1 = 0;
        if (top.level < st.Nr) run_band(top.x, h, top.n, top.y, top.z, u, st.rad2[top.level + 1], b0, b1);
        if (b0 > b1) {
            emit(top.x, top.y, top.z, top.n, top.level);
        } else {
            if (b0 > 0) emit(top.x, top.y, top.z, b0, top.level);
            if (b1 < top.n - 1) emit(top.x + (b1 + 1) * h, top.y, top.z, top.n - 1 - b1, top.level);
            // children of the split points at +-h/4 per axis: four child runs of spacing h/2
            const double q = 0.25 * h;
            for (int s = 3; s >= 0; s--) {
                if (sp < 16)
                    stack[sp++] = Run{top.x + b0 * h - q, top.y + ((s & 1) ? q : -q), top.z + ((s & 2) ? q : -q),
                                      2 * (b1 - b0 + 1), top.level + 1};
            }
        }
        if (sp == 0) break;
        top = stack[--sp];
    }
    return cnt;
}

// Lays the cell's velocity set out as items in w->items (deterministic order: level-0
// rows by z, then y); returns the total count (more than kW3Items: the set does not fit)
// and the number of points in *q.
__device__ int build_items(Warp3* w, const double* u, const Stencil<3>& st, int lane, long long* q) {
    const double rr = sqrt(st.rr2);
    const int y0 = (int)floor(u[1] - rr) - 1, y1 = (int)ceil(u[1] + rr) + 1;
    const int z0 = (int)floor(u[2] - rr) - 1, z1 = (int)ceil(u[2] + rr) + 1;
    const int ny = y1 - y0 + 1, ncand = ny * (z1 - z0 + 1);
    int total = 0;
    long long pts = 0;
    for (int base = 0; base < ncand; base += 32) {
        const int idx = base + lane;
        const int cy = y0 + idx % ny, cz = z0 + idx / ny;
        const int cnt = idx < ncand ? row_items<false>(cy, cz, u, st, nullptr, 0) : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int off = total + incl - cnt;
        if (cnt > 0 && off < kW3Items) row_items<true>(cy, cz, u, st, w->items + off, kW3Items - off);
        total += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    const int n = total < kW3Items ? total : kW3Items;
    for (int i = lane; i < n; i += 32) pts += w->items[i].nl & 0xfff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pts += __shfl_xor_sync(0xffffffffu, pts, o);
    *q = pts;
    return total;
}

// Geometry of item i in thermal units: first x, spacing, y, z and the volume element.
struct ItemGeo {
    double tx, th, ty, tz, dC;
    int n, level;
    double cx, cy, cz, h;  // lattice frame: first velocity and spacing
};

__device__ __forceinline__ ItemGeo item_geo(const Item3& it, const CellState<3>& c) {
    ItemGeo g;
    g.n = it.nl & 0xfff;
    g.level = it.nl >> 12;
    g.h = ldexp(1.0, -g.level);
    g.dC = ldexp(1.0, -3 * g.level);
    g.cx = it.x * (1.0 / kSub);
    g.cy = it.y * (1.0 / kSub);
    g.cz = it.z * (1.0 / kSub);
    g.tx = (g.cx - c.u[0]) * c.inv_sig;
    g.ty = (g.cy - c.u[1]) * c.inv_sig;
    g.tz = (g.cz - c.u[2]) * c.inv_sig;
    g.th = g.h * c.inv_sig;
    return g;
}

// Coefficients of 1 + sum_j lam_j T_j as a cubic (fluons) or quadratic (phonons) in x on
// the run at (ty, tz).
__device__ __forceinline__ void run_coeffs(const double* lf, const double* lg, double ty, double tz, double* cf,
                                           double* cg) {
    double yp[4], zp[4];
    yp[0] = zp[0] = 1.0;
#pragma unroll
    for (int k = 1; k < 4; k++) {
        yp[k] = yp[k - 1] * ty;
        zp[k] = zp[k - 1] * tz;
    }
#pragma unroll
    for (int k = 0; k < 4; k++) cf[k] = 0.0;
#pragma unroll
    for (int k = 0; k < 3; k++) cg[k] = 0.0;
    cf[0] = 1.0;
    cg[0] = 1.0;
#pragma unroll
    for (int j = 0; j < kNF3; j++) cf[c_bex[j]] += lf[j] * (yp[c_bey[j]] * zp[c_bez[j]]);
#pragma unroll
    for (int j = 0; j < kNG3; j++) cg[c_bex[j]] += lg[j] * (yp[c_bey[j]] * zp[c_bez[j]]);
}

// One Newton pass over the velocity set: the population moments x^a y^b z^c f of degree
// <= 6 (fluons, if doF) and <= 4 (phonons, if doG) into w->MF, w->MG.
__device__ void moment_pass3(Warp3* w, const CellState<3>& c, int n_items, bool doF, bool doG, int lane,
                             const int* ma, const int* mb, const int* mcz, const int* msel, int nown,
                             unsigned long long& npts) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int base = 0; base < n_items; base += 32) {
        const int i = base + lane;
        if (i < n_items) {
            const ItemGeo gi = item_geo(w->items[i], c);
            double cf[4], cg[3];
            run_coeffs(w->lf, w->lg, gi.ty, gi.tz, cf, cg);
            double Sf[7], Sg[5];
#pragma unroll
            for (int a = 0; a < 7; a++) Sf[a] = 0.0;
#pragma unroll
            for (int a = 0; a < 5; a++) Sg[a] = 0.0;
            auto point = [&](int, double x, double f, double g) {
                double pf = f * gi.dC, pg = g * gi.dC;
#pragma unroll
                for (int a = 0; a < 7; a++) {
                    Sf[a] += pf;
                    pf *= x;
                }
#pragma unroll
                for (int a = 0; a < 5; a++) {
                    Sg[a] += pg;
                    pg *= x;
                }
            };
            row_eval(cf, cg, doF, doG, gi.tx, gi.th, gi.n, point);
            npts += (unsigned long long)gi.n;
#pragma unroll
            for (int a = 0; a < 7; a++) w->S[lane][a] = Sf[a];
#pragma unroll
            for (int a = 0; a < 5; a++) w->S[lane][7 + a] = Sg[a];
            // the row's transverse monomials, once per row (the lanes then need one product
            // per monomial and row)
            double yp[7];
            yp[0] = 1.0;
#pragma unroll
            for (int k = 1; k < 7; k++) yp[k] = yp[k - 1] * gi.ty;
            double zp = 1.0;
#pragma unroll
            for (int cz = 0; cz < 7; cz++) {
#pragma unroll
                for (int b = 0; b + cz < 7; b++) w->YZ[lane][yz_index(b, cz)] = yp[b] * zp;
                zp *= gi.tz;
            }
        }
        __syncwarp();
        const int nr = n_items - base < 32 ? n_items - base : 32;
        bool act[4];
        int si[4], yi[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            act[k] = k < nown && ((msel[k] == 0 && doF) || (msel[k] == 1 && doG));
            si[k] = k < nown ? (msel[k] ? 7 : 0) + ma[k] : 0;
            yi[k] = k < nown ? yz_index(mb[k], mcz[k]) : 0;
        }
        for (int r = 0; r < nr; r++) {
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (act[k]) acc[k] = fma(w->S[r][si[k]], w->YZ[r][yi[k]], acc[k]);
        }
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (k < nown) {
            const int e = lane + 32 * k;
            if (msel[k] == 0 && doF) w->MF[e] = acc[k];
            if (msel[k] == 1 && doG) w->MG[e - kMF3] = acc[k];
        }
    }
    __syncwarp();
}

// Cholesky factorisation A = L L^T (row-major N x N, lower triangle) and solve A x = b,
// shared by the lanes of a warp; b is overwritten by x.  Returns false on a non-positive
// pivot (the same test as the oracle's plain factorisation).
__device__ bool warp_chol_solve(double* A, double* b, int N, int lane) {
    for (int k = 0; k < N; k++) {
        __syncwarp();
        const double akk = A[k * N + k];
        if (!(akk > 0.0)) return false;
        const double d = sqrt(akk);
        __syncwarp();
        if (lane == 0) A[k * N + k] = d;
        for (int i = k + 1 + lane; i < N; i += 32) A[i * N + k] /= d;
        __syncwarp();
        for (int i = k + 1; i < N; i++) {
            const double lik = A[i * N + k];
            for (int j = k + 1 + lane; j <= i; j += 32) A[i * N + j] -= lik * A[j * N + k];
        }
    }
    __syncwarp();
    for (int k = 0; k < N; k++) {  // L y = b
        const double yk = b[k] / A[k * N + k];
        __syncwarp();
        if (lane == 0) b[k] = yk;
        for (int i = k + 1 + lane; i < N; i += 32) b[i] -= A[i * N + k] * yk;
        __syncwarp();
    }
    for (int k = N - 1; k >= 0; k--) {  // L^T x = y
        const double xk = b[k] / A[k * N + k];
        __syncwarp();
        if (lane == 0) b[k] = xk;
        for (int i = lane; i < k; i += 32) b[i] -= A[k * N + i] * xk;
        __syncwarp();
    }
    return true;
}

// Residual and Newton update of one population from its moments (Eq. IID9-IID11):
// N = 19, P = 6 (fluons) or N = 10, P = 4 (phonons).  Returns 1 when the population has
// converged (the update just applied is the polishing one), 0 to go on, -1 on a
// breakdown and -2 at the iteration cap (the oracle's Newton loop).
__device__ int newton_update3(const double* Mom, const double* con, double* lam, double* A, double* r, int N, int P,
                              int it, double tol, int max_iter, int lane) {
    double rj = 0.0;
    if (lane < N) {
        rj = Mom[mon_index(c_bex[lane], c_bey[lane], c_bez[lane], P)] - con[lane];
        r[lane] = rj;
    }
    double rmax = lane < N ? fabs(rj) : 0.0;
    bool fin = lane < N ? isfinite(rj) : true;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    fin = __all_sync(0xffffffffu, fin);
    if (!fin) return -1;
    const bool conv = rmax <= tol;
    if (!conv && it >= max_iter) return -2;
    for (int e = lane; e < N * N; e += 32) {
        const int i = e / N, j = e - (e / N) * N;
        A[e] = Mom[mon_index(c_bex[i] + c_bex[j], c_bey[i] + c_bey[j], c_bez[i] + c_bez[j], P)];
    }
    __syncwarp();
    if (!warp_chol_solve(A, r, N, lane)) return -1;
    bool ok = true;
    if (lane < N) {
        lam[lane] += r[lane];
        ok = isfinite(lam[lane]);
    }
    ok = __all_sync(0xffffffffu, ok);
    __syncwarp();
    if (!ok) return -1;
    return conv ? 1 : 0;
}

// EPR of both populations (Eq. IID7-IID11) from the multipliers in w->lf, w->lg and the
// constraints in w->cf, w->cg.  sf, sg: Newton updates (>= 0) or -1 / -2.
__device__ void solve3(Warp3* w, const CellState<3>& c, const Model& m, bool has_g, int n_items, int lane,
                       const int* ma, const int* mb, const int* mcz, const int* msel, int nown, int& sf, int& sg,
                       unsigned long long& np_f, unsigned long long& np_g) {
    bool actF = true, actG = has_g;
    int uf = 0, ug = 0;
    sf = 0;
    sg = 0;
    for (int it = 0; actF || actG; it++) {
        unsigned long long np = 0;
        moment_pass3(w, c, n_items, actF, actG, lane, ma, mb, mcz, msel, nown, np);
        if (actF) np_f += np;
        if (actG) np_g += np;
        if (actF) {
            const int s = newton_update3(w->MF, w->cf, w->lf, w->A, w->rf, kNF3, kPF3, it, m.tol, m.max_iter, lane);
            if (s < 0) {
                sf = s;
                actF = false;
            } else {
                uf++;
                if (s == 1) {
                    sf = uf;
                    actF = false;
                }
            }
        }
        if (actG) {
            const int s = newton_update3(w->MG, w->cg, w->lg, w->Ag, w->rg, kNG3, kPG3, it, m.tol, m.max_iter, lane);
            if (s < 0) {
                sg = s;
                actG = false;
            } else {
                ug++;
                if (s == 1) {
                    sg = ug;
                    actG = false;
                }
            }
        }
        __syncwarp();
    }
}

__device__ __forceinline__ int land_axis3(int i, int n, int pad, int periodic) {
    if (periodic) {
        const int r = i % n;
        return r < 0 ? r + n : r;
    }
    return (i < pad || i >= pad + n) ? -1 : i;
}

// Moment streaming (Eq. IIE3) of the cell's populations with the multipliers in w->lf,
// w->lg: T_N(c_i) rho f'_i and T_N(c_i) rho K RT g'_i added at x + c_i; a refined child
// landing between cells is shared by cloud-in-cell weights; what lands on a pad or outside
// the grid is discarded.
__device__ void stream3(Warp3* w, const CellState<3>& c, const Model& m, const Geometry3& g, double* Mout, int ix,
                        int iy, int iz, int n_items, bool has_g, int lane, unsigned long long& nms, double& disp2) {
    const double ms = c.rho, gs = c.rho * m.K * c.RT;
    for (int i = lane; i < n_items; i += 32) {
        const ItemGeo gi = item_geo(w->items[i], c);
        double cf[4], cg[3];
        run_coeffs(w->lf, w->lg, gi.ty, gi.tz, cf, cg);
        auto point = [&](int k, double, double f, double gg) {
            const double cx = gi.cx + k * gi.h, cy = gi.cy, cz = gi.cz;
            const double mf = ms * (f * gi.dC), mg = has_g ? gs * (gg * gi.dC) : 0.0;
            const double csq = cx * cx + cy * cy + cz * cz;
            disp2 = fmax(disp2, csq);
            double dM[17];
            dM[0] = mf;
            dM[1] = cx * mf;
            dM[2] = cy * mf;
            dM[3] = cz * mf;
            dM[4] = cx * cx * mf;
            dM[5] = cx * cy * mf;
            dM[6] = cx * cz * mf;
            dM[7] = cy * cy * mf;
            dM[8] = cy * cz * mf;
            dM[9] = cz * cz * mf;
            dM[10] = csq * cx * mf;
            dM[11] = csq * cy * mf;
            dM[12] = csq * cz * mf;
            dM[13] = mg;
            dM[14] = cx * mg;
            dM[15] = cy * mg;
            dM[16] = cz * mg;
            const double pos[3] = {ix + cx, iy + cy, iz + cz};
            int i0[3];
            double w1[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const double fl = floor(pos[a]);
                i0[a] = (int)fl;
                w1[a] = pos[a] - fl;
            }
            const int ncx = w1[0] > 0.0 ? 2 : 1, ncy = w1[1] > 0.0 ? 2 : 1, ncz = w1[2] > 0.0 ? 2 : 1;
            for (int sz = 0; sz < ncz; sz++)
                for (int sy = 0; sy < ncy; sy++)
                    for (int sx = 0; sx < ncx; sx++) {
                        const int tx = land_axis3(i0[0] + sx, g.nx, g.px, g.periodic[0]);
                        const int ty = land_axis3(i0[1] + sy, g.ny, g.py, g.periodic[1]);
                        const int tz = land_axis3(i0[2] + sz, g.nz, g.pz, g.periodic[2]);
                        if (tx < 0 || ty < 0 || tz < 0) continue;
                        const double wgt = (sx ? w1[0] : 1.0 - w1[0]) * (sy ? w1[1] : 1.0 - w1[1]) *
                                           (sz ? w1[2] : 1.0 - w1[2]);
                        const long long t = ((long long)tz * g.NY + ty) * g.NX + tx;
#pragma unroll
                        for (int q = 0; q < 17; q++) atomicAdd(&Mout[q * g.ncell + t], wgt * dM[q]);
                    }
        };
        row_eval(cf, cg, true, has_g, gi.tx, gi.th, gi.n, point);
        nms += (unsigned long long)gi.n;
    }
}

// The monomials this lane accumulates: entries lane, lane + 32, ... of the list of the
// 84 fluon monomials (degree <= 6) followed by the 35 phonon ones (degree <= 4).
__device__ __forceinline__ int own_monomials(int lane, int* ma, int* mb, int* mcz, int* msel) {
    int nown = 0;
    for (int k = 0; k < 4; k++) {
        const int e = lane + 32 * k;
        if (e >= kMon3) break;
        const int P = e < kMF3 ? kPF3 : kPG3;
        int t = e < kMF3 ? e : e - kMF3;
        for (int cz = 0; cz <= P; cz++)
            for (int by = 0; by <= P - cz; by++)
                for (int ax = 0; ax <= P - cz - by; ax++) {
                    if (t == 0) {
                        ma[k] = ax;
                        mb[k] = by;
                        mcz[k] = cz;
                    }
                    t--;
                }
        msel[k] = e < kMF3 ? 0 : 1;
        nown++;
    }
    return nown;
}

// Eq. (IID13) in thermal units, with the constraints of the collision (or, for the
// fallback, of the equilibrium: omega = 1).
__device__ __forceinline__ void start3(Warp3* w, const CellState<3>& c, bool equilibrium, int lane) {
    double lf[kNF3], lg[kNG3];
    maxwell_start_fg<3, kNF3, kNG3>(c.RT, lf, lg);
    if (lane < kNF3) {
        w->lf[lane] = lf[lane];
        double v = c.cf[lane];
        if (equilibrium) v = lane == 0 ? 1.0 : ((lane == 4 || lane == 7 || lane == 9) ? 1.0 : 0.0);
        w->cf[lane] = v;
    }
    if (lane < kNG3) {
        w->lg[lane] = lg[lane];
        double v = c.cg[lane];
        if (equilibrium) v = lane == 0 ? 1.0 : ((lane == 4 || lane == 7 || lane == 9) ? 1.0 : 0.0);
        w->cg[lane] = v;
    }
    __syncwarp();
}

// One time step of every cell of a padded 3D grid: each warp claims cells from a global
// counter and runs the single-cell operation (collision, LAS, EPR, moment streaming).
__global__ void __launch_bounds__(kW3Warps * 32) cell3d_kernel(const __grid_constant__ Model m,
                                                               const __grid_constant__ Geometry3 g,
                                                               const double* __restrict__ Min, double* Mout,
                                                               DevStats* stats, unsigned long long* work) {
    extern __shared__ __align__(16) unsigned char smem3[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    Warp3* w = reinterpret_cast<Warp3*>(smem3) + wid;
    int ma[4], mb[4], mcz[4], msel[4];
    const int nown = own_monomials(lane, ma, mb, mcz, msel);
    const bool has_g = m.K > 0.0;
    unsigned long long n_cells = 0, np_f = 0, np_g = 0, n_ms = 0, q_max = 0, feq = 0, fmx = 0;
    unsigned long long hist[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double disp2 = 0.0;
    for (;;) {
        long long cell = 0;
        if (lane == 0) cell = (long long)atomicAdd(work, 1ull);
        cell = __shfl_sync(0xffffffffu, cell, 0);
        if (cell >= g.ncell) break;
        const double v = lane < 17 ? Min[(long long)lane * g.ncell + cell] : 0.0;
        double M[17];
#pragma unroll
        for (int i = 0; i < 17; i++) M[i] = __shfl_sync(0xffffffffu, v, i);
        CellState<3> c;
        collide<3>(M, m, c);
        if (!c.ok) {  // non-physical cell: nothing can be reconstructed
            if (lane == 0) {
                fmx++;
                atomicMin(&stats->first_fail, (unsigned long long)cell);
            }
            continue;
        }
        Stencil<3> st;
        st.init(c, m);
        // item coordinates are 16-bit multiples of 1/64: |c| < 512
        const double reach = fmax(fabs(c.u[0]), fmax(fabs(c.u[1]), fabs(c.u[2]))) + (double)st.R + 3.0;
        long long q = 0;
        const int total = reach < 500.0 ? build_items(w, c.u, st, lane, &q) : kW3Items + 1;
        if (total > kW3Items) {  // velocity set beyond the item table: reported, not streamed
            if (lane == 0) {
                fmx++;
                atomicMin(&stats->first_fail, (unsigned long long)cell);
            }
            __syncwarp();
            continue;
        }
        n_cells++;
        q_max = q_max > (unsigned long long)q ? q_max : (unsigned long long)q;
        start3(w, c, false, lane);
        int sf, sg;
        solve3(w, c, m, has_g, total, lane, ma, mb, mcz, msel, nown, sf, sg, np_f, np_g);
        if (sf >= 0 && sg >= 0) {
            hist[sf < 7 ? sf : 7]++;
            if (has_g) hist[sg < 7 ? sg : 7]++;
        } else {
            // equilibrium constraints (omega = 1) for both populations
            start3(w, c, true, lane);
            solve3(w, c, m, has_g, total, lane, ma, mb, mcz, msel, nown, sf, sg, np_f, np_g);
            if (sf >= 0 && sg >= 0) {
                feq++;
            } else {
                // normalised Maxwellian weights: f'_i = g'_i = dC_i exp(-t^2 / 2) / S
                if (lane < kNF3) w->lf[lane] = lane == 0 ? -1.0 : ((lane == 4 || lane == 7 || lane == 9) ? 0.5 : 0.0);
                __syncwarp();
                unsigned long long np = 0;
                moment_pass3(w, c, total, true, false, lane, ma, mb, mcz, msel, nown, np);
                const double S = w->MF[0];
                __syncwarp();
                if (lane == 0) w->lf[0] = log(S) - 1.0;
                __syncwarp();
                if (lane < kNG3) w->lg[lane] = w->lf[lane];
                __syncwarp();
                fmx++;
                if (lane == 0) atomicMin(&stats->first_fail, (unsigned long long)cell);
            }
        }
        const long long pl = (long long)g.NX * g.NY;
        const int iz = (int)(cell / pl);
        const long long rem = cell - (long long)iz * pl;
        const int iy = (int)(rem / g.NX), ix = (int)(rem - (long long)iy * g.NX);
        stream3(w, c, m, g, Mout, ix, iy, iz, total, has_g, lane, n_ms, disp2);
        __syncwarp();
    }
    // counters: lane 0 holds the per-cell tallies, every lane its streamed points
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_ms += __shfl_xor_sync(0xffffffffu, n_ms, o);
        disp2 = fmax(disp2, __shfl_xor_sync(0xffffffffu, disp2, o));
    }
    if (lane == 0) {
        atomicAdd(&stats->cells, n_cells);
        atomicAdd(&stats->points_f, np_f);
        atomicAdd(&stats->points_g, np_g);
        atomicAdd(&stats->points_ms, n_ms);
        atomicAdd(&stats->fallback_eq, feq);
        atomicAdd(&stats->fallback_mx, fmx);
        atomicMax(&stats->q_max, q_max);
        atomicMax(&stats->disp_max_bits, (unsigned long long)__double_as_longlong(sqrt(disp2)));
        for (int i = 0; i < 8; i++)
            if (hist[i]) atomicAdd(&stats->newton_hist[i], hist[i]);
    }
}

// Boundary fill of the 3D pads (Sec. III.A): inflow pads hold the equilibrium of the
// inflow state, the others copy the nearest interior cell.
__global__ void fill_pads3_kernel(double K, double r_in, double ux, double uy, double uz, double RT_in, double* M,
                                  long long ncell, const long long* pad_cell, const long long* pad_src,
                                  long long npad) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < npad;
         k += (long long)gridDim.x * blockDim.x) {
        const long long dst = pad_cell[k], src = pad_src[k];
        if (src < 0) {
            const double u[3] = {ux, uy, uz};
            double Me[17];
            eq_moments<3>(K, r_in, u, RT_in, Me);
#pragma unroll
            for (int i = 0; i < 17; i++) M[i * ncell + dst] = Me[i];
        } else {
#pragma unroll
            for (int i = 0; i < 17; i++) M[i * ncell + dst] = M[i * ncell + src];
        }
    }
}

void launch_fill_pads3(const Model& m, const double inlet[5], double* M, long long ncell, const long long* pad_cell,
                       const long long* pad_src, long long npad, cudaStream_t s) {
    if (npad == 0) return;
    long long b = (npad + 255) / 256;
    if (b > 65535LL * 32) b = 65535LL * 32;
    fill_pads3_kernel<<<(int)b, 256, 0, s>>>(m.K, inlet[0], inlet[1], inlet[2], inlet[3], inlet[4], M, ncell, pad_cell,
                                            pad_src, npad);
}

int cell3d_blocks(int device) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(cell3d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(Warp3) * kW3Warps));
        attr_set = true;
    }
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cell3d_kernel, kW3Warps * 32, sizeof(Warp3) * kW3Warps);
    return sms * (per_sm < 1 ? 1 : per_sm);
}

void launch_cell3d(const Model& m, const Geometry3& g, const double* Min, double* Mout, DevStats* st,
                   unsigned long long* work, int blocks, cudaStream_t s) {
    cell3d_kernel<<<blocks, kW3Warps * 32, sizeof(Warp3) * kW3Warps, s>>>(m, g, Min, Mout, st, work);
}

}  // namespace lbm
