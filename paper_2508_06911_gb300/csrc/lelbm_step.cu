// Device code of the LELBM time step (arXiv:2508.06911) for sm_103a.
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

#include <cfloat>
#include <cstdint>

#include "lelbm_internal.h"

namespace lbm {

template <int D>
struct Dim;
template <>
struct Dim<1> {
    static constexpr int NM = 6, NF = 4, NG = 3;
};
template <>
struct Dim<2> {
    static constexpr int NM = 11, NF = 10, NG = 6;
};

// Stored-moment positions, Eq. (IIB5).
template <int D>
__device__ __forceinline__ constexpr int iM2(int a, int b) {
    return D == 1 ? 2 : (a == 0 && b == 0 ? 3 : (a == 1 && b == 1 ? 5 : 4));
}
template <int D>
__device__ __forceinline__ constexpr int iMD(int g) {
    return D == 1 ? 3 : 6 + g;
}
template <int D>
__device__ __forceinline__ constexpr int iG0() {
    return D == 1 ? 4 : 8;
}
template <int D>
__device__ __forceinline__ constexpr int iG1(int g) {
    return D == 1 ? 5 : 9 + g;
}

// ---------------------------------------------------------------------------
// Collision module: Eq. (IIB6), (IIB9)-(IIB18), App. C (C7)-(C8), App. D.
// ---------------------------------------------------------------------------
template <int D>
struct CellState {
    double rho, u[D], RT, sig, inv_sig;
    double cf[Dim<D>::NF];  // fluon constraints in thermal units
    double cg[Dim<D>::NG];  // phonon constraints in thermal units
    bool ok;
};

template <int D>
__device__ __forceinline__ void collide(const double* M, const Model& m, CellState<D>& c) {
    constexpr int NF = Dim<D>::NF, NG = Dim<D>::NG;
    const double K = m.K;
    // Eq. (IIB6), with the operation order of a plain loop and one rounding each.
    const double rho = M[0];
    double usq = 0.0, tr = 0.0;
#pragma unroll
    for (int a = 0; a < D; a++) {
        c.u[a] = __ddiv_rn(M[1 + a], rho);
        usq = __dadd_rn(usq, __dmul_rn(c.u[a], c.u[a]));
        tr = __dadd_rn(tr, M[iM2<D>(a, a)]);
    }
    const double RT = __ddiv_rn(__dsub_rn(__ddiv_rn(__dadd_rn(tr, M[iG0<D>()]), rho), usq),
                                __dadd_rn((double)D, K));
    c.rho = rho;
    c.RT = RT;
    c.ok = rho > 0.0 && RT > 0.0 && isfinite(rho) && isfinite(RT);
    if (!c.ok) return;
    c.sig = sqrt(RT);
    c.inv_sig = 1.0 / c.sig;

    // Eq. (IIB9): non-equilibrium central moments.
    double P[D][D];
#pragma unroll
    for (int a = 0; a < D; a++)
#pragma unroll
        for (int b = 0; b < D; b++)
            P[a][b] = M[iM2<D>(a, b)] - rho * (c.u[a] * c.u[b] + (a == b ? RT : 0.0));
    double trP = 0.0;
#pragma unroll
    for (int a = 0; a < D; a++) trP += P[a][a];
    double Q[D];
#pragma unroll
    for (int g = 0; g < D; g++) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < D; a++) s += c.u[a] * P[a][g];
        Q[g] = M[iMD<D>(g)] - 2.0 * s - c.u[g] * trP - rho * (usq + (D + 2) * RT) * c.u[g];
    }
    const double G0 = M[iG0<D>()];
    const double G0n = G0 - rho * K * RT;
    double Gn[D];
#pragma unroll
    for (int g = 0; g < D; g++) Gn[g] = M[iG1<D>(g)] - c.u[g] * G0;

    // App. C: implicit collision frequencies from the kinematic coefficients.
    const double inv_f = m.nu_s / RT + 0.5;
    double wf = 1.0 / inv_f;
    const double fb = 2.0 / D - 2.0 / (D + K);
    double wb = (m.nu_b < 0.0 || fb <= 0.0) ? 1.0 : 1.0 / (m.nu_b / (RT * fb) + 0.5);
    double wh = 1.0 / ((inv_f - 0.5) / m.Pr + 0.5);

    // App. D: Knudsen number (moments normalised by rho) and limiter.
    if (m.limiter) {
        double s2 = 0.0, s3 = 0.0;
        const double ir = 1.0 / rho;
#pragma unroll
        for (int a = 0; a < D; a++)
#pragma unroll
            for (int b = 0; b < D; b++) s2 += fabs(P[a][b] * ir);
        s2 += fabs(G0n * ir);
#pragma unroll
        for (int g = 0; g < D; g++) s3 += fabs(Q[g] * ir) + fabs(Gn[g] * ir);
        const double k2 = s2 / ((D + K) * RT);
        const double k3 = s3 / ((D + K + 2) * RT * c.sig);
        const double Kn = fmax(k2, k3);
        if (Kn > 0.0) {
            const double ks = log10(Kn);
            if (ks >= -1.0) {
                wf = wb = wh = 1.0;
            } else if (ks > -2.0) {
                const double x = ks + 2.0;
                wf += (1.0 - wf) * x;
                wb += (1.0 - wb) * x;
                wh += (1.0 - wh) * x;
            }
        }
    }

    // Eq. (IIB10)-(IIB18), then divided by sqrt(RT)^order (thermal units).
    const double bulk = -G0n / D;
    const double ir = 1.0 / rho;
    const double iRT = 1.0 / RT;
    c.cf[0] = 1.0;
#pragma unroll
    for (int a = 0; a < D; a++) c.cf[1 + a] = 0.0;
    int j = 1 + D;
#pragma unroll
    for (int a = 0; a < D; a++)
#pragma unroll
        for (int b = a; b < D; b++) {
            const double sh = P[a][b] - (a == b ? bulk : 0.0);
            const double mm = (a == b ? rho * RT : 0.0) + (1.0 - wf) * sh + (1.0 - wb) * (a == b ? bulk : 0.0);
            c.cf[j++] = mm * ir * iRT;
        }
    const double s3 = iRT * c.inv_sig;
#pragma unroll
    for (int g = 0; g < D; g++)
#pragma unroll
        for (int a = 0; a < D; a++) c.cf[j++] = (1.0 - wh) * ((1.0 + 2.0 * (a == g)) / (D + 2) * Q[g]) * ir * s3;
    (void)NF;
    if (K > 0.0) {
        const double nrm = 1.0 / (rho * K * RT);
        c.cg[0] = (rho * K * RT + (1.0 - wb) * G0n) * nrm;
#pragma unroll
        for (int g = 0; g < D; g++) c.cg[1 + g] = (1.0 - wh) * Gn[g] * nrm * c.inv_sig;
        int k = 1 + D;
#pragma unroll
        for (int a = 0; a < D; a++)
#pragma unroll
            for (int b = a; b < D; b++) c.cg[k++] = (a == b) ? 1.0 : 0.0;  // Eq. (IIB17) / RT
    } else {
#pragma unroll
        for (int k = 0; k < NG; k++) c.cg[k] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// LAS module: Eq. (IIC6), (IIC9)-(IIC11).  Level-0 points are the integer
// velocities within R_ac + 1/2 of u; for Lvl = 1..N_r a point of level Lvl-1
// within refine_rad * 0.5^Lvl of u is split into 2^D children at +-h/4.
// ---------------------------------------------------------------------------
template <int D>
struct Stencil {
    double u[D];
    double rr2;      // (R_ac + 1/2)^2
    int R;           // acoustic radius
    int Nr;          // refinement levels
    double rad2[5];  // squared refinement radius of level 1..4 (index = level)

    __device__ __forceinline__ void init(const CellState<D>& c, const Model& m) {
#pragma unroll
        for (int a = 0; a < D; a++) u[a] = c.u[a];
        double r = round(__dmul_rn(m.n_conf, c.sig));
        if (r < m.r_min) r = m.r_min;
        R = (int)r;
        const double rr = (double)R + 0.5;
        rr2 = rr * rr;
        double nr = round(__ddiv_rn(1.0, __dmul_rn(m.refine_div, c.sig)));
        if (nr > (double)m.max_refine) nr = (double)m.max_refine;
        Nr = (int)nr;
#pragma unroll
        for (int L = 0; L < 5; L++) {
            const double rad = m.refine_rad * ldexp(1.0, -L);
            rad2[L] = rad * rad;
        }
    }

    __device__ __forceinline__ double dist2(const double* c) const {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < D; a++) {
            const double d = __dsub_rn(c[a], u[a]);
            s = __dadd_rn(s, __dmul_rn(d, d));
        }
        return s;
    }

    // Visit one level-0 point and its refinement subtree.
    template <class F>
    __device__ __forceinline__ void visit0(const double* c0, F& f) const {
        if (Nr == 0 || dist2(c0) > rad2[1]) {
            f(c0, 1.0);
            return;
        }
        const int nfine = 1 << (D * Nr);
        for (int idx = 0; idx < nfine; idx++) {
            double ctr[D];
#pragma unroll
            for (int a = 0; a < D; a++) ctr[a] = c0[a];
            double h = 1.0;
            int L = 0;
            while (L < Nr && dist2(ctr) <= rad2[L + 1]) {
#pragma unroll
                for (int a = 0; a < D; a++) {
                    const int bit = (idx >> (a * Nr + (Nr - 1 - L))) & 1;
                    ctr[a] += bit ? 0.25 * h : -0.25 * h;
                }
                h *= 0.5;
                L++;
            }
            const int mask = (1 << (Nr - L)) - 1;
            bool first = true;
#pragma unroll
            for (int a = 0; a < D; a++) first = first && (((idx >> (a * Nr)) & mask) == 0);
            if (first) f(ctr, ldexp(1.0, -D * L));
        }
    }

    template <class F>
    __device__ __forceinline__ void for_each(F& f) const {
        const double rr = sqrt(rr2);
        if constexpr (D == 1) {
            int x0 = (int)floor(u[0] - rr) - 1, x1 = (int)ceil(u[0] + rr) + 1;
            for (int cx = x0; cx <= x1; cx++) {
                const double c[1] = {(double)cx};
                if (dist2(c) <= rr2) visit0(c, f);
            }
        } else {
            const int y0 = (int)floor(u[D - 1] - rr) - 1, y1 = (int)ceil(u[D - 1] + rr) + 1;
            for (int cy = y0; cy <= y1; cy++) {
                const double dy = __dsub_rn((double)cy, u[D - 1]);
                const double dy2 = __dmul_rn(dy, dy);
                if (dy2 > rr2) continue;
                const double s = sqrt(fmax(rr2 - dy2, 0.0));
                int x0 = (int)floor(u[0] - s) - 1, x1 = (int)ceil(u[0] + s) + 1;
                double c[D];
                c[D - 1] = (double)cy;
                c[0] = (double)x0;
                while (x0 <= x1 && dist2(c) > rr2) c[0] = (double)(++x0);
                c[0] = (double)x1;
                while (x1 >= x0 && dist2(c) > rr2) c[0] = (double)(--x1);
                for (int cx = x0; cx <= x1; cx++) {
                    c[0] = (double)cx;
                    visit0(c, f);
                }
            }
        }
    }
};

// ---------------------------------------------------------------------------
// EPR module: Eq. (IID7)-(IID13) in thermal units.
// ---------------------------------------------------------------------------
template <int D, bool FLUON>
struct Basis {
    static constexpr int N = FLUON ? Dim<D>::NF : Dim<D>::NG;
    // fluons: 1, t_a, t_a t_b (a <= b), t_a^2 t_g (g-major); phonons: first 1 + D + D(D+1)/2
    __device__ __forceinline__ static void eval(const double* t, double* T) {
        T[0] = 1.0;
        if constexpr (D == 1) {
            T[1] = t[0];
            T[2] = t[0] * t[0];
            if constexpr (FLUON) T[3] = T[2] * t[0];
        } else {
            const double xx = t[0] * t[0], yy = t[D - 1] * t[D - 1];
            T[1] = t[0];
            T[2] = t[D - 1];
            T[3] = xx;
            T[4] = t[0] * t[D - 1];
            T[5] = yy;
            if constexpr (FLUON) {
                T[6] = xx * t[0];
                T[7] = yy * t[0];
                T[8] = xx * t[D - 1];
                T[9] = yy * t[D - 1];
            }
        }
    }
};

__device__ __forceinline__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// Cholesky factorisation of the packed lower triangle and solve A x = b.
template <int N>
__device__ __forceinline__ bool chol_solve(double* A, double* b) {
#pragma unroll
    for (int j = 0; j < N; j++) {
        double s = A[tri(j, j)];
#pragma unroll
        for (int k = 0; k < j; k++) s -= A[tri(j, k)] * A[tri(j, k)];
        if (!(s > 0.0)) return false;
        const double d = sqrt(s);
        const double id = 1.0 / d;
        A[tri(j, j)] = d;
#pragma unroll
        for (int i = j + 1; i < N; i++) {
            double t = A[tri(i, j)];
#pragma unroll
            for (int k = 0; k < j; k++) t -= A[tri(i, k)] * A[tri(j, k)];
            A[tri(i, j)] = t * id;
        }
    }
#pragma unroll
    for (int i = 0; i < N; i++) {
        double t = b[i];
#pragma unroll
        for (int k = 0; k < i; k++) t -= A[tri(i, k)] * b[k];
        b[i] = t / A[tri(i, i)];
    }
#pragma unroll
    for (int i = N - 1; i >= 0; i--) {
        double t = b[i];
#pragma unroll
        for (int k = i + 1; k < N; k++) t -= A[tri(k, i)] * b[k];
        b[i] = t / A[tri(i, i)];
    }
    return true;
}

// Eq. (IID13) in thermal units: lambda_0 = -1 + D/2 ln(2 pi RT), lambda_aa = 1/2.
template <int D, int N>
__device__ __forceinline__ void maxwell_start(double RT, double* lam) {
#pragma unroll
    for (int j = 0; j < N; j++) lam[j] = 0.0;
    lam[0] = -1.0 + 0.5 * D * log(2.0 * 3.14159265358979323846 * RT);
    int j = 1 + D;
#pragma unroll
    for (int a = 0; a < D; a++)
#pragma unroll
        for (int b = a; b < D; b++) lam[j++] = (a == b) ? 0.5 : 0.0;
}

// Newton-Raphson on the multipliers (Eq. IID8-IID11): returns the number of
// updates (converged, one polishing update included), -1 on a breakdown
// (non-finite residual, non-positive pivot), -2 at the iteration cap.
template <int D, bool FLUON>
__device__ int epr_newton(const CellState<D>& c, const Stencil<D>& st, const double* con, double* lam,
                          const Model& m, unsigned long long& npts) {
    using B = Basis<D, FLUON>;
    constexpr int N = B::N;
    constexpr int NA = N * (N + 1) / 2;
    int updates = 0;
    bool polished = false;
    for (int it = 0;; it++) {
        double A[NA];
#pragma unroll
        for (int i = 0; i < NA; i++) A[i] = 0.0;
        const bool needA = !polished;
        auto acc = [&](const double* cp, double dC) {
            npts++;
            double t[D];
#pragma unroll
            for (int a = 0; a < D; a++) t[a] = (cp[a] - c.u[a]) * c.inv_sig;
            double T[N];
            B::eval(t, T);
            double e = 1.0;
#pragma unroll
            for (int j = 0; j < N; j++) e += lam[j] * T[j];
            const double f = dC * exp(-e);
            if (needA) {
#pragma unroll
                for (int i = 0; i < N; i++) {
                    const double tf = T[i] * f;
#pragma unroll
                    for (int j = 0; j <= i; j++) A[tri(i, j)] += tf * T[j];
                }
            } else {
#pragma unroll
                for (int i = 0; i < N; i++) A[tri(i, 0)] += T[i] * f;
            }
        };
        st.for_each(acc);
        double r[N];
        double rmax = 0.0;
        bool finite = true;
#pragma unroll
        for (int j = 0; j < N; j++) {
            r[j] = A[tri(j, 0)] - con[j];
            finite = finite && isfinite(r[j]);
            rmax = fmax(rmax, fabs(r[j]));
        }
        if (!finite) return -1;
        if (polished) return updates;
        const bool conv = rmax <= m.tol;
        if (!conv && it >= m.max_iter) return -2;
        if (!chol_solve<N>(A, r)) return -1;
#pragma unroll
        for (int j = 0; j < N; j++) lam[j] += r[j];
        updates++;
        if (conv) polished = true;
    }
}

// ---------------------------------------------------------------------------
// The fused single-cell kernel.
// ---------------------------------------------------------------------------
struct LocalStats {
    unsigned long long q_max;
    double disp_max;
    unsigned long long points;
};

template <int D>
__device__ __forceinline__ void scatter_cell(const Model& m, const Geometry& g, const uint8_t* type,
                                             double* Mout, long long cell, const CellState<D>& c,
                                             const Stencil<D>& st, const double* lf, const double* lg,
                                             LocalStats& ls) {
    constexpr int NM = Dim<D>::NM, NF = Dim<D>::NF, NG = Dim<D>::NG;
    const bool has_g = m.K > 0.0;
    const double mfs = c.rho;                // rho dV f'   (Eq. IIE3a)
    const double mgs = c.rho * m.K * c.RT;   // rho K RT dV g'
    // position of the emitting cell
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
    double dmax2 = 0.0;
    auto emit = [&](const double* cp, double dC) {
        q++;
        double t[D];
#pragma unroll
        for (int a = 0; a < D; a++) t[a] = (cp[a] - c.u[a]) * c.inv_sig;
        double T[NF];
        Basis<D, true>::eval(t, T);
        double e = 1.0;
#pragma unroll
        for (int j = 0; j < NF; j++) e += lf[j] * T[j];
        const double mf = mfs * dC * exp(-e);
        double mg = 0.0;
        if (has_g) {
            double eg = 1.0;
#pragma unroll
            for (int j = 0; j < NG; j++) eg += lg[j] * T[j];
            mg = mgs * dC * exp(-eg);
        }
        double csq = 0.0;
#pragma unroll
        for (int a = 0; a < D; a++) csq += cp[a] * cp[a];
        dmax2 = fmax(dmax2, csq);
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
        // cloud-in-cell split of the landing point x + c (exact for integer c)
        int base[D];
        double w1[D];
#pragma unroll
        for (int a = 0; a < D; a++) {
            const double fl = floor(cp[a]);
            base[a] = (int)fl;
            w1[a] = cp[a] - fl;
        }
        const int ncx = w1[0] > 0.0 ? 2 : 1;
        const int ncy = (D == 2 && w1[D - 1] > 0.0) ? 2 : 1;
        for (int sy = 0; sy < ncy; sy++)
            for (int sx = 0; sx < ncx; sx++) {
                double w = sx ? w1[0] : 1.0 - w1[0];
                long long tgt;
                if constexpr (D == 1) {
                    long long x = cell + base[0] + sx;
                    if (g.periodic[0]) {
                        long long r = (x - lo) % n;
                        if (r < 0) r += n;
                        x = lo + r;
                    } else if (x < lo || x >= lo + n) {
                        continue;
                    }
                    tgt = x;
                } else {
                    w *= sy ? w1[D - 1] : 1.0 - w1[D - 1];
                    int tx = ix + base[0] + sx;
                    int ty = iy + base[D - 1] + sy;
                    if (g.periodic[0]) {
                        tx %= g.nx;
                        if (tx < 0) tx += g.nx;
                    } else if (tx < g.pad || tx >= g.pad + g.nx) {
                        continue;
                    }
                    if (g.periodic[1]) {
                        ty %= g.ny;
                        if (ty < 0) ty += g.ny;
                    } else if (ty < g.pad || ty >= g.pad + g.ny) {
                        continue;
                    }
                    tgt = (long long)ty * g.NX + tx;
                }
                if (type[tgt] != CELL_FLUID) continue;
#pragma unroll
                for (int mm = 0; mm < NM; mm++) atomicAdd(Mout + mm * g.ncell + tgt, w * dM[mm]);
            }
    };
    st.for_each(emit);
    if (q > ls.q_max) ls.q_max = q;
    ls.points += q;
    ls.disp_max = fmax(ls.disp_max, sqrt(dmax2));
}

template <int D>
__global__ void __launch_bounds__(128) cell_update_kernel(Model m, Geometry g, const uint8_t* __restrict__ type,
                                                          const double* __restrict__ Min, double* Mout,
                                                          DevStats* stats) {
    constexpr int NM = Dim<D>::NM, NF = Dim<D>::NF, NG = Dim<D>::NG;
    __shared__ unsigned long long s_hist[64];
    __shared__ unsigned long long s_cells, s_feq, s_fmx, s_q;
    __shared__ unsigned long long s_dmax, s_pf, s_pg, s_pm;
    for (int i = threadIdx.x; i < 64; i += blockDim.x) s_hist[i] = 0;
    if (threadIdx.x == 0) s_cells = s_feq = s_fmx = s_q = s_dmax = s_pf = s_pg = s_pm = 0;
    __syncthreads();

    LocalStats ls{0, 0.0, 0};
    unsigned long long my_cells = 0, my_pf = 0, my_pg = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell; cell += stride) {
        const uint8_t ty = type[cell];
        if (ty == CELL_SOLID) continue;
        double M[NM];
#pragma unroll
        for (int i = 0; i < NM; i++) M[i] = Min[i * g.ncell + cell];
        CellState<D> c;
        collide<D>(M, m, c);
        if (!c.ok) {  // non-physical cell: nothing can be reconstructed
            atomicAdd(&s_fmx, 1ull);
            atomicMin(&stats->first_fail, (unsigned long long)cell);
            continue;
        }
        my_cells++;
        Stencil<D> st;
        st.init(c, m);
        const bool has_g = m.K > 0.0;
        double lf[NF], lg[NG];
        maxwell_start<D, NF>(c.RT, lf);
        int sf = epr_newton<D, true>(c, st, c.cf, lf, m, my_pf);
        int sg = 0;
        if (has_g) {
            maxwell_start<D, NG>(c.RT, lg);
            sg = epr_newton<D, false>(c, st, c.cg, lg, m, my_pg);
        } else {
#pragma unroll
            for (int j = 0; j < NG; j++) lg[j] = 0.0;
        }
        if (sf >= 0 && sg >= 0) {
            atomicAdd(&s_hist[sf < 63 ? sf : 63], 1ull);
            if (has_g) atomicAdd(&s_hist[sg < 63 ? sg : 63], 1ull);
        } else {
            // equilibrium constraints (omega = 1) for both populations
            double ef[NF], eg[NG];
#pragma unroll
            for (int j = 0; j < NF; j++) ef[j] = 0.0;
#pragma unroll
            for (int j = 0; j < NG; j++) eg[j] = 0.0;
            ef[0] = eg[0] = 1.0;
            int jj = 1 + D;
#pragma unroll
            for (int a = 0; a < D; a++)
#pragma unroll
                for (int b = a; b < D; b++) {
                    ef[jj] = eg[jj] = (a == b) ? 1.0 : 0.0;
                    jj++;
                }
            maxwell_start<D, NF>(c.RT, lf);
            sf = epr_newton<D, true>(c, st, ef, lf, m, my_pf);
            sg = 0;
            if (has_g) {
                maxwell_start<D, NG>(c.RT, lg);
                sg = epr_newton<D, false>(c, st, eg, lg, m, my_pg);
            }
            if (sf >= 0 && sg >= 0) {
                atomicAdd(&s_feq, 1ull);
            } else {
                // normalised Maxwellian weights: f'_i = dC_i exp(-t^2/2) / S
                double S = 0.0;
                auto sum = [&](const double* cp, double dC) {
                    double t2 = 0.0;
#pragma unroll
                    for (int a = 0; a < D; a++) {
                        const double t = (cp[a] - c.u[a]) * c.inv_sig;
                        t2 += t * t;
                    }
                    S += dC * exp(-0.5 * t2);
                };
                st.for_each(sum);
#pragma unroll
                for (int j = 0; j < NF; j++) lf[j] = 0.0;
                lf[0] = log(S) - 1.0;
                jj = 1 + D;
#pragma unroll
                for (int a = 0; a < D; a++)
#pragma unroll
                    for (int b = a; b < D; b++) {
                        lf[jj] = (a == b) ? 0.5 : 0.0;
                        jj++;
                    }
#pragma unroll
                for (int j = 0; j < NG; j++) lg[j] = lf[j];
                atomicAdd(&s_fmx, 1ull);
                atomicMin(&stats->first_fail, (unsigned long long)cell);
            }
        }
        scatter_cell<D>(m, g, type, Mout, cell, c, st, lf, lg, ls);
    }
    atomicAdd(&s_cells, my_cells);
    atomicAdd(&s_pf, my_pf);
    atomicAdd(&s_pg, my_pg);
    atomicAdd(&s_pm, ls.points);
    atomicMax(&s_q, ls.q_max);
    atomicMax(&s_dmax, (unsigned long long)__double_as_longlong(ls.disp_max));
    __syncthreads();
    for (int i = threadIdx.x; i < 64; i += blockDim.x)
        if (s_hist[i]) atomicAdd(&stats->newton_hist[i], s_hist[i]);
    if (threadIdx.x == 0) {
        atomicAdd(&stats->cells, s_cells);
        atomicAdd(&stats->points_f, s_pf);
        atomicAdd(&stats->points_g, s_pg);
        atomicAdd(&stats->points_ms, s_pm);
        if (s_feq) atomicAdd(&stats->fallback_eq, s_feq);
        if (s_fmx) atomicAdd(&stats->fallback_mx, s_fmx);
        atomicMax(&stats->q_max, s_q);
        atomicMax(&stats->disp_max_bits, s_dmax);
    }
}

// ---------------------------------------------------------------------------
// Boundary fill, state set-up and macroscopic fields.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ void eq_moments(double K, double rho, const double* u, double RT, double* M) {
    double usq = 0.0;
#pragma unroll
    for (int a = 0; a < D; a++) usq += u[a] * u[a];
    M[0] = rho;
#pragma unroll
    for (int a = 0; a < D; a++) M[1 + a] = rho * u[a];
#pragma unroll
    for (int a = 0; a < D; a++)
#pragma unroll
        for (int b = a; b < D; b++) M[iM2<D>(a, b)] = rho * (u[a] * u[b] + (a == b ? RT : 0.0));
#pragma unroll
    for (int g = 0; g < D; g++) M[iMD<D>(g)] = rho * (usq + (D + 2) * RT) * u[g];
    M[iG0<D>()] = rho * K * RT;
#pragma unroll
    for (int g = 0; g < D; g++) M[iG1<D>(g)] = rho * K * RT * u[g];
}

template <int D>
__global__ void fill_pads_kernel(double K, double r_in, double ux, double uy, double RT_in, double* M,
                                 long long ncell, const long long* pad_cell, const long long* pad_src,
                                 long long npad) {
    constexpr int NM = Dim<D>::NM;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < npad;
         k += (long long)gridDim.x * blockDim.x) {
        const long long dst = pad_cell[k], src = pad_src[k];
        if (src < 0) {
            double u[2] = {ux, uy};
            double Me[NM];
            eq_moments<D>(K, r_in, u, RT_in, Me);
#pragma unroll
            for (int i = 0; i < NM; i++) M[i * ncell + dst] = Me[i];
        } else {
#pragma unroll
            for (int i = 0; i < NM; i++) M[i * ncell + dst] = M[i * ncell + src];
        }
    }
}

template <int D>
__global__ void eq_state_kernel(double K, const uint8_t* type, const double* rho, const double* u,
                                const double* RT, double* M, long long ncell) {
    constexpr int NM = Dim<D>::NM;
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < ncell;
         cell += (long long)gridDim.x * blockDim.x) {
        double Me[NM];
        if (type[cell] == CELL_FLUID) {
            double uu[D];
#pragma unroll
            for (int a = 0; a < D; a++) uu[a] = u[a * ncell + cell];
            eq_moments<D>(K, rho[cell], uu, RT[cell], Me);
        } else {
#pragma unroll
            for (int i = 0; i < NM; i++) Me[i] = 0.0;
        }
#pragma unroll
        for (int i = 0; i < NM; i++) M[i * ncell + cell] = Me[i];
    }
}

template <int D>
__global__ void macros_kernel(double K, const uint8_t* type, const double* M, double* rho, double* u, double* RT,
                              long long ncell) {
    for (long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x; cell < ncell;
         cell += (long long)gridDim.x * blockDim.x) {
        double r = 0.0, T = 0.0, uu[D];
#pragma unroll
        for (int a = 0; a < D; a++) uu[a] = 0.0;
        if (type[cell] == CELL_FLUID) {
            r = M[cell];
            double usq = 0.0, tr = 0.0;
#pragma unroll
            for (int a = 0; a < D; a++) {
                uu[a] = __ddiv_rn(M[(1 + a) * ncell + cell], r);
                usq = __dadd_rn(usq, __dmul_rn(uu[a], uu[a]));
                tr = __dadd_rn(tr, M[iM2<D>(a, a) * ncell + cell]);
            }
            T = __ddiv_rn(__dsub_rn(__ddiv_rn(__dadd_rn(tr, M[iG0<D>() * ncell + cell]), r), usq),
                          __dadd_rn((double)D, K));
        }
        rho[cell] = r;
        RT[cell] = T;
#pragma unroll
        for (int a = 0; a < D; a++) u[a * ncell + cell] = uu[a];
    }
}

static int grid_for(long long n, int block) {
    long long b = (n + block - 1) / block;
    if (b < 1) b = 1;
    if (b > 65535LL * 32) b = 65535LL * 32;
    return (int)b;
}

void launch_fill_pads(int D, const Model& m, const double inlet[4], double* M, long long ncell,
                      const long long* pad_cell, const long long* pad_src, long long npad, cudaStream_t s) {
    if (npad == 0) return;
    const int blocks = grid_for(npad, 256);
    if (D == 1)
        fill_pads_kernel<1><<<blocks, 256, 0, s>>>(m.K, inlet[0], inlet[1], inlet[2], inlet[3], M, ncell, pad_cell,
                                                   pad_src, npad);
    else
        fill_pads_kernel<2><<<blocks, 256, 0, s>>>(m.K, inlet[0], inlet[1], inlet[2], inlet[3], M, ncell, pad_cell,
                                                   pad_src, npad);
}

int cell_update_blocks(int D, int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int per_sm = 0;
    if (D == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cell_update_kernel<1>, 128, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cell_update_kernel<2>, 128, 0);
    if (per_sm < 1) per_sm = 1;
    if (sms < 1) sms = 1;
    return sms * per_sm;
}

void launch_cell_update(const Model& m, const Geometry& g, const uint8_t* type, const double* Min, double* Mout,
                        DevStats* st, int grid_blocks, cudaStream_t s) {
    long long need = (g.ncell + 127) / 128;
    int blocks = (int)(need < grid_blocks ? need : grid_blocks);
    if (blocks < 1) blocks = 1;
    if (g.D == 1)
        cell_update_kernel<1><<<blocks, 128, 0, s>>>(m, g, type, Min, Mout, st);
    else
        cell_update_kernel<2><<<blocks, 128, 0, s>>>(m, g, type, Min, Mout, st);
}

void launch_eq_state(int D, double K, const uint8_t* type, const double* rho, const double* u, const double* RT,
                     double* M, long long ncell, cudaStream_t s) {
    const int blocks = grid_for(ncell, 256);
    if (D == 1)
        eq_state_kernel<1><<<blocks, 256, 0, s>>>(K, type, rho, u, RT, M, ncell);
    else
        eq_state_kernel<2><<<blocks, 256, 0, s>>>(K, type, rho, u, RT, M, ncell);
}

void launch_macros(int D, double K, const uint8_t* type, const double* M, double* rho, double* u, double* RT,
                   long long ncell, cudaStream_t s) {
    const int blocks = grid_for(ncell, 256);
    if (D == 1)
        macros_kernel<1><<<blocks, 256, 0, s>>>(K, type, M, rho, u, RT, ncell);
    else
        macros_kernel<2><<<blocks, 256, 0, s>>>(K, type, M, rho, u, RT, ncell);
}

}  // namespace lbm
