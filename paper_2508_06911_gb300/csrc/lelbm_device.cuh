// Device building blocks of the LELBM single-cell operation (arXiv:2508.06911):
// collision module, LAS stencil enumeration, EPR Newton and equilibrium moments.
// Included by the translation units that define kernels; everything here is
// __device__ and header-only.
#pragma once

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
template <>
struct Dim<3> {
    static constexpr int NM = 17, NF = 19, NG = 10;
};

// Position of the pair (a <= b) among the D(D+1)/2 second-order entries, row by row.
__device__ __forceinline__ constexpr int pair3(int a, int b) {
    return a > b ? b * 3 - b * (b - 1) / 2 + (a - b) : a * 3 - a * (a - 1) / 2 + (b - a);
}
// Stored-moment positions, Eq. (IIB5): M0, M_a, M_ab (a <= b, row by row), MD_g, G0, G_g.
template <int D>
__device__ __forceinline__ constexpr int iM2(int a, int b) {
    return D == 1 ? 2 : (D == 2 ? (a == 0 && b == 0 ? 3 : (a == 1 && b == 1 ? 5 : 4)) : 4 + pair3(a, b));
}
template <int D>
__device__ __forceinline__ constexpr int iMD(int g) {
    return D == 1 ? 3 : (D == 2 ? 6 + g : 10 + g);
}
template <int D>
__device__ __forceinline__ constexpr int iG0() {
    return D == 1 ? 4 : (D == 2 ? 8 : 13);
}
template <int D>
__device__ __forceinline__ constexpr int iG1(int g) {
    return D == 1 ? 5 : (D == 2 ? 9 + g : 14 + g);
}

// ---------------------------------------------------------------------------
// Collision module: Eq. (IIB6), (IIB9)-(IIB18), App. C (C7)-(C8), App. D.
// ---------------------------------------------------------------------------
template <int D>
struct CellState {
    double rho, u[D], RT, sig, inv_sig;
    double cf[Dim<D>::NF];  // fluon constraints in thermal units
    double cg[Dim<D>::NG];  // phonon constraints in thermal units
    float cf32[Dim<D>::NF], cg32[Dim<D>::NG];  // the same in FP32 (collide32 sets these only)
    float RT32, sig32, isig32;                 // RT, sqrt(RT), 1/sqrt(RT) in FP32 (collide32)
    bool ok;
};

// Eq. (IIB6), with the operation order of a plain loop and one rounding each: rho, u, RT
// and whether they describe a gas (rho > 0, RT > 0, finite).  usq receives |u|^2.
template <int D>
__device__ __forceinline__ bool cell_macros(const double* M, double K, double& rho, double* u, double& RT,
                                            double& usq) {
    rho = M[0];
    usq = 0.0;
    double tr = 0.0;
#pragma unroll
    for (int a = 0; a < D; a++) {
        u[a] = __ddiv_rn(M[1 + a], rho);
        usq = __dadd_rn(usq, __dmul_rn(u[a], u[a]));
        tr = __dadd_rn(tr, M[iM2<D>(a, a)]);
    }
    RT = __ddiv_rn(__dsub_rn(__ddiv_rn(__dadd_rn(tr, M[iG0<D>()]), rho), usq), __dadd_rn((double)D, K));
    return rho > 0.0 && RT > 0.0 && isfinite(rho) && isfinite(RT);
}

template <int D>
__device__ __forceinline__ void collide(const double* M, const Model& m, CellState<D>& c) {
    constexpr int NF = Dim<D>::NF, NG = Dim<D>::NG;
    const double K = m.K;
    double rho, RT, usq;
    c.ok = cell_macros<D>(M, K, rho, c.u, RT, usq);
    c.rho = rho;
    c.RT = RT;
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
        if (Kn > 0.01) {  // below 0.01 the limiter leaves omega unchanged
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

// The FP32 part of collide32 (App. C, App. D, Eq. IIB10-IIB18 in thermal units) from the
// non-equilibrium central moments P, Q, G0n, Gn.
template <int D>
__device__ __forceinline__ void collide32_tail(const Model& m, CellState<D>& c, const float (&P)[D][D],
                                               const float* Q, float G0n, const float* Gn) {
    constexpr int NG = Dim<D>::NG;
    // App. C and App. D in FP32
    const float rf = (float)c.rho, RTf = c.RT32, sf = c.sig32, Kf = m.K32;
    const float inv_f = m.nu_s32 / RTf + 0.5f;
    float wf = 1.f / inv_f;
    const float fb = 2.f / D - 2.f / (D + Kf);
    float wb = (m.nu_b32 < 0.f || fb <= 0.f) ? 1.f : 1.f / (m.nu_b32 / (RTf * fb) + 0.5f);
    float wh = 1.f / ((inv_f - 0.5f) / m.Pr32 + 0.5f);
    const float ir = 1.f / rf;
    if (m.limiter) {
        float s2 = 0.f, s3 = 0.f;
#pragma unroll
        for (int a = 0; a < D; a++)
#pragma unroll
            for (int b = 0; b < D; b++) s2 += fabsf(P[a][b] * ir);
        s2 += fabsf(G0n * ir);
#pragma unroll
        for (int g = 0; g < D; g++) s3 += fabsf(Q[g] * ir) + fabsf(Gn[g] * ir);
        const float k2 = s2 / ((D + Kf) * RTf);
        const float k3 = s3 / ((D + Kf + 2.f) * RTf * sf);
        const float Kn = fmaxf(k2, k3);
        if (Kn > 0.01f) {
            const float ks = log10f(Kn);
            if (ks >= -1.f) {
                wf = wb = wh = 1.f;
            } else if (ks > -2.f) {
                const float x = ks + 2.f;
                wf += (1.f - wf) * x;
                wb += (1.f - wb) * x;
                wh += (1.f - wh) * x;
            }
        }
    }
    // Eq. (IIB10)-(IIB18), thermal units
    const float bulk = -G0n / D;
    const float iRT = 1.f / RTf;
    c.cf32[0] = 1.f;
#pragma unroll
    for (int a = 0; a < D; a++) c.cf32[1 + a] = 0.f;
    int j = 1 + D;
#pragma unroll
    for (int a = 0; a < D; a++)
#pragma unroll
        for (int b = a; b < D; b++) {
            const float sh = P[a][b] - (a == b ? bulk : 0.f);
            const float mm = (a == b ? rf * RTf : 0.f) + (1.f - wf) * sh + (1.f - wb) * (a == b ? bulk : 0.f);
            c.cf32[j++] = mm * ir * iRT;
        }
    const float s3 = iRT / sf;
#pragma unroll
    for (int g = 0; g < D; g++)
#pragma unroll
        for (int a = 0; a < D; a++)
            c.cf32[j++] = (1.f - wh) * ((1.f + 2.f * (a == g)) / (D + 2) * Q[g]) * ir * s3;
    if (Kf > 0.f) {
        const float nrm = 1.f / (rf * Kf * RTf);
        c.cg32[0] = (rf * Kf * RTf + (1.f - wb) * G0n) * nrm;
#pragma unroll
        for (int g = 0; g < D; g++) c.cg32[1 + g] = (1.f - wh) * Gn[g] * nrm / sf;
        int k = 1 + D;
#pragma unroll
        for (int a = 0; a < D; a++)
#pragma unroll
            for (int b = a; b < D; b++) c.cg32[k++] = (a == b) ? 1.f : 0.f;
    } else {
#pragma unroll
        for (int k = 0; k < NG; k++) c.cg32[k] = 0.f;
    }
}

// The collision module of the FP32 path: the macroscopic variables and the
// non-equilibrium central moments (differences of nearly equal numbers) in FP64, the
// relaxation frequencies, the Knudsen limiter and the normalised constraints in FP32
// (they feed an FP32 Newton solve).  Same equations as collide.
// ALL32: every step in FP32, from the moments rounded to FP32 once (the warm-start
// network's inputs, where the FP32 cancellation in the non-equilibrium moments is far below
// the network's own error).
template <int D, bool ALL32 = false>
__device__ __forceinline__ void collide32(const double* M, const Model& m, CellState<D>& c) {
    constexpr int NG = Dim<D>::NG;
    if constexpr (ALL32) {
        float Mf[Dim<D>::NM];
#pragma unroll
        for (int i = 0; i < Dim<D>::NM; i++) Mf[i] = (float)M[i];
        const float rf = Mf[0], irf = 1.f / rf;
        float uf[D], usq = 0.f, tr = 0.f;
#pragma unroll
        for (int a = 0; a < D; a++) {
            uf[a] = Mf[1 + a] * irf;
            usq = fmaf(uf[a], uf[a], usq);
            tr += Mf[iM2<D>(a, a)];
        }
        const float RTf = ((tr + Mf[iG0<D>()]) * irf - usq) / ((float)D + m.K32);
        c.rho = (double)rf;
        c.RT = (double)RTf;
#pragma unroll
        for (int a = 0; a < D; a++) c.u[a] = (double)uf[a];
        c.ok = rf > 0.f && RTf > 0.f && isfinite(rf) && isfinite(RTf);
        if (!c.ok) return;
        c.RT32 = RTf;
        c.sig32 = sqrtf(RTf);
        c.isig32 = 1.f / c.sig32;
        c.sig = (double)c.sig32;
        c.inv_sig = (double)c.isig32;
        float P[D][D], Q[D], Gn[D];
        float trP = 0.f;
#pragma unroll
        for (int a = 0; a < D; a++)
#pragma unroll
            for (int b = 0; b < D; b++) {
                P[a][b] = Mf[iM2<D>(a, b)] - rf * (uf[a] * uf[b] + (a == b ? RTf : 0.f));
                if (a == b) trP += P[a][b];
            }
#pragma unroll
        for (int g = 0; g < D; g++) {
            float s = 0.f;
#pragma unroll
            for (int a = 0; a < D; a++) s += uf[a] * P[a][g];
            Q[g] = Mf[iMD<D>(g)] - 2.f * s - uf[g] * trP - rf * (usq + (D + 2) * RTf) * uf[g];
            Gn[g] = Mf[iG1<D>(g)] - uf[g] * Mf[iG0<D>()];
        }
        const float G0n = Mf[iG0<D>()] - rf * m.K32 * RTf;
        collide32_tail<D>(m, c, P, Q, G0n, Gn);
        return;
    }
    const double K = m.K;
    const double rho = M[0];
    // 1 / rho from the FP32 reciprocal and two Newton steps (24 -> 48 -> 53 bits), not
    // an FP64 division; 1 / (D + K) is a constant of the handle
    double irho;
    if (rho > 1e-30 && rho < 1e30) {
        irho = (double)(1.f / (float)rho);
        irho = fma(irho, fma(-rho, irho, 1.0), irho);
        irho = fma(irho, fma(-rho, irho, 1.0), irho);
    } else {
        irho = 1.0 / rho;
    }
    double usq = 0.0, tr = 0.0;
#pragma unroll
    for (int a = 0; a < D; a++) {
        c.u[a] = M[1 + a] * irho;
        usq += c.u[a] * c.u[a];
        tr += M[iM2<D>(a, a)];
    }
    const double RT = ((tr + M[iG0<D>()]) * irho - usq) * m.inv_dk;
    c.rho = rho;
    c.RT = RT;
    c.ok = rho > 0.0 && RT > 0.0 && isfinite(rho) && isfinite(RT);
    if (!c.ok) return;
    {
        c.RT32 = (float)RT;
        const float sf = sqrtf(c.RT32);  // FP32 is enough: it only scales FP32 coordinates
        c.sig32 = sf;
        c.isig32 = 1.f / sf;
        c.sig = (double)sf;
        c.inv_sig = (double)c.isig32;
    }
    // Eq. (IIB9) in FP64
    float P[D][D];
    double trP = 0.0;
    double Pd[D][D];
#pragma unroll
    for (int a = 0; a < D; a++)
#pragma unroll
        for (int b = 0; b < D; b++) {
            Pd[a][b] = M[iM2<D>(a, b)] - rho * (c.u[a] * c.u[b] + (a == b ? RT : 0.0));
            P[a][b] = (float)Pd[a][b];
        }
#pragma unroll
    for (int a = 0; a < D; a++) trP += Pd[a][a];
    float Q[D];
#pragma unroll
    for (int g = 0; g < D; g++) {
        double s = 0.0;
#pragma unroll
        for (int a = 0; a < D; a++) s += c.u[a] * Pd[a][g];
        Q[g] = (float)(M[iMD<D>(g)] - 2.0 * s - c.u[g] * trP - rho * (usq + (D + 2) * RT) * c.u[g]);
    }
    const double G0 = M[iG0<D>()];
    const float G0n = (float)(G0 - rho * K * RT);
    float Gn[D];
#pragma unroll
    for (int g = 0; g < D; g++) Gn[g] = (float)(M[iG1<D>(g)] - c.u[g] * G0);

    collide32_tail<D>(m, c, P, Q, G0n, Gn);
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

    // The same set-up in FP32 for the FP32 path (R_ac and N_r differ from the FP64
    // decision only when n sqrt(RT) or 1 / (3 sqrt(RT)) lies within FP32 rounding of a
    // half-integer).
    __device__ __forceinline__ void init32(const CellState<D>& c, const Model& m) {
#pragma unroll
        for (int a = 0; a < D; a++) u[a] = c.u[a];
        const float sf = c.sig32;
        float r = roundf(m.n_conf32 * sf);
        if (r < m.r_min32) r = m.r_min32;
        R = (int)r;
        const float rr = (float)R + 0.5f;
        rr2 = (double)(rr * rr);
        float nr = roundf(1.f / (m.refine_div32 * sf));
        if (nr > (float)m.max_refine) nr = (float)m.max_refine;
        Nr = (int)nr;
#pragma unroll
        for (int L = 0; L < 5; L++) rad2[L] = m.rad2_32[L];
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

    // Row form of the same velocity set: row(cy, xa, xb) receives the level-0
    // integer points cx = xa..xb of row cy (cy = 0 in 1D, dC = 1); leaf(c, dC)
    // receives every refined point.  Membership is tested only at segment ends:
    // the exact test is monotone along a row, so every segment is an interval.
    template <class RowF, class LeafF>
    __device__ __forceinline__ void for_each_row(RowF& row, LeafF& leaf) const {
        const double rr = sqrt(rr2);
        int y0 = 0, y1 = 0;
        if constexpr (D == 2) {
            y0 = (int)floor(u[1] - rr) - 1;
            y1 = (int)ceil(u[1] + rr) + 1;
        }
        const double r1 = sqrt(rad2[1]);
        for (int cy = y0; cy <= y1; cy++) {
            double c[D];
            double s = rr;
            if constexpr (D == 2) {
                c[1] = (double)cy;
                const double dy = __dsub_rn((double)cy, u[1]);
                const double dy2 = __dmul_rn(dy, dy);
                if (dy2 > rr2) continue;
                s = sqrt(fmax(rr2 - dy2, 0.0));
            }
            int x0 = (int)floor(u[0] - s) - 1, x1 = (int)ceil(u[0] + s) + 1;
            c[0] = (double)x0;
            while (x0 <= x1 && dist2(c) > rr2) c[0] = (double)(++x0);
            c[0] = (double)x1;
            while (x1 >= x0 && dist2(c) > rr2) c[0] = (double)(--x1);
            if (x0 > x1) continue;
            if (Nr > 0) {
                int a = (int)floor(u[0] - r1) - 1, b = (int)ceil(u[0] + r1) + 1;
                a = a < x0 ? x0 : a;
                b = b > x1 ? x1 : b;
                c[0] = (double)a;
                while (a <= b && dist2(c) > rad2[1]) c[0] = (double)(++a);
                c[0] = (double)b;
                while (b >= a && dist2(c) > rad2[1]) c[0] = (double)(--b);
                if (a <= b) {
                    if (x0 <= a - 1) row(cy, x0, a - 1);
                    for (int cx = a; cx <= b; cx++) {
                        c[0] = (double)cx;
                        visit0(c, leaf);
                    }
                    if (b + 1 <= x1) row(cy, b + 1, x1);
                    continue;
                }
            }
            row(cy, x0, x1);
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
// Row table of the velocity set for the FP32 passes.  The stencil's membership
// decisions are exact FP64 tests; when there is at most one refinement level they
// are taken once per cell and kept as integer extents per row -- the level-0 points
// [x0, x1] and the band [a, b] of level-0 points that split into 2^D children at
// +-1/4 -- so every FP32 pass and the FP32 streaming pass enumerate the same set
// with FP32 and integer arithmetic only.  1D keeps its one row in registers; 2D
// keeps the extents of up to kRowsMax rows (offsets from floor(u)) in the caller's
// shared memory and the split points of up to kBandMax rows packed in registers.
// A cell with more levels, rows or split-point rows, or offsets beyond int8, uses
// Stencil directly.
// ---------------------------------------------------------------------------
constexpr int kRowsMax = 56;
constexpr int kBandMax = 4;  // rows with split points: |y - u_y| <= 3/2 spans at most 4

template <int D>
struct RowTable {
    bool ok;
    int xc, yc;          // floor(u)
    int y_first, nrows;  // 2D rows y_first .. y_first + nrows - 1
    int x0, x1, a, b;    // 1D: the row
    const char2* rows;   // 2D: (x0, x1) - xc per row; x0 > x1: empty
    int band_first, band_n;        // 2D: rows band_first .. + band_n - 1 have split points
    unsigned long long band;       // 2D: their (a, b) - xc, 16 bits per row
    float fux, fuy;      // (u - floor(u)) / sqrt(RT), FP32
    float s32;           // 1 / sqrt(RT), FP32

    // 2D: records (ea, eb) (offsets from xc) of row r as a split-point row; false when the
    // rows with split points are not consecutive or more than kBandMax
    __device__ __forceinline__ bool add_band(int r, int ea, int eb) {
        if (band_n == 0) band_first = r;
        if (r != band_first + band_n || band_n == kBandMax) return false;
        const unsigned long long w = (unsigned long long)(((unsigned)(ea & 0xff)) | ((unsigned)(eb & 0xff) << 8));
        band |= w << (16 * band_n);
        band_n++;
        return true;
    }
    // 2D: extents of row r as lattice offsets: level-0 points x0..x1, split points a..b
    // (a > b: none)
    __device__ __forceinline__ void row_ext(int r, int& rx0, int& rx1, int& ra, int& rb) const {
        const char2 e = rows[r];
        rx0 = xc + e.x;
        rx1 = xc + e.y;
        const int k = r - band_first;
        if ((unsigned)k < (unsigned)band_n) {
            const unsigned w = (unsigned)(band >> (16 * k));
            ra = xc + (int)(signed char)(w & 0xffu);
            rb = xc + (int)(signed char)((w >> 8) & 0xffu);
        } else {
            ra = rx1 + 1;
            rb = rx1;
        }
    }

    // The membership decisions are those of the FP64 stencil (Stencil::dist2 against
    // (R + 1/2)^2 and the refinement radius), taken in FP32 first: a test whose FP32 value
    // lies more than 1e-3 + 1e-5 thr from the threshold thr is decided there (the FP32
    // rounding of (k - u_x)^2 + dy^2 is below 3e-4 for offsets up to 30), and only the
    // others are recomputed in FP64 exactly as the stencil computes them.  GB300's FP64
    // pipe is slow, and a cell makes a few dozen of these tests.
    __device__ __forceinline__ void build(const CellState<D>& c, const Stencil<D>& st, char2* buf) {
        xc = (int)floor(c.u[0]);
        yc = D == 2 ? (int)floor(c.u[D - 1]) : 0;
        s32 = (float)c.inv_sig;
        const double ux = c.u[0] - (double)xc, uy = D == 2 ? c.u[D - 1] - (double)yc : 0.0;
        fux = (float)(ux * c.inv_sig);
        fuy = D == 2 ? (float)(uy * c.inv_sig) : 0.f;
        rows = buf;
        band_first = band_n = 0;
        band = 0ull;
        ok = st.Nr <= 1;
        if (!ok) return;
        const float uxf = (float)ux, uyf = (float)uy;
        const float rr2f = (float)st.rr2, r12f = (float)st.rad2[1];
        const float rrf = sqrtf(rr2f), r1f = sqrtf(r12f);
        // is the level-0 point (xc + k, yc + ky) within distance^2 thr of u?
        auto inside = [&](int k, int ky, float dy2f, double thr, float thrf) -> bool {
            const float d = (float)k - uxf;
            const float v = fmaf(d, d, dy2f);
            const float mg = 1e-3f + 1e-5f * thrf;
            if (v < thrf - mg) return true;
            if (v > thrf + mg) return false;
            double p[D];
            p[0] = (double)(xc + k);
            if constexpr (D == 2) p[1] = (double)(yc + ky);
            return st.dist2(p) <= thr;
        };
        // offsets from xc of the row ky: level-0 points e0..e1, split points ea..eb
        auto extents = [&](int ky, float dy2f, int& e0, int& e1, int& ea, int& eb) {
            const float sr = sqrtf(fmaxf(rr2f - dy2f, 0.f));
            e0 = (int)floorf(uxf - sr) - 1;
            e1 = (int)ceilf(uxf + sr) + 1;
            while (e0 <= e1 && !inside(e0, ky, dy2f, st.rr2, rr2f)) ++e0;
            while (e1 >= e0 && !inside(e1, ky, dy2f, st.rr2, rr2f)) --e1;
            ea = 1;
            eb = 0;
            if (st.Nr == 1 && e0 <= e1) {
                ea = max((int)floorf(uxf - r1f) - 1, e0);
                eb = min((int)ceilf(uxf + r1f) + 1, e1);
                while (ea <= eb && !inside(ea, ky, dy2f, st.rad2[1], r12f)) ++ea;
                while (eb >= ea && !inside(eb, ky, dy2f, st.rad2[1], r12f)) --eb;
                if (ea > eb) {
                    ea = 1;
                    eb = 0;
                }
            }
        };
        if constexpr (D == 1) {
            int e0, e1, ea, eb;
            extents(0, 0.f, e0, e1, ea, eb);
            x0 = xc + e0;
            x1 = xc + e1;
            if (ea > eb) {
                a = x1 + 1;
                b = x1;
            } else {
                a = xc + ea;
                b = xc + eb;
            }
        } else {
            const int k_first = (int)floorf(uyf - rrf) - 1, k_last = (int)ceilf(uyf + rrf) + 1;
            y_first = yc + k_first;
            nrows = k_last - k_first + 1;
            if (nrows > kRowsMax) {
                ok = false;
                return;
            }
            for (int r = 0; r < nrows; r++) {
                const int ky = k_first + r;
                const float dy = (float)ky - uyf;
                const float dy2f = dy * dy;
                int e0 = 1, e1 = 0, ea = 1, eb = 0;
                // a row clearly beyond the radius is empty; any other is tested point by point
                if (dy2f <= rr2f + 1e-3f + 1e-5f * rr2f) extents(ky, dy2f, e0, e1, ea, eb);
                if (e0 > e1) {
                    e0 = 1;
                    e1 = 0;
                }
                if (ea > eb) {
                    ea = e1 + 1;
                    eb = e1;
                }
                if (e0 < -127 || e1 > 127 || ea < -127 || eb > 127) {
                    ok = false;
                    return;
                }
                buf[r] = make_char2((signed char)e0, (signed char)e1);
                if (ea <= eb && !add_band(r, ea, eb)) {
                    ok = false;
                    return;
                }
            }
        }
    }

    // The same table with FP32 membership tests for the FP32 path, on offsets from
    // floor(u) (so the tests stay exact for the dyadic cases: integer or half-integer u,
    // (R + 1/2)^2, 9/4).
    __device__ __forceinline__ void build32(const CellState<D>& c, const Stencil<D>& st, char2* buf) {
        xc = (int)floor(c.u[0]);
        yc = D == 2 ? (int)floor(c.u[D - 1]) : 0;
        s32 = c.isig32;
        const float ux = (float)(c.u[0] - (double)xc);
        const float uy = D == 2 ? (float)(c.u[D - 1] - (double)yc) : 0.f;
        fux = ux * s32;
        fuy = uy * s32;
        rows = buf;
        band_first = band_n = 0;
        band = 0ull;
        ok = st.Nr <= 1;
        if (!ok) return;
        const float rr = (float)st.R + 0.5f, rr2f = rr * rr, r12 = (float)st.rad2[1];
        const float r1 = sqrtf(r12);
        // extents, as offsets from xc, of the row at squared y-distance dy2
        auto extents = [&](float dy2, float s, int& e0, int& e1, int& ea, int& eb) {
            auto d2 = [&](int k) {
                const float d = (float)k - ux;
                return d * d + dy2;
            };
            e0 = (int)floorf(ux - s) - 1;
            e1 = (int)ceilf(ux + s) + 1;
            while (e0 <= e1 && d2(e0) > rr2f) ++e0;
            while (e1 >= e0 && d2(e1) > rr2f) --e1;
            ea = 1;
            eb = 0;
            if (st.Nr == 1 && e0 <= e1) {
                ea = max((int)floorf(ux - r1) - 1, e0);
                eb = min((int)ceilf(ux + r1) + 1, e1);
                while (ea <= eb && d2(ea) > r12) ++ea;
                while (eb >= ea && d2(eb) > r12) --eb;
                if (ea > eb) {
                    ea = 1;
                    eb = 0;
                }
            }
        };
        if constexpr (D == 1) {
            int e0, e1, ea, eb;
            extents(0.f, rr, e0, e1, ea, eb);
            x0 = xc + e0;
            x1 = xc + e1;
            if (ea > eb) {
                a = x1 + 1;
                b = x1;
            } else {
                a = xc + ea;
                b = xc + eb;
            }
        } else {
            const int k_first = (int)floorf(uy - rr) - 1, k_last = (int)ceilf(uy + rr) + 1;
            y_first = yc + k_first;
            nrows = k_last - k_first + 1;
            if (nrows > kRowsMax) {
                ok = false;
                return;
            }
            for (int r = 0; r < nrows; r++) {
                const float dy = (float)(k_first + r) - uy;
                const float dy2 = dy * dy;
                int e0 = 1, e1 = 0, ea = 1, eb = 0;
                if (dy2 <= rr2f) extents(dy2, sqrtf(fmaxf(rr2f - dy2, 0.f)), e0, e1, ea, eb);
                if (e0 > e1) {
                    e0 = 1;
                    e1 = 0;
                }
                if (ea > eb) {
                    ea = e1 + 1;
                    eb = e1;
                }
                if (e0 < -127 || e1 > 127 || ea < -127 || eb > 127) {
                    ok = false;
                    return;
                }
                buf[r] = make_char2((signed char)e0, (signed char)e1);
                if (ea <= eb && !add_band(r, ea, eb)) {
                    ok = false;
                    return;
                }
            }
        }
    }

    // row(cy, xa, xb) for level-0 segments; child(p, cy, sx, sy) for the 2^D children
    // of each split point (at p + sx/4, cy + sy/4, dC = 2^-D).
    template <class RowF, class ChildF>
    __device__ __forceinline__ void visit(RowF& row, ChildF& child) const {
        auto one = [&](int cy, int e0, int e1, int ea, int eb) {
            if (ea <= eb) {
                if (e0 <= ea - 1) row(cy, e0, ea - 1);
                for (int p = ea; p <= eb; p++) {
#pragma unroll
                    for (int k = 0; k < (1 << D); k++) child(p, cy, (k & 1) ? 1 : -1, (k & 2) ? 1 : -1);
                }
                if (eb + 1 <= e1) row(cy, eb + 1, e1);
            } else if (e0 <= e1) {
                row(cy, e0, e1);
            }
        };
        if constexpr (D == 1) {
            one(0, x0, x1, a, b);
        } else {
            for (int r = 0; r < nrows; r++) {
                int rx0, rx1, ra, rb;
                row_ext(r, rx0, rx1, ra, rb);
                one(y_first + r, rx0, rx1, ra, rb);
            }
        }
    }

    // FP32 thermal coordinate of lattice coordinate p (+ q/4) along x or y
    __device__ __forceinline__ float tx(int p, float q4 = 0.f) const {
        return fmaf((float)(p - xc) + q4, s32, -fux);
    }
    __device__ __forceinline__ float ty(int p, float q4 = 0.f) const {
        return fmaf((float)(p - yc) + q4, s32, -fuy);
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

// lambda_0 of Eq. (IID13).
template <int D>
__device__ __forceinline__ double maxwell_l0(double RT) {
    return -1.0 + 0.5 * D * log(2.0 * 3.14159265358979323846 * RT);
}

// Eq. (IID13) for both populations with one logarithm.
template <int D, int NFv, int NGv>
__device__ __forceinline__ void maxwell_start_fg(double RT, double* lf, double* lg) {
    const double l0 = -1.0 + 0.5 * D * log(2.0 * 3.14159265358979323846 * RT);
#pragma unroll
    for (int j = 0; j < NFv; j++) lf[j] = 0.0;
#pragma unroll
    for (int j = 0; j < NGv; j++) lg[j] = 0.0;
    lf[0] = lg[0] = l0;
    int j = 1 + D;
#pragma unroll
    for (int a = 0; a < D; a++)
#pragma unroll
        for (int b = a; b < D; b++) {
            lf[j] = lg[j] = (a == b) ? 0.5 : 0.0;
            j++;
        }
}

// Eq. (IID13) in FP32 for the FP32 path.
template <int D, int NFv, int NGv>
__device__ __forceinline__ void maxwell_start32(float RT, float* lf, float* lg) {
    const float l0 = -1.f + 0.5f * D * logf(6.2831853071795865f * RT);
#pragma unroll
    for (int j = 0; j < NFv; j++) lf[j] = 0.f;
#pragma unroll
    for (int j = 0; j < NGv; j++) lg[j] = 0.f;
    lf[0] = lg[0] = l0;
    int j = 1 + D;
#pragma unroll
    for (int a = 0; a < D; a++)
#pragma unroll
        for (int b = a; b < D; b++) {
            lf[j] = lg[j] = (a == b) ? 0.5f : 0.f;
            j++;
        }
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
// EPR Newton in moment form.  The fluon basis is every monomial x^a y^b of total
// degree <= 3 and the phonon basis every monomial of degree <= 2 (Eq. IIB14-17 in
// thermal units), so A_ij = sum_k T_i T_j f_k is the population moment of
// x^(a_i + a_j) y^(b_i + b_j): degree <= 6 (fluons) or <= 4 (phonons).  Along a
// stencil row (fixed y) those moments are y^b times the row sums S_a = sum x^a f,
// so a point costs the powers of x and one FMA per row sum instead of the
// N(N+1)/2 products of Eq. (IID11a).  The residual (IID11c) is the first column.
// ---------------------------------------------------------------------------
__device__ __forceinline__ constexpr int tix(int a, int b, int P) { return b * (P + 1) - b * (b - 1) / 2 + a; }

template <int D>
struct MomentSet {
    static constexpr int PF = 6, PG = 4;
    static constexpr int NF = D == 1 ? PF + 1 : (PF + 1) * (PF + 2) / 2;
    static constexpr int NG = D == 1 ? PG + 1 : (PG + 1) * (PG + 2) / 2;
};

// exponents (a_j, b_j) of the basis entries, in the order of Basis<D, FLUON>::eval
template <int D, bool FLUON>
__device__ __forceinline__ constexpr int bx(int j) {
    if constexpr (D == 1) {
        return j;
    } else {
        constexpr int a[10] = {0, 1, 0, 2, 1, 0, 3, 1, 2, 0};
        return a[j];
    }
}
template <int D, bool FLUON>
__device__ __forceinline__ constexpr int by(int j) {
    if constexpr (D == 1) {
        return 0;
    } else {
        constexpr int b[10] = {0, 0, 1, 0, 1, 2, 0, 2, 1, 3};
        return b[j];
    }
}

// Coefficients of the exponent 1 + sum_j lam_j T_j as a polynomial in x on the row y.
template <int D>
__device__ __forceinline__ void row_coeffs(const double* lf, const double* lg, double y, double* cf, double* cg) {
    if constexpr (D == 1) {
        cf[0] = 1.0 + lf[0];
        cf[1] = lf[1];
        cf[2] = lf[2];
        cf[3] = lf[3];
        cg[0] = 1.0 + lg[0];
        cg[1] = lg[1];
        cg[2] = lg[2];
    } else {
        cf[0] = 1.0 + lf[0] + y * (lf[2] + y * (lf[5] + y * lf[9]));
        cf[1] = lf[1] + y * (lf[4] + y * lf[7]);
        cf[2] = lf[3] + y * lf[8];
        cf[3] = lf[6];
        cg[0] = 1.0 + lg[0] + y * (lg[2] + y * lg[5]);
        cg[1] = lg[1] + y * lg[4];
        cg[2] = lg[3];
    }
}

// Populations along one stencil row: x_k = x_a + k h (k = 0..n-1), f_k = exp(-e_f(x_k))
// and g_k = exp(-e_g(x_k)) with e_f cubic and e_g quadratic in x (row_coeffs).  Rows
// of fewer than 4 points call exp per point.  Longer rows use multiplicative forward
// differences,
// exp(-e(x + h)) = exp(-e(x)) exp(-d1), d1 <- d1 + d2, d2 <- d2 + d3 (d3 constant for
// a cubic), with d1, d2, d3 taken from the exact difference polynomials; each row is
// swept in one pass when short and outwards from its centre when long, so the rounding
// growth (~k^3/6 ulp after k steps) stays far below the Newton tolerance.
// point(k, x, f, g) is called once per point (in sweep order for long rows).
constexpr int kRecurrenceMinRow = 24;

template <class Pt>
__device__ __forceinline__ void row_sweep(const double* cf, const double* cg, bool doF, bool doG, double x, double h,
                                          int k0, int dir, int m, Pt& point) {
    const double h2 = h * h, h3 = h2 * h;
    double Ef = 0.0, R1f = 0.0, R2f = 0.0, R3f = 0.0, Eg = 0.0, R1g = 0.0, R2g = 0.0;
    if (doF) {
        const double d1 = cf[1] * h + cf[2] * (2.0 * x * h + h2) + cf[3] * (3.0 * x * x * h + 3.0 * x * h2 + h3);
        const double d2 = 2.0 * cf[2] * h2 + cf[3] * (6.0 * x * h2 + 6.0 * h3);
        Ef = exp(-(((cf[3] * x + cf[2]) * x + cf[1]) * x + cf[0]));
        R1f = exp(-d1);
        R2f = exp(-d2);
        R3f = exp(-6.0 * cf[3] * h3);
    }
    if (doG) {
        const double d1 = cg[1] * h + cg[2] * (2.0 * x * h + h2);
        Eg = exp(-((cg[2] * x + cg[1]) * x + cg[0]));
        R1g = exp(-d1);
        R2g = exp(-2.0 * cg[2] * h2);
    }
    for (int i = 0; i < m; i++) {
        point(k0 + dir * i, x, Ef, Eg);
        Ef *= R1f;
        R1f *= R2f;
        R2f *= R3f;
        Eg *= R1g;
        R1g *= R2g;
        x += h;
    }
}

template <class Pt>
__device__ __forceinline__ void row_eval(const double* cf, const double* cg, bool doF, bool doG, double xa, double h,
                                         int n, Pt& point) {
    if (n < 4) {
        double x = xa;
        for (int k = 0; k < n; k++, x += h) {
            const double f = doF ? exp(-(((cf[3] * x + cf[2]) * x + cf[1]) * x + cf[0])) : 0.0;
            const double g = doG ? exp(-((cg[2] * x + cg[1]) * x + cg[0])) : 0.0;
            point(k, x, f, g);
        }
        return;
    }
    if (n < kRecurrenceMinRow) {  // one sweep: at most ~kRecurrenceMinRow^3/6 ulp at the far end
        row_sweep(cf, cg, doF, doG, xa, h, 0, 1, n, point);
        return;
    }
    const int kc = n >> 1;
    row_sweep(cf, cg, doF, doG, xa + kc * h, h, kc, 1, n - kc, point);
    row_sweep(cf, cg, doF, doG, xa + (kc - 1) * h, -h, kc - 1, -1, kc, point);
}

// One pass over the velocity set accumulating the population moments of f
// (if doF) and g (if doG) for the multipliers lf, lg.  Returns the point count.
template <int D>
__device__ __forceinline__ unsigned long long moment_pass(const CellState<D>& c, const Stencil<D>& st,
                                                          const double* lf, const double* lg, bool doF, bool doG,
                                                          double* MF, double* MG) {
    using MS = MomentSet<D>;
#pragma unroll
    for (int i = 0; i < MS::NF; i++) MF[i] = 0.0;
#pragma unroll
    for (int i = 0; i < MS::NG; i++) MG[i] = 0.0;
    unsigned long long q = 0;
    auto row = [&](int cy, int xa, int xb) {
        double y = 0.0;
        if constexpr (D == 2) y = ((double)cy - c.u[1]) * c.inv_sig;
        double cf[4], cg[3];
        row_coeffs<D>(lf, lg, y, cf, cg);
        double SF[MS::PF + 1], SG[MS::PG + 1];
#pragma unroll
        for (int a = 0; a <= MS::PF; a++) SF[a] = 0.0;
#pragma unroll
        for (int a = 0; a <= MS::PG; a++) SG[a] = 0.0;
        auto point = [&](int, double x, double f, double g) {
            double p[MS::PF + 1];
            p[0] = 1.0;
#pragma unroll
            for (int k = 1; k <= MS::PF; k++) p[k] = p[k - 1] * x;
            if (doF) {
#pragma unroll
                for (int a = 0; a <= MS::PF; a++) SF[a] += p[a] * f;
            }
            if (doG) {
#pragma unroll
                for (int a = 0; a <= MS::PG; a++) SG[a] += p[a] * g;
            }
        };
        row_eval(cf, cg, doF, doG, ((double)xa - c.u[0]) * c.inv_sig, c.inv_sig, xb - xa + 1, point);
        q += (unsigned long long)(xb - xa + 1);
        if constexpr (D == 1) {
#pragma unroll
            for (int a = 0; a <= MS::PF; a++) MF[a] += SF[a];
#pragma unroll
            for (int a = 0; a <= MS::PG; a++) MG[a] += SG[a];
        } else {
            double yp[MS::PF + 1];
            yp[0] = 1.0;
#pragma unroll
            for (int k = 1; k <= MS::PF; k++) yp[k] = yp[k - 1] * y;
#pragma unroll
            for (int b = 0; b <= MS::PF; b++)
#pragma unroll
                for (int a = 0; a + b <= MS::PF; a++) MF[tix(a, b, MS::PF)] += SF[a] * yp[b];
#pragma unroll
            for (int b = 0; b <= MS::PG; b++)
#pragma unroll
                for (int a = 0; a + b <= MS::PG; a++) MG[tix(a, b, MS::PG)] += SG[a] * yp[b];
        }
    };
    auto leaf = [&](const double* cp, double dC) {
        const double x = (cp[0] - c.u[0]) * c.inv_sig;
        double y = 0.0;
        if constexpr (D == 2) y = (cp[1] - c.u[1]) * c.inv_sig;
        double cf[4], cg[3];
        row_coeffs<D>(lf, lg, y, cf, cg);
        double px[MS::PF + 1], py[MS::PF + 1];
        px[0] = py[0] = 1.0;
#pragma unroll
        for (int k = 1; k <= MS::PF; k++) {
            px[k] = px[k - 1] * x;
            py[k] = py[k - 1] * y;
        }
        if (doF) {
            const double f = dC * exp(-(((cf[3] * x + cf[2]) * x + cf[1]) * x + cf[0]));
#pragma unroll
            for (int b = 0; b <= (D == 2 ? MS::PF : 0); b++)
#pragma unroll
                for (int a = 0; a + b <= MS::PF; a++) MF[tix(a, b, MS::PF)] += px[a] * py[b] * f;
        }
        if (doG) {
            const double g = dC * exp(-((cg[2] * x + cg[1]) * x + cg[0]));
#pragma unroll
            for (int b = 0; b <= (D == 2 ? MS::PG : 0); b++)
#pragma unroll
                for (int a = 0; a + b <= MS::PG; a++) MG[tix(a, b, MS::PG)] += px[a] * py[b] * g;
        }
        q++;
    };
    st.for_each_row(row, leaf);
    return q;
}

// Reciprocal of an LDL^T pivot: IEEE in FP64; in FP32 (the FP32 Newton, which corrects
// its own step errors) the hardware approximation, within 2 ulp.
__device__ __forceinline__ double pivot_recip(double d) { return 1.0 / d; }
__device__ __forceinline__ float pivot_recip(float d) { return __fdividef(1.f, d); }

// LDL^T factorisation of the packed lower triangle and solve A x = b: the same
// SPD solve as Cholesky without square roots, one reciprocal per column.
template <typename T, int N>
__device__ __forceinline__ bool ldlt_solve(T* A, T* b) {
    T inv[N];
#pragma unroll
    for (int j = 0; j < N; j++) {
        T d = A[tri(j, j)];
#pragma unroll
        for (int k = 0; k < j; k++) d -= A[tri(j, k)] * A[tri(j, k)] * A[tri(k, k)];
        if (!(d > T(0))) return false;
        A[tri(j, j)] = d;
        inv[j] = pivot_recip(d);
#pragma unroll
        for (int i = j + 1; i < N; i++) {
            T t = A[tri(i, j)];
#pragma unroll
            for (int k = 0; k < j; k++) t -= A[tri(i, k)] * A[tri(j, k)] * A[tri(k, k)];
            A[tri(i, j)] = t * inv[j];
        }
    }
#pragma unroll
    for (int i = 0; i < N; i++) {
        T t = b[i];
#pragma unroll
        for (int k = 0; k < i; k++) t -= A[tri(i, k)] * b[k];
        b[i] = t;
    }
#pragma unroll
    for (int i = N - 1; i >= 0; i--) {
        T t = b[i] * inv[i];
#pragma unroll
        for (int k = i + 1; k < N; k++) t -= A[tri(k, i)] * b[k];
        b[i] = t;
    }
    return true;
}

// Newton update from the moments of the current pass (Eq. IID8-IID11).
// Returns 0 (updated), 1 (converged: the polishing update was applied),
// -1 (non-finite residual or non-positive pivot), -2 (iteration cap).
template <int D, bool FLUON>
__device__ __forceinline__ int newton_step_tol(const double* Mom, const double* con, double* lam, double tol,
                                               int max_iter, int it) {
    constexpr int N = Basis<D, FLUON>::N;
    constexpr int P = FLUON ? MomentSet<D>::PF : MomentSet<D>::PG;
    double r[N];
    double rmax = 0.0;
    bool finite = true;
#pragma unroll
    for (int j = 0; j < N; j++) {
        r[j] = Mom[tix(bx<D, FLUON>(j), by<D, FLUON>(j), P)] - con[j];
        finite = finite && isfinite(r[j]);
        rmax = fmax(rmax, fabs(r[j]));
    }
    if (!finite) return -1;
    const bool conv = rmax <= tol;
    if (!conv && it >= max_iter) return -2;
    double A[N * (N + 1) / 2];
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j <= i; j++)
            A[tri(i, j)] = Mom[tix(bx<D, FLUON>(i) + bx<D, FLUON>(j), by<D, FLUON>(i) + by<D, FLUON>(j), P)];
    if (!ldlt_solve<double, N>(A, r)) return -1;
#pragma unroll
    for (int j = 0; j < N; j++) lam[j] += r[j];
    return conv ? 1 : 0;
}

// The same update from FP32 moments with an FP32 solve (FP32 Newton phase); the
// multipliers and constraints are FP32 as well.
template <int D, bool FLUON>
__device__ __forceinline__ int newton_step32(const float* Mom, const float* con, float* lam, float tol, int max_iter,
                                             int it) {
    constexpr int N = Basis<D, FLUON>::N;
    constexpr int P = FLUON ? MomentSet<D>::PF : MomentSet<D>::PG;
    float r[N];
    float rmax = 0.f;
    bool finite = true;
#pragma unroll
    for (int j = 0; j < N; j++) {
        r[j] = Mom[tix(bx<D, FLUON>(j), by<D, FLUON>(j), P)] - con[j];
        finite = finite && isfinite(r[j]);
        rmax = fmaxf(rmax, fabsf(r[j]));
    }
    if (!finite) return -1;
    const bool conv = rmax <= tol;
    if (!conv && it >= max_iter) return -2;
    float A[N * (N + 1) / 2];
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
        for (int j = 0; j <= i; j++)
            A[tri(i, j)] = Mom[tix(bx<D, FLUON>(i) + bx<D, FLUON>(j), by<D, FLUON>(i) + by<D, FLUON>(j), P)];
    if (!ldlt_solve<float, N>(A, r)) return -1;
#pragma unroll
    for (int j = 0; j < N; j++) lam[j] += r[j];
    return conv ? 1 : 0;
}

template <int D, bool FLUON>
__device__ __forceinline__ int newton_step(const double* Mom, const double* con, double* lam, const Model& m, int it) {
    return newton_step_tol<D, FLUON>(Mom, con, lam, m.tol, m.max_iter, it);
}

// Joint Newton iterations of the fluon and phonon multipliers: every pass
// accumulates the moments of each population that is still iterating.
// sf, sg: number of updates (>= 0) or failure (< 0).
template <int D>
__device__ __forceinline__ void solve_fg(const CellState<D>& c, const Stencil<D>& st, const double* conF,
                                         const double* conG, bool has_g, double* lf, double* lg, const Model& m,
                                         int& sf, int& sg, unsigned int& npf, unsigned int& npg) {
    using MS = MomentSet<D>;
    bool fa = true, ga = has_g;
    sf = 0;
    sg = 0;
    for (int it = 0; fa || ga; it++) {
        double MF[MS::NF], MG[MS::NG];
        const unsigned long long q = moment_pass<D>(c, st, lf, lg, fa, ga, MF, MG);
        // phonons first: their moments are dead before the larger fluon system is built
        if (ga) {
            npg += q;
            const int r = newton_step<D, false>(MG, conG, lg, m, it);
            if (r < 0) {
                sg = r;
                ga = false;
            } else {
                sg++;
                if (r == 1) ga = false;
            }
        }
        if (fa) {
            npf += q;
            const int r = newton_step<D, true>(MF, conF, lf, m, it);
            if (r < 0) {
                sf = r;
                fa = false;
            } else {
                sf++;
                if (r == 1) fa = false;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Mixed precision: the Newton passes over the velocity set run in FP32 (FP32 is
// about 60x the FP64 rate on GB300); the small Cholesky solves stay FP64.  The
// FP32 iterate is then corrected by one full FP64 Newton pass, and the
// streaming pass checks the FP64 residual of exactly the populations it
// deposits against the same tolerance as the FP64 path.
// ---------------------------------------------------------------------------
// Coefficients of the FP32 exponent polynomials on the row y (as row_coeffs).
template <int D>
__device__ __forceinline__ void row_coeffs32(const float* lf, const float* lg, float y, float* cf, float* cg) {
    if constexpr (D == 1) {
        cf[0] = 1.f + lf[0];
        cf[1] = lf[1];
        cf[2] = lf[2];
        cf[3] = lf[3];
        cg[0] = 1.f + lg[0];
        cg[1] = lg[1];
        cg[2] = lg[2];
    } else {
        cf[0] = 1.f + lf[0] + y * (lf[2] + y * (lf[5] + y * lf[9]));
        cf[1] = lf[1] + y * (lf[4] + y * lf[7]);
        cf[2] = lf[3] + y * lf[8];
        cf[3] = lf[6];
        cg[0] = 1.f + lg[0] + y * (lg[2] + y * lg[5]);
        cg[1] = lg[1] + y * lg[4];
        cg[2] = lg[3];
    }
}

// One FP32 pass over the velocity set (row table when valid, else Stencil)
// accumulating the population moments of f (doF) and g (doG) for the FP32
// multipliers lf, lg.  Returns the point count.
// TAB: the caller guarantees a valid row table (no Stencil fallback compiled in).
template <int D, bool TAB = false>
__device__ __forceinline__ unsigned long long moment_pass32(const CellState<D>& c, const Stencil<D>& st,
                                                            const RowTable<D>& tab, const float* lf, const float* lg,
                                                            bool doF, bool doG, float* MF, float* MG) {
    using MS = MomentSet<D>;
#pragma unroll
    for (int i = 0; i < MS::NF; i++) MF[i] = 0.f;
#pragma unroll
    for (int i = 0; i < MS::NG; i++) MG[i] = 0.f;
    unsigned long long q = 0;
    const float s32 = tab.s32;
    // a point (x, y) of weight w, folded into the moments directly
    auto add_point = [&](float x, float y, float w) {
        float cf[4], cg[3];
        row_coeffs32<D>(lf, lg, y, cf, cg);
        static_assert(MS::PF == 6, "moment degree of the FP32 pass");
        const float x2 = x * x, x3 = x2 * x, x4 = x2 * x2, y2 = y * y, y3 = y2 * y, y4 = y2 * y2;
        const float px[7] = {1.f, x, x2, x3, x4, x4 * x, x3 * x3};
        const float py[7] = {1.f, y, y2, y3, y4, y4 * y, y3 * y3};
        if (doF) {
            const float f = w * __expf(-fmaf(x2, fmaf(cf[3], x, cf[2]), fmaf(cf[1], x, cf[0])));
#pragma unroll
            for (int b = 0; b <= (D == 2 ? MS::PF : 0); b++)
#pragma unroll
                for (int a = 0; a + b <= MS::PF; a++) MF[tix(a, b, MS::PF)] += px[a] * py[b] * f;
        }
        if (doG) {
            const float g = w * __expf(-fmaf(x2, cg[2], fmaf(cg[1], x, cg[0])));
#pragma unroll
            for (int b = 0; b <= (D == 2 ? MS::PG : 0); b++)
#pragma unroll
                for (int a = 0; a + b <= MS::PG; a++) MG[tix(a, b, MS::PG)] += px[a] * py[b] * g;
        }
        q++;
    };
    // np points at thermal x = x0 + k dx on the row at thermal y, each of weight wgt
    auto sweep = [&](float y, float x0, float dx, int np, float wgt) {
        float cfv[4], cgv[3];
        row_coeffs32<D>(lf, lg, y, cfv, cgv);
        const float cf0 = cfv[0], cf1 = cfv[1], cf2 = cfv[2], cf3 = cfv[3];
        const float cg0 = cgv[0], cg1 = cgv[1], cg2 = cgv[2];
        float SF[MS::PF + 1], SG[MS::PG + 1];
#pragma unroll
        for (int a = 0; a <= MS::PF; a++) SF[a] = 0.f;
#pragma unroll
        for (int a = 0; a <= MS::PG; a++) SG[a] = 0.f;
        // one point: powers and exponents as shallow trees (x^6 = (x^3)^2, Estrin's
        // scheme for the polynomials), so that two points in flight overlap well
        static_assert(MS::PF == 6 && MS::PG == 4, "moment degrees of the FP32 pass");
        auto point = [&](float x) {
            const float x2 = x * x;
            const float x3 = x2 * x, x4 = x2 * x2;
            const float pw[7] = {1.f, x, x2, x3, x4, x4 * x, x3 * x3};
            if (doF) {
                const float f = __expf(-fmaf(x2, fmaf(cf3, x, cf2), fmaf(cf1, x, cf0)));
#pragma unroll
                for (int a = 0; a <= MS::PF; a++) SF[a] = fmaf(pw[a], f, SF[a]);
            }
            if (doG) {
                const float g = __expf(-fmaf(x2, cg2, fmaf(cg1, x, cg0)));
#pragma unroll
                for (int a = 0; a <= MS::PG; a++) SG[a] = fmaf(pw[a], g, SG[a]);
            }
        };
        float kf = 0.f;  // the point index as a float (exact), with no conversion per point
        int k = 0;
        for (; k + 2 <= np; k += 2, kf += 2.f) {
            point(fmaf(kf, dx, x0));
            point(fmaf(kf + 1.f, dx, x0));
        }
        if (k < np) point(fmaf(kf, dx, x0));
        q += (unsigned long long)np;
        if (wgt != 1.f) {
#pragma unroll
            for (int a = 0; a <= MS::PF; a++) SF[a] *= wgt;
#pragma unroll
            for (int a = 0; a <= MS::PG; a++) SG[a] *= wgt;
        }
        if constexpr (D == 1) {
#pragma unroll
            for (int a = 0; a <= MS::PF; a++) MF[a] += SF[a];
#pragma unroll
            for (int a = 0; a <= MS::PG; a++) MG[a] += SG[a];
        } else {
            float yp[MS::PF + 1];
            yp[0] = 1.f;
#pragma unroll
            for (int e = 1; e <= MS::PF; e++) yp[e] = yp[e - 1] * y;
#pragma unroll
            for (int b = 0; b <= MS::PF; b++)
#pragma unroll
                for (int a = 0; a + b <= MS::PF; a++) MF[tix(a, b, MS::PF)] = fmaf(SF[a], yp[b], MF[tix(a, b, MS::PF)]);
#pragma unroll
            for (int b = 0; b <= MS::PG; b++)
#pragma unroll
                for (int a = 0; a + b <= MS::PG; a++) MG[tix(a, b, MS::PG)] = fmaf(SG[a], yp[b], MG[tix(a, b, MS::PG)]);
        }
    };
    auto row = [&](int cy, int xa, int xb) { sweep(D == 2 ? tab.ty(cy) : 0.f, tab.tx(xa), s32, xb - xa + 1, 1.f); };
    if (TAB || tab.ok) {
        // level-0 runs as rows; the children of the split points a..b of a row as child rows
        // (cy -/+ 1/4) of 2 (b - a + 1) points at p -/+ 1/4, spacing 1/2, weight 2^-D each
        constexpr float wch = D == 1 ? 0.5f : 0.25f;
#pragma unroll 1
        for (int r = 0; r < (D == 2 ? tab.nrows : 1); r++) {
            int rx0, rx1, ra, rb, cy = 0;
            if constexpr (D == 2) {
                tab.row_ext(r, rx0, rx1, ra, rb);
                cy = tab.y_first + r;
            } else {
                rx0 = tab.x0;
                rx1 = tab.x1;
                ra = tab.a;
                rb = tab.b;
            }
            if (ra <= rb) {
                if (rx0 <= ra - 1) row(cy, rx0, ra - 1);
                if (rb + 1 <= rx1) row(cy, rb + 1, rx1);
#pragma unroll 1
                for (int sy = (D == 2 ? -1 : 0); sy <= (D == 2 ? 1 : 0); sy += 2)
                    sweep(D == 2 ? tab.ty(cy, 0.25f * (float)sy) : 0.f, tab.tx(ra, -0.25f), 0.5f * s32,
                          2 * (rb - ra + 1), wch);
            } else if (rx0 <= rx1) {
                row(cy, rx0, rx1);
            }
        }
    } else if constexpr (!TAB) {
        auto leaf = [&](const double* cp, double dC) {
            add_point((float)((cp[0] - c.u[0]) * c.inv_sig), D == 2 ? (float)((cp[D - 1] - c.u[D - 1]) * c.inv_sig) : 0.f,
                      (float)dC);
        };
        st.for_each_row(row, leaf);
    }
    return q;
}

// FP32 Newton phase followed by one FP64 Newton pass.  Returns false when a
// solve broke down (the caller then runs the plain FP64 solve).  sf, sg count
// the FP64 updates; np32 counts the points of the FP32 passes.
template <int D>
__device__ __forceinline__ bool solve_fg_mixed(const CellState<D>& c, const Stencil<D>& st, const RowTable<D>& tab,
                                               const double* conF, const double* conG, bool has_g, double* lf,
                                               double* lg, const Model& m, int& sf, int& sg, unsigned int& npf,
                                               unsigned int& npg, unsigned int& np32) {
    using MS = MomentSet<D>;
    constexpr int NF = Basis<D, true>::N, NG = Basis<D, false>::N;
    constexpr float tol32 = 2e-5f;  // thermal units; the FP64 pass takes it to round-off
    constexpr int max32 = 12;
    float lf32[NF], lg32[NG], cf32[NF], cg32[NG];
#pragma unroll
    for (int j = 0; j < NF; j++) {
        lf32[j] = (float)lf[j];
        cf32[j] = (float)conF[j];
    }
#pragma unroll
    for (int j = 0; j < NG; j++) {
        lg32[j] = (float)lg[j];
        cg32[j] = (float)conG[j];
    }
    bool fa = true, ga = has_g;
    for (int it = 0; (fa || ga) && it < max32; it++) {
        float MF32[MS::NF], MG32[MS::NG];
        np32 += moment_pass32<D>(c, st, tab, lf32, lg32, fa, ga, MF32, MG32);
        if (ga) {
            const int r = newton_step32<D, false>(MG32, cg32, lg32, tol32, max32, it);
            if (r < 0) return false;
            if (r == 1) ga = false;
        }
        if (fa) {
            const int r = newton_step32<D, true>(MF32, cf32, lf32, tol32, max32, it);
            if (r < 0) return false;
            if (r == 1) fa = false;
        }
    }
#pragma unroll
    for (int j = 0; j < NF; j++) lf[j] = (double)lf32[j];
#pragma unroll
    for (int j = 0; j < NG; j++) lg[j] = (double)lg32[j];
    double MF[MS::NF], MG[MS::NG];
    const unsigned long long q = moment_pass<D>(c, st, lf, lg, true, has_g, MF, MG);
    sg = 0;
    if (has_g) {
        npg += q;
        if (newton_step_tol<D, false>(MG, conG, lg, m.tol, 1, 0) < 0) return false;
        sg = 1;
    }
    npf += q;
    if (newton_step_tol<D, true>(MF, conF, lf, m.tol, 1, 0) < 0) return false;
    sf = 1;
    return true;
}

// FP32 Newton alone (the FP32 path): FP32 passes and FP32 solves until the FP32
// residual is within tol32 (thermal units), the polishing update included, on FP32
// multipliers lf32, lg32 (in: the start, out: the solution).  Newton converges
// quadratically here, so the polishing update takes a residual of 3e-4 to about 1e-7,
// the FP32 noise floor of the passes: a tighter stop costs passes and buys nothing.
// Returns false on a breakdown or at the iteration cap (the caller then runs the FP64
// EPR).  sf, sg count the FP32 updates; np32 the points of the FP32 passes.
template <int D, bool TAB = false>
__device__ __forceinline__ bool solve_fg32(const CellState<D>& c, const Stencil<D>& st, const RowTable<D>& tab,
                                           const float* cf32, const float* cg32, bool has_g, float* lf32,
                                           float* lg32, int& sf, int& sg, unsigned int& np32) {
    using MS = MomentSet<D>;
    constexpr float tol32 = 3e-4f;
    constexpr int max32 = 16;
    bool fa = true, ga = has_g;
    sf = 0;
    sg = 0;
    for (int it = 0; fa || ga; it++) {
        float MF32[MS::NF], MG32[MS::NG];
        np32 += moment_pass32<D, TAB>(c, st, tab, lf32, lg32, fa, ga, MF32, MG32);
        if (ga) {
            const int r = newton_step32<D, false>(MG32, cg32, lg32, tol32, max32, it);
            if (r < 0) return false;
            sg++;
            if (r == 1) ga = false;
        }
        if (fa) {
            const int r = newton_step32<D, true>(MF32, cf32, lf32, tol32, max32, it);
            if (r < 0) return false;
            sf++;
            if (r == 1) fa = false;
        }
    }
    return true;
}

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

}  // namespace lbm
