// Double-float finish of the EPR Newton (Eq. IID7-IID11) for the mixed path
// (LELBM_MIXED) on the FP32 pipe.  GB300 runs FP64 at 1/64 of the FP32 rate, so the
// part of the solve that needs more than FP32 precision -- the residual that the
// 1e-12 tolerance of Sec. II.D judges, and the populations that moment streaming
// (Eq. IIE3) deposits -- is evaluated in double-float arithmetic: a value is the
// unevaluated sum h + l of two FP32 numbers (Dekker 1971), about 48 significant bits.
//
// Per population and stencil point the work is FP32 and integer only:
//   - the exponent -(1 + lambda . T(t)) / ln 2 is a polynomial in the lattice offsets
//     (X, Y) of the point from floor(u); its coefficients are rounded once per cell to
//     int64 fixed point, and along a stencil row it is advanced by forward differences
//     in exact integer arithmetic, so every point gets the exact value of the rounded
//     polynomial (children of split points get it by an exact Horner evaluation);
//   - 2^w is evaluated from the fixed-point w by a table-driven method (Tang, ACM TOMS
//     15, 1989): w = n + j/512 + rho, 2^(j/512) from a double-float table, 2^rho =
//     exp(rho ln 2) by its Taylor series (|rho ln 2| < 1.4e-3, four terms);
//   - the residual moments sum x^a f over a row in double-float with Knuth's TwoSum
//     and the FMA-based TwoProduct, in lattice units where x^a is exact.
// The FP64 pipe keeps only per-cell work (coefficient set-up, the lattice -> thermal
// moment transform of the residual).
#pragma once

#include <cstdint>

#include "lelbm_device.cuh"
#include "lelbm_internal.h"
#include "lelbm_land.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// FP32 <-> FP64 bit helpers (integer operations only; GB300's FP64 pipe also runs
// the FP32 <-> FP64 conversion instructions).
// ---------------------------------------------------------------------------
// Subnormals become zero.
__device__ __forceinline__ float flush_sub(float v) { return (__float_as_uint(v) & 0x7f800000u) ? v : 0.f; }

// FP32 -> FP64: the exponent is rebiased from 127 to 1023 by one addition and the
// mantissa shifted into place.  Normal numbers widen exactly; zeros and subnormals give
// zero.  Infinities and NaNs, which a converged solve does not produce, come out finite.
__device__ __forceinline__ double widen(float v) {
    const unsigned int b = __float_as_uint(v);
    const bool tiny = (b & 0x7f800000u) == 0u;
    const unsigned int hi = (((b >> 3) & 0x0fffffffu) + 0x38000000u) | (b & 0x80000000u);
    return __hiloint2double(tiny ? 0 : (int)hi, tiny ? 0 : (int)(b << 29));
}

// ---------------------------------------------------------------------------
// Error-free transformations (explicitly rounded, so they cannot be contracted).
// ---------------------------------------------------------------------------
// Knuth's TwoSum: s + e = a + b exactly, for any a, b.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Dekker's Fast2Sum: s + e = a + b exactly when |a| >= |b| (or a = 0).
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// TwoProduct with a fused multiply-add: p + e = a b exactly.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Double-float accumulator.  The low word collects the exact rounding errors of the
// high-word additions and the low words of the terms; it is not renormalised between
// additions (n terms lose about n 2^-48 relative, far below what the residual needs).
struct DFAcc {
    float h, l;
    __device__ __forceinline__ void zero() { h = l = 0.f; }
    __device__ __forceinline__ void add(float vh, float vl) {
        float s, e;
        two_sum(h, vh, s, e);
        h = s;
        l = __fadd_rn(l, __fadd_rn(e, vl));
    }
    // += k (vh + vl), with the product of k and vh formed exactly
    __device__ __forceinline__ void add_scaled(float k, float vh, float vl) {
        float p, pe;
        two_prod(k, vh, p, pe);
        add(p, __fmaf_rn(k, vl, pe));
    }
    __device__ __forceinline__ double value() const { return widen(h) + widen(l); }
};

// (ah + al)(bh + bl) as a normalised double-float (the al bl term, below 2^-48 of the
// product, is dropped).
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float& ph, float& pl) {
    float p, e;
    two_prod(ah, bh, p, e);
    e = __fadd_rn(e, __fmaf_rn(ah, bl, __fmul_rn(al, bh)));
    fast_two_sum(p, e, ph, pl);
}

// FP64 -> double-float (per-cell set-up only).
__device__ __forceinline__ void df_split(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// ---------------------------------------------------------------------------
// 2^w for a fixed-point exponent (Tang's table-driven method).
// ---------------------------------------------------------------------------
constexpr int kFixBits = 54;                           // fractional bits of the exponents
constexpr double kFixOne = 18014398509481984.0;        // 2^54
constexpr double kFixBound = 200.0;                    // |exponent| bound (int64 holds 512)
constexpr int kExpTab = 512;                           // table entries 2^(j/512)
constexpr double kLn2 = 0.69314718055994530941723212145818;
constexpr double kLog2e = 1.44269504088896340735992468100189;
constexpr float kLn2H = (float)kLn2;
constexpr float kLn2L = (float)(kLn2 - (double)kLn2H);
constexpr float kRhoH = kLn2H * 4.656612873077392578125e-10f;   // ln2_hi 2^-31
constexpr float kRhoM = kLn2L * 4.656612873077392578125e-10f;   // ln2_lo 2^-31
constexpr float kRhoL = kLn2H * 5.5511151231257827e-17f;        // ln2_hi 2^-54

// Each block fills the table once: entry j = 2^(j/512) as a double-float.
__device__ __forceinline__ void exp2_table_init(float2* tab) {
    for (int j = threadIdx.x; j < kExpTab; j += blockDim.x) {
        const double v = exp2((double)j * (1.0 / kExpTab));
        const float h = (float)v;
        tab[j] = make_float2(h, (float)(v - (double)h));
    }
}

// fh + fl = 2^(w 2^-54 + dn) to about 2^-47 relative (the precision of a double-float).  w = n + j/512 + rho with
// n = floor, j the next 9 bits and rho in [0, 2^-9) the remaining 45 bits (split into
// two exact FP32 integers); exp(r) - 1 for r = rho ln 2 < 1.36e-3 by r + r^2/2 + r^3/6 +
// r^4/24 (the r^5 term is below 4e-17).  Results below 2^-126 are zero.
__device__ __forceinline__ void exp2_fix(long long w, const float2* __restrict__ tab, int dn, float& fh, float& fl) {
    const int hi = (int)(w >> 32);
    const unsigned lo = (unsigned)w;
    int n = (hi >> 22) + dn;
    const int j = (hi >> 13) & (kExpTab - 1);
    const unsigned ih = ((unsigned)(hi & 0x1fff) << 9) | (lo >> 23);  // bits 23..44
    const unsigned il = lo & 0x7fffffu;                                // bits 0..22
    const float rh = __fsub_rn(__uint_as_float(0x4b000000u | ih), 8388608.f);
    const float rl = __fsub_rn(__uint_as_float(0x4b000000u | il), 8388608.f);
    float r, re;
    two_prod(rh, kRhoH, r, re);
    const float rlo = __fmaf_rn(rh, kRhoM, __fmaf_rn(rl, kRhoL, re));
    float s, se;
    two_prod(r, r, s, se);
    const float c = __fmaf_rn(r, 1.f / 24.f, 1.f / 6.f);
    const float t = __fmaf_rn(__fmul_rn(s, r), c, __fmul_rn(r, rlo));
    float eh, ee;
    fast_two_sum(r, __fmul_rn(0.5f, s), eh, ee);
    const float el = __fadd_rn(ee, __fadd_rn(rlo, __fmaf_rn(0.5f, se, t)));
    const float2 T = tab[j];
    float ph, pe;
    two_prod(T.x, eh, ph, pe);
    const float q = __fadd_rn(pe, __fmaf_rn(T.x, el, __fmaf_rn(T.y, eh, T.y)));
    float Rh, Re;
    fast_two_sum(T.x, ph, Rh, Re);
    const float Rl = __fadd_rn(Re, q);
    n = n > 127 ? 127 : n;
    const float sc = n >= -126 ? __int_as_float((n + 127) << 23) : 0.f;
    fh = __fmul_rn(Rh, sc);
    fl = __fmul_rn(Rl, sc);
}

// ---------------------------------------------------------------------------
// The exponent polynomial of one population in fixed point.
// ---------------------------------------------------------------------------
template <int D, bool FLUON>
struct DFPop {
    static constexpr int P = FLUON ? 3 : 2;                                    // exponent degree
    static constexpr int PJ = FLUON ? MomentSet<D>::PF : MomentSet<D>::PG;     // Jacobian moment degree
    static constexpr int NB = D == 1 ? P + 1 : (P + 1) * (P + 2) / 2;          // coefficients
    static constexpr int NJ = D == 1 ? PJ + 1 : (PJ + 1) * (PJ + 2) / 2;       // Jacobian moments
    static constexpr int N = Basis<D, FLUON>::N;                               // constraints
    __device__ __forceinline__ static constexpr int ix(int a, int b) { return D == 1 ? a : tix(a, b, P); }
};

// Coefficients beta[ix(a, b)] of X^a Y^b in w(X, Y) = -log2(e) (1 + sum_j lam_j T_j(t)),
// t = ((X - fx) s, (Y - fy) s), as int64 with kFixBits fractional bits; (X, Y) are the
// lattice offsets of a velocity from (floor u_x, floor u_y), (fx, fy) = u - floor(u) and
// s = 1 / sqrt(RT).  Returns false when the polynomial can exceed kFixBound on the offsets
// |X|, |Y| <= xm (the int64 evaluation would then not be safe).
template <int D, bool FLUON>
__device__ __forceinline__ bool fix_poly(const double* lam, double s, double fx, double fy, double xm,
                                         long long* beta) {
    using Q = DFPop<D, FLUON>;
    constexpr int P = Q::P, NB = Q::NB;
    double d[NB];
#pragma unroll
    for (int k = 0; k < NB; k++) d[k] = 0.0;
#pragma unroll
    for (int j = 0; j < Q::N; j++) d[Q::ix(bx<D, FLUON>(j), by<D, FLUON>(j))] = lam[j];
    d[0] += 1.0;
    double sp[P + 1];
    sp[0] = -kLog2e;
#pragma unroll
    for (int k = 1; k <= P; k++) sp[k] = sp[k - 1] * s;
#pragma unroll
    for (int b = 0; b <= (D == 2 ? P : 0); b++)
#pragma unroll
        for (int a = 0; a + b <= P; a++) d[Q::ix(a, b)] *= sp[a + b];
    // Taylor shift by -fx along X (each power of Y), then by -fy along Y
#pragma unroll
    for (int b = 0; b <= (D == 2 ? P : 0); b++) {
        const int n = P - b;
#pragma unroll
        for (int k = 0; k < P; k++)
#pragma unroll
            for (int i = P - 1; i >= 0; i--)
                if (k < n && i >= k && i < n) d[Q::ix(i, b)] = fma(-fx, d[Q::ix(i + 1, b)], d[Q::ix(i, b)]);
    }
    if constexpr (D == 2) {
#pragma unroll
        for (int a = 0; a <= P; a++) {
            const int n = P - a;
#pragma unroll
            for (int k = 0; k < P; k++)
#pragma unroll
                for (int i = P - 1; i >= 0; i--)
                    if (k < n && i >= k && i < n) d[Q::ix(a, i)] = fma(-fy, d[Q::ix(a, i + 1)], d[Q::ix(a, i)]);
        }
    }
    double bound = 0.0;
    double xp[P + 1];
    xp[0] = 1.0;
#pragma unroll
    for (int k = 1; k <= P; k++) xp[k] = xp[k - 1] * xm;
#pragma unroll
    for (int b = 0; b <= (D == 2 ? P : 0); b++)
#pragma unroll
        for (int a = 0; a + b <= P; a++) bound += fabs(d[Q::ix(a, b)]) * xp[a] * xp[b];
    if (!(bound < kFixBound)) return false;
#pragma unroll
    for (int k = 0; k < NB; k++) beta[k] = __double2ll_rn(d[k] * kFixOne);
    return true;
}

// Row coefficients gamma_a(Y) = sum_b beta_ab Y^b of the polynomial on the integer row Y.
template <int D, bool FLUON>
__device__ __forceinline__ void fix_row(const long long* beta, int Y, long long* gm) {
    using Q = DFPop<D, FLUON>;
    if constexpr (D == 1) {
#pragma unroll
        for (int a = 0; a <= Q::P; a++) gm[a] = beta[a];
    } else {
        const long long y = Y;
#pragma unroll
        for (int a = 0; a <= Q::P; a++) {
            long long v = beta[Q::ix(a, Q::P - a)];
#pragma unroll
            for (int b = Q::P - a - 1; b >= 0; b--) v = v * y + beta[Q::ix(a, b)];
            gm[a] = v;
        }
    }
}

// Child rows: X = m/4, Y = n4/4 (quarter offsets).  Returns the coefficients B_a of
// N(m) = sum_a B_a m^a = 64 w, with beta shifted to 48 fractional bits first, so that N
// carries kFixBits fractional bits and every partial sum stays below 2^62 (|w| < 200).
template <int D, bool FLUON>
__device__ __forceinline__ void fix_child_row(const long long* beta, int n4, long long* B) {
    using Q = DFPop<D, FLUON>;
    const long long y = n4;
#pragma unroll
    for (int a = 0; a <= Q::P; a++) {
        long long v = 0;
        if constexpr (D == 1) {
            v = (beta[a] >> 6) * (1LL << (2 * (3 - a)));
        } else {
#pragma unroll
            for (int b = Q::P - a; b >= 0; b--) v = v * y + (beta[Q::ix(a, b)] >> 6) * (1LL << (2 * (3 - a - b)));
        }
        B[a] = v;
    }
}

// w (kFixBits fractional bits) of the child at quarter offset m on a child row.
template <int P>
__device__ __forceinline__ long long fix_child_w(const long long* B, int m) {
    const long long x = m;
    long long v = B[P];
#pragma unroll
    for (int a = P - 1; a >= 0; a--) v = v * x + B[a];
    return v;
}

// Moments K_i = sum_a C(i, a) (-h)^(i - a) L_a of a distribution about a new origin h.
template <int P>
__device__ __forceinline__ void origin_shift(const double* L, double h, double* K) {
#pragma unroll
    for (int i = 0; i <= P; i++) {
        double acc = 0.0, hp = 1.0, bin = 1.0;
#pragma unroll
        for (int a = i; a >= 0; a--) {
            acc = fma(bin * hp, L[a], acc);
            hp *= -h;
            bin = bin * (double)a / (double)(i - a + 1);
        }
        K[i] = acc;
    }
}

// ---------------------------------------------------------------------------
// One double-float pass of one population over the row table.
//   DF_CORR:   residual (double-float sums) and the FP32 Jacobian moments MJ in thermal
//              units (as moment_pass32 accumulates them) at the multipliers lam;
//   DF_STREAM: residual and moment streaming of the populations (sign = -1 takes a
//              previous deposit back).
// The residual r (thermal units, FP64) and rmax are returned.  False: the exponent is
// out of the fixed-point range (the caller falls back to the FP64 solve).
// ---------------------------------------------------------------------------
enum : int { DF_CORR = 0, DF_STREAM = 1 };

struct DFStream {
    const Geometry* g;
    const uint8_t* type;
    double* Mout;
    long long cell;
    long long lo;   // 1D: first interior cell of the instance
    int n;          // 1D: interior length of the instance
    int ix, iy;     // 2D: padded coordinates of the cell
    bool near_wall;
    float mh, ml;   // rho dV (fluons) or rho K RT dV (phonons), signed, as a double-float
    long long* beta;  // the thread's slot for the exponent coefficients (shared memory)
};

// Out of line: one object per (dimension, population, mode), called two to three times per
// cell; the cell enters as u (ux, uy) and 1 / sqrt(RT) only.  beta: a per-thread slot of
// DFPop::NB fixed-point coefficients (shared memory).
template <int D, bool FLUON, int MODE>
static __device__ __noinline__ bool df_pass(double ux, double uy, double inv_sig, const RowTable<D>& tab_in,
                                            const double* __restrict__ lam, const double* __restrict__ con,
                                            const float2* __restrict__ etab, double xm, double* __restrict__ r_out,
                                            double& rmax_out, float* __restrict__ MJ_out, const DFStream& ds_in,
                                            LocalStats& ls, unsigned int& npts, long long* __restrict__ beta) {
    using Q = DFPop<D, FLUON>;
    constexpr int P = Q::P, PJ = Q::PJ, NB = Q::NB;
    // private copies (registers): nothing the pass writes can alias them
    const RowTable<D> tab = tab_in;
    const DFStream ds = ds_in;
    float MJ[MODE == DF_CORR ? Q::NJ : 1];
    const double fx = ux - (double)tab.xc;
    const double fy = D == 2 ? uy - (double)tab.yc : 0.0;
    // beta: the cell's slot in shared memory (read at every row start)
    if (!fix_poly<D, FLUON>(lam, inv_sig, fx, fy, xm, beta)) return false;
    DFAcc L[NB];
#pragma unroll
    for (int k = 0; k < NB; k++) L[k].zero();
    if constexpr (MODE == DF_CORR) {
#pragma unroll
        for (int k = 0; k < Q::NJ; k++) MJ[k] = 0.f;
    }
    const float s32 = tab.s32;
    unsigned long long q = 0;
    long long walls = 0;
    int dmax = 0;
    // deposit of T_N(c) m (m = ds.m f) at cell tgt: the population's stored moments, each
    // as two FP64 atomic additions (the high and the low word, both widened exactly)
    auto put = [&](long long tgt, int mm, float T, float vh, float vl) {
        if (T == 0.f) return;
        float p, e;
        two_prod(T, vh, p, e);
        e = __fmaf_rn(T, vl, e);
        double* a = ds.Mout + (long long)mm * ds.g->ncell + tgt;
        atomicAdd(a, widen(p));
        atomicAdd(a, widen(e));
    };
    auto deposit = [&](long long tgt, float cx, float cy, float vh, float vl) {
        if (tgt < 0 || !lands_on_fluid<D>(*ds.g, ds.type, tgt)) return;
        if constexpr (FLUON) {
            put(tgt, 0, 1.f, vh, vl);
            put(tgt, 1, cx, vh, vl);
            if constexpr (D == 2) put(tgt, 2, cy, vh, vl);
            put(tgt, iM2<D>(0, 0), cx * cx, vh, vl);
            const float csq = D == 2 ? fmaf(cx, cx, cy * cy) : cx * cx;
            if constexpr (D == 2) {
                put(tgt, iM2<D>(0, 1), cx * cy, vh, vl);
                put(tgt, iM2<D>(1, 1), cy * cy, vh, vl);
                put(tgt, iMD<D>(1), csq * cy, vh, vl);
            }
            put(tgt, iMD<D>(0), csq * cx, vh, vl);
        } else {
            put(tgt, iG0<D>(), 1.f, vh, vl);
            put(tgt, iG1<D>(0), cx, vh, vl);
            if constexpr (D == 2) put(tgt, iG1<D>(1), cy, vh, vl);
        }
    };
    // a streamed point at lattice velocity (cx, cy) of population weight f; refined points
    // (frac != 0) are shared by cloud-in-cell weights
    auto stream_point = [&](float cx, float cy, float fh, float fl, bool refined) {
        float vh, vl;
        df_mul(ds.mh, ds.ml, fh, fl, vh, vl);
        if constexpr (D == 2) {
            if (ds.near_wall) {
                const double cpd[2] = {(double)cx, (double)cy};
                const double v = widen(vh) + widen(vl);
                const bool hit =
                    stream_traced(*ds.g, ds.type, ds.Mout, ds.ix, ds.iy, cpd, FLUON ? v : 0.0, FLUON ? 0.0 : v);
                if (FLUON && hit) walls += ds.mh > 0.f ? 1 : -1;  // a path is counted once, with its fluons
                return;
            }
        }
        if (!refined) {
            deposit(land<D>(*ds.g, ds.cell, ds.lo, ds.n, ds.ix, ds.iy, (int)cx, (int)cy), cx, cy, vh, vl);
            return;
        }
        // children sit at +-1/4: along each axis 3/4 on the nearer cell, 1/4 on the other
        const float flx = floorf(cx), fly = floorf(cy);
        const float w1x = cx - flx, w1y = cy - fly;
#pragma unroll 1
        for (int sy = 0; sy < (D == 2 ? 2 : 1); sy++)
#pragma unroll 1
            for (int sx = 0; sx < 2; sx++) {
                float w = sx ? w1x : 1.f - w1x;
                if constexpr (D == 2) w *= sy ? w1y : 1.f - w1y;
                float sh, sl;
                two_prod(w, vh, sh, sl);
                sl = __fmaf_rn(w, vl, sl);
                deposit(land<D>(*ds.g, ds.cell, ds.lo, ds.n, ds.ix, ds.iy, (int)flx + sx, D == 2 ? (int)fly + sy : 0),
                        cx, cy, sh, sl);
            }
    };
    // folds the row sums S (residual) and SJ (Jacobian) of a row at lattice offset Yf
    // (thermal y32) into the cell moments
    auto fold = [&](const DFAcc* S, const float* SJ, float Yf, float y32) {
        if constexpr (D == 1) {
#pragma unroll
            for (int a = 0; a <= P; a++) L[a].add(S[a].h, S[a].l);
            if constexpr (MODE == DF_CORR) {
#pragma unroll
                for (int a = 0; a <= PJ; a++) MJ[a] += SJ[a];
            }
        } else {
            float yp = 1.f;
#pragma unroll
            for (int b = 0; b <= P; b++) {
#pragma unroll
                for (int a = 0; a + b <= P; a++) L[Q::ix(a, b)].add_scaled(yp, S[a].h, S[a].l);
                yp *= Yf;
            }
            if constexpr (MODE == DF_CORR) {
                float yq = 1.f;
#pragma unroll
                for (int b = 0; b <= PJ; b++) {
#pragma unroll
                    for (int a = 0; a + b <= PJ; a++) MJ[tix(a, b, PJ)] = fmaf(SJ[a], yq, MJ[tix(a, b, PJ)]);
                    yq *= y32;
                }
            }
        }
    };
    // one point of a row: residual sums at lattice offset Xf, Jacobian sums at thermal x
    auto accumulate = [&](DFAcc* S, float* SJ, float Xf, float fh, float fl) {
        S[0].add(fh, fl);
        S[1].add_scaled(Xf, fh, fl);
        const float X2 = Xf * Xf;
        S[2].add_scaled(X2, fh, fl);
        if constexpr (P == 3) S[3].add_scaled(X2 * Xf, fh, fl);
        if constexpr (MODE == DF_CORR) {
            const float x = fmaf(Xf, s32, -tab.fux);
            const float x2 = x * x, x3 = x2 * x, x4 = x2 * x2;
            const float pw[7] = {1.f, x, x2, x3, x4, x4 * x, x3 * x3};
#pragma unroll
            for (int a = 0; a <= PJ; a++) SJ[a] = fmaf(pw[a], fh, SJ[a]);
        }
    };
    // Every segment of a row -- its level-0 runs (lattice step 1) and, for split points, its
    // child rows (children at p -/+ 1/4, step 1/2, weight 2^-D) -- is one arithmetic
    // progression of points along x, swept by the same loop: the exponent advances by exact
    // forward differences D0..D3 (int64, kFixBits fractional bits) from its first point.
    const int nrows = D == 2 ? tab.nrows : 1;
#pragma unroll 1
    for (int rr = 0; rr < nrows; rr++) {
        int rx0, rx1, ra, rb, cy = 0;
        if constexpr (D == 2) {
            tab.row_ext(rr, rx0, rx1, ra, rb);
            cy = tab.y_first + rr;
        } else {
            rx0 = tab.x0;
            rx1 = tab.x1;
            ra = tab.a;
            rb = tab.b;
        }
        const int Y = cy - tab.yc;
        const bool split = ra <= rb;
        long long gm[P + 1];
        if (rx0 <= rx1) fix_row<D, FLUON>(beta, Y, gm);
        // segments 0, 1: level-0 runs rx0..ra-1 and rb+1..rx1 (the whole row when no point
        // splits); 2 (and 3 in 2D): the child rows at cy - 1/4 and cy + 1/4
#pragma unroll 1
        for (int seg = 0; seg < (D == 2 ? 4 : 3); seg++) {
            long long D0, D1, D2 = 0, D3 = 0;
            float Xf, h, Yf, y32;
            int np, dn;
            if (seg < 2) {
                if (rx0 > rx1 || (seg == 1 && !split)) continue;
                const int xa = seg == 0 ? rx0 : rb + 1;
                const int xb = seg == 0 ? (split ? ra - 1 : rx1) : rx1;
                if (xa > xb) continue;
                const long long x0 = xa - tab.xc;
                if constexpr (P == 3) {
                    D3 = 6 * gm[3];
                    D2 = 2 * gm[2] + 6 * gm[3] * (x0 + 1);
                    D1 = gm[1] + gm[2] * (2 * x0 + 1) + gm[3] * (3 * x0 * x0 + 3 * x0 + 1);
                    D0 = ((gm[3] * x0 + gm[2]) * x0 + gm[1]) * x0 + gm[0];
                } else {
                    D2 = 2 * gm[2];
                    D1 = gm[1] + gm[2] * (2 * x0 + 1);
                    D0 = (gm[2] * x0 + gm[1]) * x0 + gm[0];
                }
                Xf = (float)x0;
                h = 1.f;
                np = xb - xa + 1;
                dn = 0;
                Yf = (float)Y;
                y32 = D == 2 ? tab.ty(cy) : 0.f;
                const int ex = max(abs(xa), abs(xb));
                dmax = max(dmax, ex * ex + cy * cy);
            } else {
                if (!split) break;
                const int sy = D == 2 ? (seg == 2 ? -1 : 1) : 0;
                const int n4 = 4 * Y + sy;
                long long B[P + 1];
                fix_child_row<D, FLUON>(beta, n4, B);
                // N(m) = 64 w at the quarter offsets m = m0, m0 + 2, ... (exact integers)
                const int m0 = 4 * (ra - tab.xc) - 1;
                const long long N0 = fix_child_w<P>(B, m0), N1 = fix_child_w<P>(B, m0 + 2),
                                N2 = fix_child_w<P>(B, m0 + 4);
                D0 = N0;
                D1 = N1 - N0;
                D2 = N2 - 2 * N1 + N0;
                if constexpr (P == 3) D3 = fix_child_w<P>(B, m0 + 6) - 3 * N2 + 3 * N1 - N0;
                Xf = 0.25f * (float)m0;
                h = 0.5f;
                np = 2 * (rb - ra + 1);
                dn = -D;
                Yf = 0.25f * (float)n4;
                y32 = D == 2 ? tab.ty(cy, 0.25f * (float)sy) : 0.f;
            }
            DFAcc S[P + 1];
            float SJ[PJ + 1];
#pragma unroll
            for (int a = 0; a <= P; a++) S[a].zero();
#pragma unroll
            for (int a = 0; a <= PJ; a++) SJ[a] = 0.f;
            const float cyf = (float)tab.yc + Yf;  // c_y of the segment's points
#pragma unroll 1
            for (int k = 0; k < np; k++) {
                float fh, fl;
                exp2_fix(D0, etab, dn, fh, fl);
                accumulate(S, SJ, Xf, fh, fl);
                if constexpr (MODE == DF_STREAM) stream_point((float)tab.xc + Xf, cyf, fh, fl, dn != 0);
                D0 += D1;
                D1 += D2;
                if constexpr (P == 3) D2 += D3;
                Xf += h;
            }
            q += (unsigned long long)np;
            fold(S, SJ, Yf, y32);
        }
    }
    npts += (unsigned int)q;
    if constexpr (MODE == DF_STREAM) {
        if (FLUON && ds.mh > 0.f) {  // counted once per cell: the fluon deposit, not a take-back
            if (q > ls.q_max) ls.q_max = q;
            ls.points += q;
            ls.disp_max2 = fmax(ls.disp_max2, (double)dmax);
        }
        ls.walls += walls;
    }
    // lattice moments about floor(u) -> thermal moments about u -> residual
    double Ld[NB];
#pragma unroll
    for (int k = 0; k < NB; k++) Ld[k] = L[k].value();
    double sp[P + 1];
    sp[0] = 1.0;
#pragma unroll
    for (int k = 1; k <= P; k++) sp[k] = sp[k - 1] * inv_sig;
    double Mth[NB];
    if constexpr (D == 1) {
        origin_shift<P>(Ld, fx, Mth);
#pragma unroll
        for (int a = 0; a <= P; a++) Mth[a] *= sp[a];
    } else {
        // along X for every power of Y, then along Y for every power of X
#pragma unroll
        for (int b = 0; b <= P; b++) {
            double col[P + 1], out[P + 1];
#pragma unroll
            for (int a = 0; a <= P; a++) col[a] = a + b <= P ? Ld[Q::ix(a, b)] : 0.0;
            origin_shift<P>(col, fx, out);
#pragma unroll
            for (int a = 0; a + b <= P; a++) Mth[Q::ix(a, b)] = out[a];
        }
#pragma unroll
        for (int a = 0; a <= P; a++) {
            double col[P + 1], out[P + 1];
#pragma unroll
            for (int b = 0; b <= P; b++) col[b] = a + b <= P ? Mth[Q::ix(a, b)] : 0.0;
            origin_shift<P>(col, fy, out);
#pragma unroll
            for (int b = 0; a + b <= P; b++) Mth[Q::ix(a, b)] = out[b] * sp[a + b];
        }
    }
    double rmax = 0.0;
    bool finite = true;
#pragma unroll
    for (int j = 0; j < Q::N; j++) {
        const double rj = Mth[Q::ix(bx<D, FLUON>(j), by<D, FLUON>(j))] - con[j];
        r_out[j] = rj;
        finite = finite && isfinite(rj);
        rmax = fmax(rmax, fabs(rj));
    }
    rmax_out = finite ? rmax : INFINITY;
    if constexpr (MODE == DF_CORR) {
#pragma unroll
        for (int k = 0; k < Q::NJ; k++) MJ_out[k] = MJ[k];
    }
    return true;
}

// Newton update from a double-float residual and the FP32 Jacobian of the same pass
// (Eq. IID11 with A in FP32): lam += A^-1 r.  False on a non-positive pivot.
template <int D, bool FLUON>
__device__ __forceinline__ bool df_update(const float* MJ, const double* r, double* lam) {
    using Q = DFPop<D, FLUON>;
    constexpr int N = Q::N, PJ = Q::PJ;
    float A[N * (N + 1) / 2], x[N];
#pragma unroll
    for (int i = 0; i < N; i++) {
        x[i] = (float)r[i];
#pragma unroll
        for (int j = 0; j <= i; j++)
            A[tri(i, j)] = MJ[D == 1 ? bx<D, FLUON>(i) + bx<D, FLUON>(j)
                                     : tix(bx<D, FLUON>(i) + bx<D, FLUON>(j), by<D, FLUON>(i) + by<D, FLUON>(j), PJ)];
    }
    if (!ldlt_solve<float, N>(A, x)) return false;
#pragma unroll
    for (int j = 0; j < N; j++) lam[j] += (double)x[j];
    return true;
}

}  // namespace lbm
