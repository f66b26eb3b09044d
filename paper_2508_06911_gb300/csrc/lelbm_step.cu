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

#include "lelbm_device.cuh"
#include "lelbm_internal.h"
#include "lelbm_mlp.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// The fused single-cell kernel.
// ---------------------------------------------------------------------------
struct LocalStats {
    unsigned long long q_max;
    double disp_max2;
    unsigned long long points;
};

// Landing cell of an integer displacement (dx, dy) from the emitting cell, or -1
// when the population leaves the interior of its instance (Sec. III: discarded).
template <int D>
__device__ __forceinline__ long long land(const Geometry& g, long long cell, long long lo, int n, int ix, int iy,
                                          int dx, int dy) {
    if constexpr (D == 1) {
        long long x = cell + dx;
        if (g.periodic[0]) {
            long long r = (x - lo) % n;
            if (r < 0) r += n;
            return lo + r;
        }
        return (x < lo || x >= lo + n) ? -1 : x;
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

// Moment streaming, Eq. (IIE3): T_N(c_i) rho f'_i and T_N(c_i) rho K RT g'_i added at
// x + c_i.  Level-0 points land on one cell; refined points are shared between the
// cells they overlap (cloud-in-cell).
//
// With CHECK, the same pass also accumulates the moments of degree <= 3 (fluons)
// and <= 2 (phonons) of the deposited populations and returns whether their
// residual against conF / conG is within the tolerance (the FP64 judge of the
// mixed path).  sign = -1 removes a previous deposit of the same populations.
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
    double dmax2 = 0.0;
    auto deposit = [&](long long tgt, const double* cp, double mf, double mg) {
        if (tgt < 0 || type[tgt] != CELL_FLUID) return;
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
    if (q > ls.q_max) ls.q_max = q;
    ls.points += q;
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
    unsigned long long cells, feq, fmx, q, dmax, pf, pg, pm, p32, redo, retry;
};

// Per-thread tallies.
struct ThreadCounters {
    unsigned long long cells, pf, pg, p32, redo, retry;
    LocalStats ls;
};

__device__ __forceinline__ void counters_init(BlockCounters& bc) {
    for (int i = threadIdx.x; i < 64; i += blockDim.x) bc.hist[i] = 0;
    if (threadIdx.x == 0)
        bc.cells = bc.feq = bc.fmx = bc.q = bc.dmax = bc.pf = bc.pg = bc.pm = bc.p32 = bc.redo = bc.retry = 0;
}

// Adds the thread tallies to the block counters, then (after a barrier) the block
// counters to the device counters.  Every thread of the block must call it.
__device__ __forceinline__ void counters_flush(BlockCounters& bc, const ThreadCounters& tc, DevStats* stats) {
    atomicAdd(&bc.cells, tc.cells);
    atomicAdd(&bc.p32, tc.p32);
    atomicAdd(&bc.redo, tc.redo);
    atomicAdd(&bc.retry, tc.retry);
    atomicAdd(&bc.pf, tc.pf);
    atomicAdd(&bc.pg, tc.pg);
    atomicAdd(&bc.pm, tc.ls.points);
    atomicMax(&bc.q, tc.ls.q_max);
    atomicMax(&bc.dmax, (unsigned long long)__double_as_longlong(sqrt(tc.ls.disp_max2)));
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
        if (bc.feq) atomicAdd(&stats->fallback_eq, bc.feq);
        if (bc.fmx) atomicAdd(&stats->fallback_mx, bc.fmx);
        atomicMax(&stats->q_max, bc.q);
        atomicMax(&stats->disp_max_bits, bc.dmax);
    }
}

// The single-cell operation of Fig. 5 in two halves around the (warp-wide) warm-start
// network: prepare_cell loads the moments, runs the collision module and sets up the
// stencil; finish_cell runs EPR (with the fallbacks) and moment streaming into Mout.
template <int D>
__device__ __forceinline__ bool prepare_cell(const Model& m, const Geometry& g, const double* __restrict__ Min,
                                             DevStats* stats, long long cell, BlockCounters& bc, CellState<D>& c,
                                             Stencil<D>& st) {
    constexpr int NM = Dim<D>::NM;
    double M[NM];
#pragma unroll
    for (int i = 0; i < NM; i++) M[i] = Min[i * g.ncell + cell];
    collide<D>(M, m, c);
    if (!c.ok) {  // non-physical cell: nothing can be reconstructed
        atomicAdd(&bc.fmx, 1ull);
        atomicMin(&stats->first_fail, (unsigned long long)cell);
        return false;
    }
    st.init(c, m);
    return true;
}

// dl: the learned correction of the Maxwellian start (fluons then phonons), or null.
template <int D, bool MIXED>
__device__ __forceinline__ void finish_cell(const Model& m, const Geometry& g, const uint8_t* type, double* Mout,
                                            DevStats* stats, long long cell, BlockCounters& bc, ThreadCounters& tc,
                                            double* conF, double* conG, const CellState<D>& c, const Stencil<D>& st,
                                            const float* dl) {
    constexpr int NF = Dim<D>::NF, NG = Dim<D>::NG;
    tc.cells++;
    const bool has_g = m.K > 0.0;
    double lf[NF], lg[NG];
    maxwell_start_fg<D, NF, NG>(c.RT, lf, lg);
    bool learned = false;
    if (dl) {
        bool ok = true;
#pragma unroll
        for (int k = 0; k < MlpDims<D>::NOUT; k++) ok = ok && isfinite(dl[k]);
        if (ok) {
#pragma unroll
            for (int j = 0; j < NF; j++) lf[j] += (double)dl[j];
            if (has_g) {
#pragma unroll
                for (int j = 0; j < NG; j++) lg[j] += (double)dl[NF + j];
            }
            learned = true;
        }
    }
#pragma unroll
    for (int j = 0; j < NF; j++) conF[j] = c.cf[j];
#pragma unroll
    for (int j = 0; j < NG; j++) conG[j] = c.cg[j];
    int sf, sg;
    if constexpr (MIXED) {
        if (solve_fg_mixed<D>(c, st, conF, conG, has_g, lf, lg, m, sf, sg, tc.pf, tc.pg, tc.p32)) {
            // stream and judge in one FP64 pass; on a miss, take the deposit back and
            // finish the solve in FP64 from the current multipliers
            if (scatter_cell<D, true>(m, g, type, Mout, cell, c, st, lf, lg, tc.ls, 1.0, conF, conG)) {
                atomicAdd(&bc.hist[1], has_g ? 2ull : 1ull);  // one FP64 update per population
                return;
            }
            scatter_cell<D, false>(m, g, type, Mout, cell, c, st, lf, lg, tc.ls, -1.0);
            tc.redo++;
        } else {
            if (learned) tc.retry++;
            maxwell_start_fg<D, NF, NG>(c.RT, lf, lg);
            learned = false;
        }
    }
    solve_fg<D>(c, st, conF, conG, has_g, lf, lg, m, sf, sg, tc.pf, tc.pg);
    if ((sf < 0 || sg < 0) && learned) {  // the plain EPR is the fallback of the learned start
        tc.retry++;
        maxwell_start_fg<D, NF, NG>(c.RT, lf, lg);
        solve_fg<D>(c, st, conF, conG, has_g, lf, lg, m, sf, sg, tc.pf, tc.pg);
    }
    if (sf >= 0 && sg >= 0) {
        atomicAdd(&bc.hist[sf < 63 ? sf : 63], 1ull);
        if (has_g) atomicAdd(&bc.hist[sg < 63 ? sg : 63], 1ull);
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
        solve_fg<D>(c, st, conF, conG, has_g, lf, lg, m, sf, sg, tc.pf, tc.pg);
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
    scatter_cell<D, false>(m, g, type, Mout, cell, c, st, lf, lg, tc.ls);
}

// One time step of the whole padded grid: warps claim chunks of 32 consecutive cells
// from a global counter (the cost of a cell varies with its temperature, q ~
// (n sqrt RT)^D, so a static split leaves SMs idle at the end).
template <int D, bool MIXED>
__global__ void __launch_bounds__(128) cell_update_kernel(Model m, Geometry g, const uint8_t* __restrict__ type,
                                                          const double* __restrict__ Min, double* Mout,
                                                          DevStats* stats, unsigned long long* work) {
    constexpr int NF = Dim<D>::NF, NG = Dim<D>::NG;
    __shared__ BlockCounters bc;
    __shared__ double s_con[128][NF + NG];  // constraints of each thread's cell (out of registers)
    extern __shared__ __align__(16) unsigned char s_mlp[];  // warm-start network (when set)
    double* conF = s_con[threadIdx.x];
    double* conG = conF + NF;
    counters_init(bc);
    const bool mlp = m.mlp_w != nullptr;
    if (mlp) mlp_stage_mma<D>(s_mlp, m.mlp_w, m.mlp_nrm);
    __syncthreads();
    ThreadCounters tc{0, 0, 0, 0, 0, 0, {0, 0.0, 0}};
    const int lane = threadIdx.x & 31;
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
        if (active) ok = prepare_cell<D>(m, g, Min, stats, cell, bc, c, st);
        float dl[MlpDims<D>::NOUT];
        if (mlp) {  // warp-uniform: every lane takes part in the tensor-core inference
            float xin[MlpDims<D>::NIN];
            if (ok) mlp_features<D>(c, st, xin);
            warp_mlp<D>(s_mlp, xin, ok, dl);
        }
        if (ok) finish_cell<D, MIXED>(m, g, type, Mout, stats, cell, bc, tc, conF, conG, c, st, mlp ? dl : nullptr);
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
template <bool MIXED>
__global__ void __launch_bounds__(128) batch_persistent_kernel(Model m, Geometry g, double in0, double in1,
                                                               double in3, int bc_left_inflow, int bc_right_inflow,
                                                               const uint8_t* __restrict__ type, double* A, double* B,
                                                               DevStats* stats, unsigned long long* work,
                                                               const int* order, const long long* inst_first,
                                                               const int* inst_pad, int* steps_left, int nsteps) {
    constexpr int D = 1, NM = Dim<1>::NM, NF = Dim<1>::NF, NG = Dim<1>::NG;
    __shared__ BlockCounters bc;
    __shared__ double s_con[128][NF + NG];
    __shared__ unsigned int s_next;
    __shared__ int s_inst;
    extern __shared__ __align__(16) unsigned char s_mlp[];  // warm-start network (when set)
    double* conF = s_con[threadIdx.x];
    double* conG = conF + NF;
    counters_init(bc);
    const bool mlp = m.mlp_w != nullptr;
    if (mlp) mlp_stage_mma<1>(s_mlp, m.mlp_w, m.mlp_nrm);
    ThreadCounters tc{0, 0, 0, 0, 0, 0, {0, 0.0, 0}};
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
            for (;;) {
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
                if (active) ok = prepare_cell<D>(m, g, Min, stats, cell, bc, c, st);
                float dl[MlpDims<D>::NOUT];
                if (mlp) {
                    float xin[MlpDims<D>::NIN];
                    if (ok) mlp_features<D>(c, st, xin);
                    warp_mlp<D>(s_mlp, xin, ok, dl);
                }
                if (ok)
                    finish_cell<D, MIXED>(m, g, type, Mout, stats, cell, bc, tc, conF, conG, c, st, mlp ? dl : nullptr);
            }
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

void launch_batch_persistent(const Model& m, const Geometry& g, const double inlet[4], int bc_left_inflow,
                             int bc_right_inflow, const uint8_t* type, double* A, double* B, DevStats* st,
                             unsigned long long* work, const int* order, const long long* inst_first,
                             const int* inst_pad, int* steps_left, int nsteps, int blocks, int threads, bool mixed,
                             cudaStream_t s) {
    const size_t sm = m.mlp_w ? MlpMma<1>::BYTES : 0;
    auto go = [&](auto kern) {
        if (sm) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kern<<<blocks, threads, sm, s>>>(m, g, inlet[0], inlet[1], inlet[3], bc_left_inflow, bc_right_inflow, type, A,
                                         B, st, work, order, inst_first, inst_pad, steps_left, nsteps);
    };
    if (mixed)
        go(batch_persistent_kernel<true>);
    else
        go(batch_persistent_kernel<false>);
}

int batch_persistent_max_blocks_per_sm(bool mixed, int threads) {
    int per_sm = 0;
    if (mixed)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel<true>, threads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel<false>, threads, 0);
    return per_sm < 1 ? 1 : per_sm;
}

// ---------------------------------------------------------------------------
// Boundary fill, state set-up and macroscopic fields.
// ---------------------------------------------------------------------------
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

int cell_update_blocks(int D, bool mixed, int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int per_sm = 0;
    if (D == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, mixed ? cell_update_kernel<1, true> : cell_update_kernel<1, false>, 128, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, mixed ? cell_update_kernel<2, true> : cell_update_kernel<2, false>, 128, 0);
    if (per_sm < 1) per_sm = 1;
    if (sms < 1) sms = 1;
    return sms * per_sm;
}

void launch_cell_update(const Model& m, const Geometry& g, const uint8_t* type, const double* Min, double* Mout,
                        DevStats* st, unsigned long long* work, int grid_blocks, bool mixed, cudaStream_t s) {
    long long need = (g.ncell + 127) / 128;
    int blocks = (int)(need < grid_blocks ? need : grid_blocks);
    if (blocks < 1) blocks = 1;
    const size_t sm = m.mlp_w ? (g.D == 1 ? MlpMma<1>::BYTES : MlpMma<2>::BYTES) : 0;
    auto go = [&](auto kern) {
        if (sm) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        kern<<<blocks, 128, sm, s>>>(m, g, type, Min, Mout, st, work);
    };
    if (g.D == 1) {
        if (mixed)
            go(cell_update_kernel<1, true>);
        else
            go(cell_update_kernel<1, false>);
    } else {
        if (mixed)
            go(cell_update_kernel<2, true>);
        else
            go(cell_update_kernel<2, false>);
    }
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
