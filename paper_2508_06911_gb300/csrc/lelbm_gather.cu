// Deterministic moment streaming (Eq. IIE3) for the FP64 2D path: a gather instead of a
// scatter.  The cell kernel leaves every cell's converged multipliers (after the polishing
// update, or of the fallback it took) in Model::det_lam; this kernel then computes, for
// each target cell, the sum of T_N(c_i) rho f'_i and T_N(c_i) rho K RT g'_i over every source
// cell whose stencil point c_i lands on the target -- a level-0 point exactly at x + c_i, a
// refined child by its cloud-in-cell share -- in a fixed order of sources and points.  No
// atomics: the result does not depend on the order in which blocks run, so two runs give
// the same bits.
//
// A block owns a 32 x 8 tile of targets.  Source cells within the reach H of the tile (H =
// the largest |u_a| + R_ac + 1/2 of the step, plus one cell for cloud-in-cell shares) are
// staged through shared memory two rows by 64 columns at a time: their macroscopic variables
// (Eq. IIB6), stencil parameters (Eq. IIC6, IIC9) and multipliers; each thread then walks
// the staged sources inside its own window.  Periodic axes wrap the source coordinate, so a
// source that reaches a target through several images contributes once per image, as in
// the scatter.
#include <cuda_runtime.h>

#include <cstdint>

#include "lelbm_device.cuh"
#include "lelbm_internal.h"

namespace lbm {

constexpr int kGTX = 32, kGTY = 8;  // target tile
constexpr int kGRB = 2, kGCW = 64;  // staged chunk: source rows x columns

struct GSrc {
    double ux, uy, inv_sig, rr2, mf, mg;  // mf = rho, mg = rho K RT (Eq. IIE3)
    double lf[10], lg[6];
    int R, Nr, ok;
};

// Adds the moment fractions of one population point c (lattice frame, relative to its
// source), volume dC and cloud-in-cell weight w, to acc (Eq. IIE3).
__device__ __forceinline__ void gather_point(const GSrc& s, bool has_g, double cx, double cy, double dC, double w,
                                             double* acc) {
    const double t[2] = {(cx - s.ux) * s.inv_sig, (cy - s.uy) * s.inv_sig};
    double T[10];
    Basis<2, true>::eval(t, T);
    double ef = 1.0;
#pragma unroll
    for (int j = 0; j < 10; j++) ef += s.lf[j] * T[j];
    const double mf = w * (s.mf * (dC * exp(-ef)));
    double mg = 0.0;
    if (has_g) {
        double eg = 1.0;
#pragma unroll
        for (int j = 0; j < 6; j++) eg += s.lg[j] * T[j];
        mg = w * (s.mg * (dC * exp(-eg)));
    }
    const double csq = cx * cx + cy * cy;
    acc[0] += mf;
    acc[1] += cx * mf;
    acc[2] += cy * mf;
    acc[3] += cx * cx * mf;
    acc[4] += cx * cy * mf;
    acc[5] += cy * cy * mf;
    acc[6] += csq * cx * mf;
    acc[7] += csq * cy * mf;
    acc[8] += mg;
    acc[9] += cx * mg;
    acc[10] += cy * mg;
}

__global__ void __launch_bounds__(kGTX * kGTY) gather2d_kernel(const __grid_constant__ Model m,
                                                               const __grid_constant__ Geometry g,
                                                               const double* __restrict__ Min, double* __restrict__ Mout,
                                                               DevStats* stats) {
    __shared__ GSrc src[kGRB][kGCW];
    const int H = *m.det_halo;
    const bool has_g = m.K > 0.0;
    const int lx = threadIdx.x % kGTX, ly = threadIdx.x / kGTX;
    const int tx0 = blockIdx.x * kGTX, ty0 = blockIdx.y * kGTY;
    const int tx = tx0 + lx, ty = ty0 + ly;
    // interior targets receive; pads and cells off the array do not (Sec. III)
    const int px = g.periodic[0] ? 0 : g.pad, py = g.periodic[1] ? 0 : g.pad;
    const bool recv = tx >= px && tx < px + g.nx && ty >= py && ty < py + g.ny;
    double acc[11];
#pragma unroll
    for (int k = 0; k < 11; k++) acc[k] = 0.0;
    unsigned long long n_dep = 0;
    double rad2[5];
#pragma unroll
    for (int L = 0; L < 5; L++) {
        const double rad = m.refine_rad * ldexp(1.0, -L);
        rad2[L] = rad * rad;  // as Stencil::init
    }
    const int sx_lo = tx0 - H, sx_hi = tx0 + kGTX - 1 + H;
    const int sy_lo = ty0 - H, sy_hi = ty0 + kGTY - 1 + H;
    for (int sy0 = sy_lo; sy0 <= sy_hi; sy0 += kGRB) {
        for (int sx0 = sx_lo; sx0 <= sx_hi; sx0 += kGCW) {
            __syncthreads();
            for (int e = threadIdx.x; e < kGRB * kGCW; e += blockDim.x) {
                const int r = e / kGCW, k = e - r * kGCW;
                int sx = sx0 + k, sy = sy0 + r;
                GSrc& s = src[r][k];
                s.ok = 0;
                if (sx > sx_hi || sy > sy_hi) continue;
                if (g.periodic[0]) {
                    sx %= g.NX;
                    if (sx < 0) sx += g.NX;
                } else if (sx < 0 || sx >= g.NX) {
                    continue;
                }
                if (g.periodic[1]) {
                    sy %= g.NY;
                    if (sy < 0) sy += g.NY;
                } else if (sy < 0 || sy >= g.NY) {
                    continue;
                }
                const long long cell = (long long)sy * g.NX + sx;
                double M[11];
#pragma unroll
                for (int i = 0; i < 11; i++) M[i] = Min[i * g.ncell + cell];
                CellState<2> c;
                double RT, usq;
                if (!cell_macros<2>(M, m.K, c.rho, c.u, RT, usq)) continue;
                c.RT = RT;
                c.sig = sqrt(RT);
                c.inv_sig = 1.0 / c.sig;
                Stencil<2> st;
                st.init(c, m);
                s.ux = c.u[0];
                s.uy = c.u[1];
                s.inv_sig = c.inv_sig;
                s.rr2 = st.rr2;
                s.mf = c.rho;
                s.mg = c.rho * m.K * c.RT;
                s.R = st.R;
                s.Nr = st.Nr;
#pragma unroll
                for (int j = 0; j < 10; j++) s.lf[j] = m.det_lam[(long long)j * g.ncell + cell];
#pragma unroll
                for (int j = 0; j < 6; j++) s.lg[j] = m.det_lam[(long long)(10 + j) * g.ncell + cell];
                s.ok = 1;
            }
            __syncthreads();
            if (!recv) continue;
            // the staged sources inside this target's window |t - s| <= H, in order
            for (int r = 0; r < kGRB; r++) {
                const int dy = ty - (sy0 + r);
                if (dy < -H || dy > H || sy0 + r > sy_hi) continue;
                const int k0 = max(0, tx - H - sx0), k1 = min(kGCW - 1, tx + H - sx0);
                for (int k = k0; k <= k1; k++) {
                    const GSrc& s = src[r][k];
                    if (!s.ok) continue;
                    const int dx = tx - (sx0 + k);  // the point c = (dx, dy) of the source
                    const double ex = (double)dx - s.ux, ey = (double)dy - s.uy;
                    const double reach = (double)s.R + 2.5;
                    if (ex * ex + ey * ey > reach * reach) continue;
                    Stencil<2> st;
                    st.u[0] = s.ux;
                    st.u[1] = s.uy;
                    st.rr2 = s.rr2;
                    st.R = s.R;
                    st.Nr = s.Nr;
#pragma unroll
                    for (int L = 0; L < 5; L++) st.rad2[L] = rad2[L];
                    const double cd[2] = {(double)dx, (double)dy};
                    const double d2 = st.dist2(cd);
                    // a level-0 point that is not split lands exactly on the target
                    if (d2 <= st.rr2 && (st.Nr == 0 || d2 > st.rad2[1])) {
                        gather_point(s, has_g, cd[0], cd[1], 1.0, 1.0, acc);
                        n_dep++;
                    }
                    // children of split points (within refine_rad / 2 of u) whose
                    // cloud-in-cell share reaches the target
                    if (st.Nr > 0 && fabs(ex) < 3.0 && fabs(ey) < 3.0) {
                        const double r1 = sqrt(st.rad2[1]);
                        const int ax = (int)floor(s.ux - r1) - 1, bx = (int)ceil(s.ux + r1) + 1;
                        const int ay = (int)floor(s.uy - r1) - 1, by = (int)ceil(s.uy + r1) + 1;
                        for (int py0 = ay; py0 <= by; py0++) {
                            if (abs(py0 - dy) > 1) continue;
                            for (int px0 = ax; px0 <= bx; px0++) {
                                if (abs(px0 - dx) > 1) continue;
                                const double c0[2] = {(double)px0, (double)py0};
                                const double p2 = st.dist2(c0);
                                if (!(p2 <= st.rr2 && p2 <= st.rad2[1])) continue;
                                auto leaf = [&](const double* cl, double dC) {
                                    const double wx = 1.0 - fabs(cl[0] - cd[0]), wy = 1.0 - fabs(cl[1] - cd[1]);
                                    if (wx > 0.0 && wy > 0.0) {
                                        gather_point(s, has_g, cl[0], cl[1], dC, wx * wy, acc);
                                        n_dep++;
                                    }
                                };
                                st.visit0(c0, leaf);
                            }
                        }
                    }
                }
            }
        }
    }
    if (tx < g.NX && ty < g.NY) {
        const long long t = (long long)ty * g.NX + tx;
#pragma unroll
        for (int k = 0; k < 11; k++) Mout[k * g.ncell + t] = recv ? acc[k] : 0.0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_dep += __shfl_xor_sync(0xffffffffu, n_dep, o);
    if ((threadIdx.x & 31) == 0 && n_dep) atomicAdd(&stats->points_ms, n_dep);
}

void launch_gather2d(const Model& m, const Geometry& g, const double* Min, double* Mout, DevStats* st,
                     cudaStream_t s) {
    const dim3 grid((g.NX + kGTX - 1) / kGTX, (g.NY + kGTY - 1) / kGTY);
    gather2d_kernel<<<grid, kGTX * kGTY, 0, s>>>(m, g, Min, Mout, st);
}

}  // namespace lbm
