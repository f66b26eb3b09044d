// Learned warm start of the EPR Newton (the Maxwellian start of Eq. IID13 plus a
// correction predicted by a small MLP).  Shared by the step kernels (inference,
// pair recording) and the training kernels.
//
// Features of a cell (thermal units, t = (c - u)/sqrt(RT)):
//   1D: c_xx - 1, c_xx|x, g_0 - 1, g_x, frac(u)/sqrt(RT), 1/sqrt(RT), R_ac/sqrt(RT), N_r     (8)
//   2D: c_xx - 1, c_xy, c_yy - 1, c_xx|x, c_yy|x, c_xx|y, c_yy|y, g_0 - 1, g_x, g_y,
//       frac(u_x)/sqrt(RT), frac(u_y)/sqrt(RT), 1/sqrt(RT), R_ac/sqrt(RT), N_r                (15)
// (c_* the normalised post-collision fluon constraints, g_* the phonon ones; the
// stencil terms matter because the multipliers of a discrete velocity set depend
// on where the lattice sits relative to u and on its resolution.)
// Targets: converged multipliers minus the Maxwellian start, fluons then phonons
// (1D 4 + 3, 2D 10 + 6).
//
// Network: in -> 64 -> 64 -> out, SiLU, BF16 weights, FP32 accumulation, inputs and
// outputs standardised.  Parameter layout (FP32 master, BF16 copy of the weights):
//   W1[H][NIN] b1[H] W2[H][H] b2[H] W3[NOUT][H] b3[NOUT] | xm[NIN] xs[NIN] ym[NOUT] ys[NOUT]
#pragma once

#include <cuda_bf16.h>

#include "lelbm_device.cuh"

namespace lbm {

template <int D>
struct MlpDims;
template <>
struct MlpDims<1> {
    static constexpr int NIN = 8, NOUT = 7, H = 64;
};
template <>
struct MlpDims<2> {
    static constexpr int NIN = 15, NOUT = 16, H = 64;
};

template <int D>
struct MlpLayout {
    using Md = MlpDims<D>;
    static constexpr int W1 = 0;
    static constexpr int B1 = W1 + Md::H * Md::NIN;
    static constexpr int W2 = B1 + Md::H;
    static constexpr int B2 = W2 + Md::H * Md::H;
    static constexpr int W3 = B2 + Md::H;
    static constexpr int B3 = W3 + Md::NOUT * Md::H;
    static constexpr int NW = B3 + Md::NOUT;  // trained parameters
    static constexpr int XM = NW;
    static constexpr int XS = XM + Md::NIN;
    static constexpr int YM = XS + Md::NIN;
    static constexpr int YS = YM + Md::NOUT;
    static constexpr int NTOT = YS + Md::NOUT;  // with the normalisation
};

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

template <int D>
__device__ __forceinline__ void mlp_features(const CellState<D>& c, const Stencil<D>& st, float* x) {
    if constexpr (D == 1) {
        x[0] = (float)(c.cf[2] - 1.0);
        x[1] = (float)c.cf[3];
        x[2] = (float)(c.cg[0] - 1.0);
        x[3] = (float)c.cg[1];
        x[4] = (float)((c.u[0] - round(c.u[0])) * c.inv_sig);
        x[5] = (float)c.inv_sig;
        x[6] = (float)(st.R * c.inv_sig);
        x[7] = (float)st.Nr;
    } else {
        x[0] = (float)(c.cf[3] - 1.0);
        x[1] = (float)c.cf[4];
        x[2] = (float)(c.cf[5] - 1.0);
        x[3] = (float)c.cf[6];
        x[4] = (float)c.cf[7];
        x[5] = (float)c.cf[8];
        x[6] = (float)c.cf[9];
        x[7] = (float)(c.cg[0] - 1.0);
        x[8] = (float)c.cg[1];
        x[9] = (float)c.cg[2];
        x[10] = (float)((c.u[0] - round(c.u[0])) * c.inv_sig);
        x[11] = (float)((c.u[1] - round(c.u[1])) * c.inv_sig);
        x[12] = (float)c.inv_sig;
        x[13] = (float)(st.R * c.inv_sig);
        x[14] = (float)st.Nr;
    }
}

// Forward pass with BF16 weights W (layout above) and FP32 normalisation nrm
// (xm, xs, ym, ys): x raw features -> y raw targets.
template <int D>
__device__ __forceinline__ void mlp_forward(const __nv_bfloat16* W, const float* nrm, const float* x, float* y) {
    using Md = MlpDims<D>;
    using Ly = MlpLayout<D>;
    float xs[Md::NIN];
#pragma unroll
    for (int m = 0; m < Md::NIN; m++) xs[m] = (x[m] - nrm[m]) / nrm[Md::NIN + m];
    float h1[Md::H];
#pragma unroll
    for (int j = 0; j < Md::H; j++) {
        float z = __bfloat162float(W[Ly::B1 + j]);
#pragma unroll
        for (int m = 0; m < Md::NIN; m++) z = fmaf(__bfloat162float(W[Ly::W1 + j * Md::NIN + m]), xs[m], z);
        h1[j] = silu(z);
    }
    float out[Md::NOUT];
#pragma unroll
    for (int k = 0; k < Md::NOUT; k++) out[k] = __bfloat162float(W[Ly::B3 + k]);
    for (int i = 0; i < Md::H; i++) {
        float z = __bfloat162float(W[Ly::B2 + i]);
#pragma unroll
        for (int j = 0; j < Md::H; j++) z = fmaf(__bfloat162float(W[Ly::W2 + i * Md::H + j]), h1[j], z);
        const float h2 = silu(z);
#pragma unroll
        for (int k = 0; k < Md::NOUT; k++) out[k] = fmaf(__bfloat162float(W[Ly::W3 + k * Md::H + i]), h2, out[k]);
    }
#pragma unroll
    for (int k = 0; k < Md::NOUT; k++) y[k] = out[k] * nrm[2 * Md::NIN + Md::NOUT + k] + nrm[2 * Md::NIN + k];
}

}  // namespace lbm
