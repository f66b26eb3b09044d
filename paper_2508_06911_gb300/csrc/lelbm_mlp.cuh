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

template <int D, bool F32 = false>
__device__ __forceinline__ void mlp_features(const CellState<D>& c, const Stencil<D>& st, float* x) {
    // the constraints in FP32: the FP32 path's own (exact), else rounded from FP64
    float cf[Dim<D>::NF], cg[Dim<D>::NG];
#pragma unroll
    for (int j = 0; j < Dim<D>::NF; j++) cf[j] = F32 ? c.cf32[j] : (float)c.cf[j];
#pragma unroll
    for (int j = 0; j < Dim<D>::NG; j++) cg[j] = F32 ? c.cg32[j] : (float)c.cg[j];
    if constexpr (D == 1) {
        x[0] = F32 ? cf[2] - 1.f : (float)(c.cf[2] - 1.0);
        x[1] = cf[3];
        x[2] = F32 ? cg[0] - 1.f : (float)(c.cg[0] - 1.0);
        x[3] = cg[1];
        x[4] = (float)((c.u[0] - round(c.u[0])) * c.inv_sig);
        x[5] = F32 ? c.isig32 : (float)c.inv_sig;
        x[6] = F32 ? (float)st.R * c.isig32 : (float)(st.R * c.inv_sig);
        x[7] = (float)st.Nr;
    } else {
        x[0] = F32 ? cf[3] - 1.f : (float)(c.cf[3] - 1.0);
        x[1] = cf[4];
        x[2] = F32 ? cf[5] - 1.f : (float)(c.cf[5] - 1.0);
        x[3] = cf[6];
        x[4] = cf[7];
        x[5] = cf[8];
        x[6] = cf[9];
        x[7] = F32 ? cg[0] - 1.f : (float)(c.cg[0] - 1.0);
        x[8] = cg[1];
        x[9] = cg[2];
        x[10] = (float)((c.u[0] - round(c.u[0])) * c.inv_sig);
        x[11] = (float)((c.u[1] - round(c.u[1])) * c.inv_sig);
        x[12] = F32 ? c.isig32 : (float)c.inv_sig;
        x[13] = F32 ? (float)st.R * c.isig32 : (float)(st.R * c.inv_sig);
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

// ---------------------------------------------------------------------------
// Inference on the tensor cores.  A warp evaluates the network for its 32 cells at
// once as three small GEMMs (32 x 16 x 64, 32 x 64 x 64, 32 x 64 x NOUT) with
// mma.sync m16n8k16 BF16 -> FP32: 88 MMAs per 32 cells instead of ~5000 FMAs per
// cell.  The weights sit in shared memory in padded rows (stride 24 / 72 BF16) so
// the fragment loads of the 8 row groups hit distinct banks; the hidden activations
// never leave registers.
// ---------------------------------------------------------------------------
template <int D>
struct MlpMma {
    static constexpr int S1 = 24;                  // row stride of W1 (inputs padded to 16)
    static constexpr int S2 = 72;                  // row stride of W2, W3 and of activations
    static constexpr int N3 = D == 1 ? 8 : 16;     // outputs padded to whole n-tiles
    static constexpr int W1 = 0;
    static constexpr int W2 = W1 + 64 * S1;
    static constexpr int W3 = W2 + 64 * S2;
    static constexpr int NWS = W3 + N3 * S2;       // BF16 elements of the staged weights
    static constexpr int WARPS = 4;                // warps per block (128 threads)
    // dynamic shared memory: weights | b1 b2 b3 | normalisation | per-warp X, then O
    // (a warp's inputs X are dead once loaded into its fragments; its outputs O reuse them)
    static constexpr size_t OFF_B = ((size_t)NWS * 2 + 15) & ~(size_t)15;
    static constexpr size_t OFF_N = OFF_B + sizeof(float) * (64 + 64 + 16);
    static constexpr size_t OFF_X = (OFF_N + sizeof(float) * 2 * (MlpDims<D>::NIN + MlpDims<D>::NOUT) + 15) & ~(size_t)15;
    static constexpr size_t WARP_IO = 32 * 16 * sizeof(float);  // >= 32 * S1 BF16
    static_assert(WARP_IO >= 32 * S1 * 2, "per-warp X fits in the O region");
    static constexpr size_t OFF_O = OFF_X;
    static constexpr size_t BYTES = OFF_X + (size_t)WARPS * WARP_IO;
};

// Stage the weights of the FP32-layout BF16 copy (W) and the FP32 normalisation into
// the padded shared-memory layout; every thread of the block must call it.  The two
// hidden layers' weights and biases are staged halved (exact in BF16 and FP32), so
// their products are h = z / 2, the argument of SiLU's tanh form.
template <int D>
__device__ __forceinline__ void mlp_stage_mma(unsigned char* smem, const __nv_bfloat16* W, const float* nrm) {
    using Md = MlpDims<D>;
    using Ly = MlpLayout<D>;
    using Mm = MlpMma<D>;
    __nv_bfloat16* w = reinterpret_cast<__nv_bfloat16*>(smem);
    float* b = reinterpret_cast<float*>(smem + Mm::OFF_B);
    float* nr = reinterpret_cast<float*>(smem + Mm::OFF_N);
    const __nv_bfloat16 z = __float2bfloat16(0.f);
    for (int i = threadIdx.x; i < 64 * Mm::S1; i += blockDim.x) {
        const int n = i / Mm::S1, k = i % Mm::S1;
        w[Mm::W1 + i] = k < Md::NIN ? __hmul(W[Ly::W1 + n * Md::NIN + k], __float2bfloat16(0.5f)) : z;
    }
    for (int i = threadIdx.x; i < 64 * Mm::S2; i += blockDim.x) {
        const int n = i / Mm::S2, k = i % Mm::S2;
        w[Mm::W2 + i] = k < 64 ? __hmul(W[Ly::W2 + n * 64 + k], __float2bfloat16(0.5f)) : z;
    }
    for (int i = threadIdx.x; i < Mm::N3 * Mm::S2; i += blockDim.x) {
        const int n = i / Mm::S2, k = i % Mm::S2;
        w[Mm::W3 + i] = (n < Md::NOUT && k < 64) ? W[Ly::W3 + n * 64 + k] : z;
    }
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        b[i] = 0.5f * __bfloat162float(W[Ly::B1 + i]);
        b[64 + i] = 0.5f * __bfloat162float(W[Ly::B2 + i]);
    }
    for (int i = threadIdx.x; i < 16; i += blockDim.x) b[128 + i] = i < Md::NOUT ? __bfloat162float(W[Ly::B3 + i]) : 0.f;
    for (int i = threadIdx.x; i < 2 * (Md::NIN + Md::NOUT); i += blockDim.x) nr[i] = nrm[i];
}

__device__ __forceinline__ void mma_bf16_16x8x16(float* d, unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                                 unsigned b0, unsigned b1) {
    asm(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned ld_b32(const __nv_bfloat16* p) { return *reinterpret_cast<const unsigned*>(p); }

// Four 8x8 BF16 tiles from shared memory in one instruction: lane L gives the address of
// row L % 8 of tile L / 8 (16-byte aligned); each lane receives, of every tile, the pair
// of row lane / 4 at columns 2 (lane % 4), +1 -- the fragment layout of mma.m16n8k16.
__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3, const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(a));
}

__device__ __forceinline__ void st_pair(__nv_bfloat16* p, float lo, float hi) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __floats2bfloat162_rn(lo, hi);
}

// SiLU on BF16 pairs from h = z / 2 (the staged halves of the weights and biases give h
// directly): z sigmoid(z) = h + h tanh(h), with the packed hardware tanh.  Returns the BF16
// pair (h0 in the low half), ready to be an operand of the next layer.
__device__ __forceinline__ unsigned silu_half_bf16x2(float h0, float h1) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(h0, h1);
    unsigned t;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(*reinterpret_cast<const unsigned*>(&h)));
    const __nv_bfloat162 s = __hfma2(h, *reinterpret_cast<const __nv_bfloat162*>(&t), h);
    return *reinterpret_cast<const unsigned*>(&s);
}

// The same SiLU in FP32, z sigmoid(z) = 2h / (1 + exp(-2h)) (the training kernels' SiLU),
// rounded once to BF16: for the inference kernels off the hot path.
__device__ __forceinline__ unsigned silu_half_f32x2(float h0, float h1) {
    const float s0 = __fdividef(2.f * h0, 1.f + __expf(fminf(-2.f * h0, 80.f)));
    const float s1 = __fdividef(2.f * h1, 1.f + __expf(fminf(-2.f * h1, 80.f)));
    const __nv_bfloat162 s = __floats2bfloat162_rn(s0, s1);
    return *reinterpret_cast<const unsigned*>(&s);
}

// Whole-warp inference: lane i supplies the raw features x of its cell (ignored when
// !valid) and receives the raw prediction y.  All 32 lanes must call it.  EXACT: SiLU in
// FP32 (silu_half_f32x2), else the packed BF16 tanh (silu_half_bf16x2, the hot path).
// The accumulator fragment of an m16n8 tile holds rows (g, g + 8) x columns (2t, 2t+1)
// of lane (g, t) -- exactly the operand fragment of the next layer's k-slice -- so
// the hidden activations stay in registers as BF16 pairs: h[m-tile][k-slice][4].
template <int D, bool EXACT = false>
__device__ __forceinline__ void warp_mlp(unsigned char* smem, const float* x, bool valid, float* y) {
    using Md = MlpDims<D>;
    using Mm = MlpMma<D>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gid = lane >> 2, tig = lane & 3;
    const __nv_bfloat16* w = reinterpret_cast<const __nv_bfloat16*>(smem);
    const float* b = reinterpret_cast<const float*>(smem + Mm::OFF_B);
    const float* nr = reinterpret_cast<const float*>(smem + Mm::OFF_N);
    __nv_bfloat16* X = reinterpret_cast<__nv_bfloat16*>(smem + Mm::OFF_X + warp * Mm::WARP_IO);
    float* O = reinterpret_cast<float*>(smem + Mm::OFF_O + warp * Mm::WARP_IO);  // the same bytes as X
    // standardised inputs, one row per lane, zero padded to 16
#pragma unroll
    for (int m = 0; m < 16; m += 2) {
        const float v0 = (valid && m < Md::NIN) ? __fdividef(x[m] - nr[m], nr[Md::NIN + m]) : 0.f;
        const float v1 = (valid && m + 1 < Md::NIN) ? __fdividef(x[m + 1] - nr[m + 1], nr[Md::NIN + m + 1]) : 0.f;
        st_pair(X + lane * Mm::S1 + m, v0, v1);
    }
    __syncwarp();
    // A fragments: tiles (rows 0-7, k 0-7), (rows 8-15, k 0-7), (rows 0-7, k 8-15), (rows 8-15, k 8-15)
    const int lr = lane & 7, lt = lane >> 3;
    unsigned ax[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
        ldsm_x4(ax[mt][0], ax[mt][1], ax[mt][2], ax[mt][3], X + (mt * 16 + (lt & 1) * 8 + lr) * Mm::S1 + (lt >> 1) * 8);
    __syncwarp();  // every lane has its fragments: X may be overwritten by O
    // layer 1: h1 = silu(X W1^T + b1)
    unsigned h1[2][4][4];
#pragma unroll
    for (int np = 0; np < 8; np += 2) {
        // B fragments of n-tiles np and np + 1: tiles (n, k 0-7), (n, k 8-15) of each
        unsigned bb[2][2];
        ldsm_x4(bb[0][0], bb[0][1], bb[1][0], bb[1][1], w + Mm::W1 + ((np + (lt >> 1)) * 8 + lr) * Mm::S1 + (lt & 1) * 8);
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int nt = np + u;
            const int col = nt * 8 + tig * 2;
            const float c0 = b[col], c1 = b[col + 1];
#pragma unroll
            for (int mt = 0; mt < 2; mt++) {
                float d[4] = {c0, c1, c0, c1};  // the accumulator starts at the (halved) bias
                mma_bf16_16x8x16(d, ax[mt][0], ax[mt][1], ax[mt][2], ax[mt][3], bb[u][0], bb[u][1]);
                h1[mt][nt >> 1][(nt & 1) * 2 + 0] = EXACT ? silu_half_f32x2(d[0], d[1]) : silu_half_bf16x2(d[0], d[1]);
                h1[mt][nt >> 1][(nt & 1) * 2 + 1] = EXACT ? silu_half_f32x2(d[2], d[3]) : silu_half_bf16x2(d[2], d[3]);
            }
        }
    }
    // layer 2: h2 = silu(h1 W2^T + b2)
    unsigned h2[2][4][4];
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const int col = nt * 8 + tig * 2;
        const float c0 = b[64 + col], c1 = b[64 + col + 1];
        float d[2][4] = {{c0, c1, c0, c1}, {c0, c1, c0, c1}};
#pragma unroll
        for (int kp = 0; kp < 4; kp += 2) {
            // B fragments of k-tiles kp and kp + 1: tiles (n, k 0-7), (n, k 8-15) of each
            unsigned bb[2][2];
            ldsm_x4(bb[0][0], bb[0][1], bb[1][0], bb[1][1], w + Mm::W2 + (nt * 8 + lr) * Mm::S2 + kp * 16 + lt * 8);
#pragma unroll
            for (int u = 0; u < 2; u++)
#pragma unroll
                for (int mt = 0; mt < 2; mt++)
                    mma_bf16_16x8x16(d[mt], h1[mt][kp + u][0], h1[mt][kp + u][1], h1[mt][kp + u][2], h1[mt][kp + u][3],
                                     bb[u][0], bb[u][1]);
        }
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            h2[mt][nt >> 1][(nt & 1) * 2 + 0] =
                EXACT ? silu_half_f32x2(d[mt][0], d[mt][1]) : silu_half_bf16x2(d[mt][0], d[mt][1]);
            h2[mt][nt >> 1][(nt & 1) * 2 + 1] =
                EXACT ? silu_half_f32x2(d[mt][2], d[mt][3]) : silu_half_bf16x2(d[mt][2], d[mt][3]);
        }
    }
    // layer 3: y = h2 W3^T + b3, transposed to one row per lane through shared memory
#pragma unroll
    for (int nt = 0; nt < Mm::N3 / 8; nt++) {
        float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
        for (int kp = 0; kp < 4; kp += 2) {
            unsigned bb[2][2];
            ldsm_x4(bb[0][0], bb[0][1], bb[1][0], bb[1][1], w + Mm::W3 + (nt * 8 + lr) * Mm::S2 + kp * 16 + lt * 8);
#pragma unroll
            for (int u = 0; u < 2; u++)
#pragma unroll
                for (int mt = 0; mt < 2; mt++)
                    mma_bf16_16x8x16(d[mt], h2[mt][kp + u][0], h2[mt][kp + u][1], h2[mt][kp + u][2], h2[mt][kp + u][3],
                                     bb[u][0], bb[u][1]);
        }
        const int col = nt * 8 + tig * 2;
#pragma unroll
        for (int mt = 0; mt < 2; mt++) {
            const int row = mt * 16 + gid;
            O[row * 16 + col] = d[mt][0] + b[128 + col];
            O[row * 16 + col + 1] = d[mt][1] + b[128 + col + 1];
            O[(row + 8) * 16 + col] = d[mt][2] + b[128 + col];
            O[(row + 8) * 16 + col + 1] = d[mt][3] + b[128 + col + 1];
        }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < Md::NOUT; k++) y[k] = O[lane * 16 + k] * nr[2 * Md::NIN + Md::NOUT + k] + nr[2 * Md::NIN + k];
    __syncwarp();
}

}  // namespace lbm
