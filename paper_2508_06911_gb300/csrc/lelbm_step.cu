// Host-side launchers of the LELBM time step and the small per-cell kernels
// (boundary fill, state set-up, macroscopic fields) for sm_103a.  The heavy
// kernels live in lelbm_cell.cu (cell update) and lelbm_batch.cu (persistent
// 1D batch), one object per variant.

#include <cstdint>

#include "lelbm_device.cuh"
#include "lelbm_internal.h"
#include "lelbm_mlp.cuh"

namespace lbm {

void launch_batch_persistent(const Model& m, const Geometry& g, const double inlet[4], int bc_left_inflow,
                             int bc_right_inflow, const uint8_t* type, double* A, double* B, DevStats* st,
                             unsigned long long* work, const int* order, const long long* inst_first,
                             const int* inst_pad, int* steps_left, int nsteps, int blocks, int threads, int prec,
                             cudaStream_t s) {
    const size_t sm = m.mlp_w ? MlpMma<1>::BYTES : 0;
    auto go = [&](auto variant) {
        decltype(variant)::launch(m, g, inlet, bc_left_inflow, bc_right_inflow, type, A, B, st, work, order,
                                  inst_first, inst_pad, steps_left, nsteps, blocks, threads, sm, s);
    };
    if (prec == PREC_MIXED)
        go(BatchVariant<PREC_MIXED>{});
    else if (prec == PREC_FP32)
        go(BatchVariant<PREC_FP32>{});
    else
        go(BatchVariant<PREC_FP64>{});
}

int batch_persistent_max_blocks_per_sm(int prec, int threads) {
    const int per_sm = prec == PREC_MIXED  ? BatchVariant<PREC_MIXED>::blocks_per_sm(threads)
                       : prec == PREC_FP32 ? BatchVariant<PREC_FP32>::blocks_per_sm(threads)
                                           : BatchVariant<PREC_FP64>::blocks_per_sm(threads);
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

template <int D>
static int cell_blocks_per_sm(int prec) {
    return prec == PREC_MIXED  ? CellVariant<D, PREC_MIXED>::blocks_per_sm()
           : prec == PREC_FP32 ? CellVariant<D, PREC_FP32>::blocks_per_sm()
                               : CellVariant<D, PREC_FP64>::blocks_per_sm();
}

int cell_update_blocks(int D, int prec, int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    int per_sm = D == 1 ? cell_blocks_per_sm<1>(prec) : cell_blocks_per_sm<2>(prec);
    if (per_sm < 1) per_sm = 1;
    if (sms < 1) sms = 1;
    return sms * per_sm;
}

template <int D>
static void cell_launch(int prec, const Model& m, const Geometry& g, const uint8_t* type, const double* Min,
                        double* Mout, DevStats* st, unsigned long long* work, int blocks, size_t sm, cudaStream_t s) {
    if (prec == PREC_MIXED)
        CellVariant<D, PREC_MIXED>::launch(m, g, type, Min, Mout, st, work, blocks, sm, s);
    else if (prec == PREC_FP32)
        CellVariant<D, PREC_FP32>::launch(m, g, type, Min, Mout, st, work, blocks, sm, s);
    else
        CellVariant<D, PREC_FP64>::launch(m, g, type, Min, Mout, st, work, blocks, sm, s);
}

void launch_cell_update(const Model& m, const Geometry& g, const uint8_t* type, const double* Min, double* Mout,
                        DevStats* st, unsigned long long* work, int grid_blocks, int prec, cudaStream_t s) {
    const int nt = prec == PREC_MIXED ? cell_threads<PREC_MIXED>() : 128;
    long long need = (g.ncell + nt - 1) / nt;
    int blocks = (int)(need < grid_blocks ? need : grid_blocks);
    if (blocks < 1) blocks = 1;
    const size_t sm = 0;  // the learned start runs in mlp_start_kernel, not in the cell update
    if (g.D == 1)
        cell_launch<1>(prec, m, g, type, Min, Mout, st, work, blocks, sm, s);
    else
        cell_launch<2>(prec, m, g, type, Min, Mout, st, work, blocks, sm, s);
}

void launch_eq_state(int D, double K, const uint8_t* type, const double* rho, const double* u, const double* RT,
                     double* M, long long ncell, cudaStream_t s) {
    const int blocks = grid_for(ncell, 256);
    if (D == 1)
        eq_state_kernel<1><<<blocks, 256, 0, s>>>(K, type, rho, u, RT, M, ncell);
    else if (D == 2)
        eq_state_kernel<2><<<blocks, 256, 0, s>>>(K, type, rho, u, RT, M, ncell);
    else
        eq_state_kernel<3><<<blocks, 256, 0, s>>>(K, type, rho, u, RT, M, ncell);
}

void launch_macros(int D, double K, const uint8_t* type, const double* M, double* rho, double* u, double* RT,
                   long long ncell, cudaStream_t s) {
    const int blocks = grid_for(ncell, 256);
    if (D == 1)
        macros_kernel<1><<<blocks, 256, 0, s>>>(K, type, M, rho, u, RT, ncell);
    else if (D == 2)
        macros_kernel<2><<<blocks, 256, 0, s>>>(K, type, M, rho, u, RT, ncell);
    else
        macros_kernel<3><<<blocks, 256, 0, s>>>(K, type, M, rho, u, RT, ncell);
}

// ---------------------------------------------------------------------------
// Learned warm start as its own kernel (the cell-update kernels read its output the way
// they read the stored start).  Each warp takes 32 consecutive cells: the collision module
// in FP32 alone gives the features, and the network (2 x 64 SiLU, BF16 weights staged in shared
// memory, FP32 accumulation, SiLU in FP32) runs on the tensor cores for the warp's 32
// cells at once.
// out[k][cell] (SoA, NOUT rows) receives the predicted correction of Eq. (IID13); a NaN
// in the first row (the others left unwritten) where the cell gets no learned start (solid, non-physical, or -- with a gate -- close
// enough to equilibrium that Eq. (IID13) is the better start).  A warp whose 32 cells all
// take Eq. (IID13) skips the network.
// ---------------------------------------------------------------------------
// Largest departure of the normalised post-collision constraints (thermal units) from
// those of the equilibrium (Eq. IIB16-IIB18 with omega = 1): 1, 0, delta_ab, 0 for the
// fluons and 1, 0, delta_ab for the phonons.
template <int D>
__device__ __forceinline__ float constraint_departure(const CellState<D>& c, bool has_g) {
    float d = 0.f;
#pragma unroll
    for (int k = 0; k < Dim<D>::NF; k++) {
        const bool diag = D == 1 ? k == 2 : (k == 3 || k == 5);  // M_aa / (rho RT)
        d = fmaxf(d, fabsf(c.cf32[k] - ((k == 0 || diag) ? 1.f : 0.f)));
    }
    if (has_g) {
#pragma unroll
        for (int k = 0; k < 1 + D; k++) d = fmaxf(d, fabsf(c.cg32[k] - (k == 0 ? 1.f : 0.f)));
    }
    return d;
}

template <int D>
__global__ void __launch_bounds__(128) mlp_start_kernel(const __grid_constant__ Model m,
                                                        const __grid_constant__ Geometry g,
                                                        const uint8_t* __restrict__ type,
                                                        const double* __restrict__ Min, float* __restrict__ out) {
    constexpr int NM = Dim<D>::NM;
    extern __shared__ __align__(16) unsigned char s_mlp[];
    mlp_stage_mma<D>(s_mlp, m.mlp_w, m.mlp_nrm);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long base = ((long long)blockIdx.x * 4 + warp) * 32; base < g.ncell;
         base += (long long)gridDim.x * 128) {  // warp-uniform
        const long long cell = base + lane;
        const bool active = cell < g.ncell && type[cell] != CELL_SOLID;
        CellState<D> c;
        Stencil<D> st;
        bool ok = false;
        if (active) {
            double M[NM];
#pragma unroll
            for (int i = 0; i < NM; i++) M[i] = Min[i * g.ncell + cell];
            collide32<D, true>(M, m, c);  // features in FP32 only
            ok = c.ok;
            if (ok) st.init32(c, m);
        }
        if (ok && m.mlp_gate > 0.f) ok = constraint_departure<D>(c, m.K > 0.0) >= m.mlp_gate;
        float xin[MlpDims<D>::NIN], dl[MlpDims<D>::NOUT];
#pragma unroll
        for (int k = 0; k < MlpDims<D>::NIN; k++) xin[k] = 0.f;
        if (ok) mlp_features<D, true>(c, st, xin);
        if (__any_sync(0xffffffffu, ok)) warp_mlp<D, true>(s_mlp, xin, ok, dl);  // warp-uniform
        if (cell < g.ncell) {
            if (ok) {
#pragma unroll
                for (int k = 0; k < MlpDims<D>::NOUT; k++) out[(long long)k * g.ncell + cell] = dl[k];
            } else {
                out[cell] = __int_as_float(0x7fc00000);  // NaN in the first row: no learned start
            }
        }
    }
}

void launch_mlp_start(const Model& m, const Geometry& g, const uint8_t* type, const double* Min, float* out,
                      int device, cudaStream_t s) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const long long warps = (g.ncell + 31) / 32;
    long long blocks = (warps + 3) / 4;
    const long long cap = (long long)(sms > 0 ? sms : 1) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (g.D == 1) {
        cudaFuncSetAttribute(mlp_start_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MlpMma<1>::BYTES);
        mlp_start_kernel<1><<<(int)blocks, 128, MlpMma<1>::BYTES, s>>>(m, g, type, Min, out);
    } else {
        cudaFuncSetAttribute(mlp_start_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MlpMma<2>::BYTES);
        mlp_start_kernel<2><<<(int)blocks, 128, MlpMma<2>::BYTES, s>>>(m, g, type, Min, out);
    }
}

// The same tensor-core inference on caller-supplied feature rows X[n][NIN] -> Y[n][NOUT]
// (lelbm_mlp_infer).
template <int D>
__global__ void __launch_bounds__(128) mlp_infer_kernel(const __nv_bfloat16* W, const float* nrm,
                                                        const float* __restrict__ X, long long n,
                                                        float* __restrict__ Y) {
    constexpr int NIN = MlpDims<D>::NIN, NOUT = MlpDims<D>::NOUT;
    extern __shared__ __align__(16) unsigned char s_mlp[];
    mlp_stage_mma<D>(s_mlp, W, nrm);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (long long base = ((long long)blockIdx.x * 4 + warp) * 32; base < n; base += (long long)gridDim.x * 128) {
        const long long row = base + lane;
        const bool valid = row < n;
        float xin[NIN], dl[NOUT];
#pragma unroll
        for (int k = 0; k < NIN; k++) xin[k] = valid ? X[row * NIN + k] : 0.f;
        warp_mlp<D, true>(s_mlp, xin, valid, dl);
        if (valid) {
#pragma unroll
            for (int k = 0; k < NOUT; k++) Y[row * NOUT + k] = dl[k];
        }
    }
}

void launch_mlp_infer(int D, const __nv_bfloat16* W, const float* nrm, const float* X, long long n, float* Y,
                      cudaStream_t s) {
    long long blocks = (n + 127) / 128;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    if (D == 1) {
        cudaFuncSetAttribute(mlp_infer_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MlpMma<1>::BYTES);
        mlp_infer_kernel<1><<<(int)blocks, 128, MlpMma<1>::BYTES, s>>>(W, nrm, X, n, Y);
    } else {
        cudaFuncSetAttribute(mlp_infer_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MlpMma<2>::BYTES);
        mlp_infer_kernel<2><<<(int)blocks, 128, MlpMma<2>::BYTES, s>>>(W, nrm, X, n, Y);
    }
}

// ---------------------------------------------------------------------------
// FMA throughput probe (the denominator of the ALU rooflines): every thread runs eight
// independent FMA chains, so each scheduler always has independent FMAs to issue.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void fma_probe_kernel(T* out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    if (s == (T)-1.2345e30) out[0] = s;  // keeps the chains live; never true
}

// Best of three timed launches, in FLOP/s; < 0 on a CUDA error.
double fma_peak(int fp64, int device) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return -1.0;
    const int blocks = sms * 8, threads = 256;
    const int iters = fp64 ? 2000 : 100000;
    void* out = nullptr;
    if (cudaMalloc(&out, 16) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0.0;
    for (int rep = 0; rep < 4; rep++) {
        cudaEventRecord(e0);
        if (fp64)
            fma_probe_kernel<double><<<blocks, threads>>>((double*)out, iters, 0.999999, 1e-6);
        else
            fma_probe_kernel<float><<<blocks, threads>>>((float*)out, iters, 0.9999f, 1e-4f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3);
        if (rep > 0 && flops > best) best = flops;  // the first launch is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const bool err = cudaGetLastError() != cudaSuccess;
    cudaFree(out);
    return err ? -1.0 : best;
}

}  // namespace lbm
