// Training of the warm-start MLP (see lelbm_mlp.cuh for features, targets and the
// parameter layout): hand-written forward/backward with BF16 weights and FP32
// accumulation, FP32 master weights updated by Adam, mean-squared loss on the
// standardised targets.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <random>
#include <vector>

#include "../../include/lelbm.h"
#include "lelbm_mlp.cuh"

namespace lbm {
namespace {

constexpr int TB = 64;  // samples per block of the gradient kernel

// Sum and sum of squares of every column of a row-major [n x cols] array.
__global__ void column_stats_kernel(const float* A, long long n, int cols, double* sums) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * cols;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % cols);
        const double v = A[i];
        atomicAdd(&sums[c], v);
        atomicAdd(&sums[cols + c], v * v);
    }
}

__global__ void to_bf16_kernel(const float* src, __nv_bfloat16* dst, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16(src[i]);
}

// Loss and gradient of one block of TB samples.  Every thread runs the forward and
// backward pass of one sample and leaves its per-sample vectors in shared memory;
// the weight gradients are then block-level products (dW2 = dZ2^T H1 and so on)
// computed by slices of the flat parameter index and added to grad.
template <int D>
__global__ void __launch_bounds__(TB) mlp_grad_kernel(const __nv_bfloat16* Wb, const float* nrm, const float* X,
                                                      const float* Y, const long long* idx, long long b0, int bsize,
                                                      float scale, float* grad, double* loss) {
    using Md = MlpDims<D>;
    using Ly = MlpLayout<D>;
    constexpr int NIN = Md::NIN, NOUT = Md::NOUT, H = Md::H;
    extern __shared__ float smem[];
    float* Wf = smem;                           // NW weights as float
    float* S_XS = Wf + ((Ly::NW + 3) & ~3);     // [TB][NIN] standardised inputs
    float* S_H1 = S_XS + TB * NIN;              // [TB][H]
    float* S_Z1 = S_H1 + TB * H;                // [TB][H] z1, then dz1
    float* S_Z2 = S_Z1 + TB * H;                // [TB][H] z2, then dz2
    float* S_H2 = S_Z2 + TB * H;                // [TB][H]
    float* S_DY = S_H2 + TB * H;                // [TB][NOUT]
    for (int i = threadIdx.x; i < Ly::NW; i += blockDim.x) Wf[i] = __bfloat162float(Wb[i]);
    __syncthreads();

    const int t = threadIdx.x;
    const int r = blockIdx.x * TB + t;
    const bool valid = r < bsize;
    float* xs = S_XS + t * NIN;
    float* h1 = S_H1 + t * H;
    float* z1 = S_Z1 + t * H;
    float* z2 = S_Z2 + t * H;
    float* h2 = S_H2 + t * H;
    float* dy = S_DY + t * NOUT;
    float myloss = 0.f;
    if (valid) {
        const long long row = idx ? idx[b0 + r] : b0 + r;
#pragma unroll
        for (int m = 0; m < NIN; m++) xs[m] = (X[row * NIN + m] - nrm[m]) / nrm[NIN + m];
        for (int j = 0; j < H; j++) {
            float z = Wf[Ly::B1 + j];
#pragma unroll
            for (int m = 0; m < NIN; m++) z = fmaf(Wf[Ly::W1 + j * NIN + m], xs[m], z);
            z1[j] = z;
            h1[j] = silu(z);
        }
        for (int i = 0; i < H; i++) {
            float z = Wf[Ly::B2 + i];
            for (int j = 0; j < H; j++) z = fmaf(Wf[Ly::W2 + i * H + j], h1[j], z);
            z2[i] = z;
            h2[i] = silu(z);
        }
        for (int k = 0; k < NOUT; k++) {
            float y = Wf[Ly::B3 + k];
            for (int i = 0; i < H; i++) y = fmaf(Wf[Ly::W3 + k * H + i], h2[i], y);
            const float tgt = (Y[row * NOUT + k] - nrm[2 * NIN + k]) / nrm[2 * NIN + NOUT + k];
            const float e = y - tgt;
            myloss += e * e;
            dy[k] = scale * e;
        }
        // dz2 = (W3^T dy) * silu'(z2), stored over z2
        for (int i = 0; i < H; i++) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < NOUT; k++) s = fmaf(Wf[Ly::W3 + k * H + i], dy[k], s);
            z2[i] = s * silu_grad(z2[i]);
        }
        // dz1 = (W2^T dz2) * silu'(z1), stored over z1
        for (int j = 0; j < H; j++) {
            float s = 0.f;
            for (int i = 0; i < H; i++) s = fmaf(Wf[Ly::W2 + i * H + j], z2[i], s);
            z1[j] = s * silu_grad(z1[j]);
        }
    } else {
        for (int m = 0; m < NIN; m++) xs[m] = 0.f;
        for (int j = 0; j < H; j++) h1[j] = z1[j] = z2[j] = h2[j] = 0.f;
        for (int k = 0; k < NOUT; k++) dy[k] = 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < Ly::NW; e += blockDim.x) {
        float s = 0.f;
        if (e < Ly::B1) {
            const int j = (e - Ly::W1) / NIN, m = (e - Ly::W1) % NIN;
            for (int q = 0; q < TB; q++) s = fmaf(S_Z1[q * H + j], S_XS[q * NIN + m], s);
        } else if (e < Ly::W2) {
            const int j = e - Ly::B1;
            for (int q = 0; q < TB; q++) s += S_Z1[q * H + j];
        } else if (e < Ly::B2) {
            const int i = (e - Ly::W2) / H, j = (e - Ly::W2) % H;
            for (int q = 0; q < TB; q++) s = fmaf(S_Z2[q * H + i], S_H1[q * H + j], s);
        } else if (e < Ly::W3) {
            const int i = e - Ly::B2;
            for (int q = 0; q < TB; q++) s += S_Z2[q * H + i];
        } else if (e < Ly::B3) {
            const int k = (e - Ly::W3) / H, i = (e - Ly::W3) % H;
            for (int q = 0; q < TB; q++) s = fmaf(S_DY[q * NOUT + k], S_H2[q * H + i], s);
        } else {
            const int k = e - Ly::B3;
            for (int q = 0; q < TB; q++) s += S_DY[q * NOUT + k];
        }
        atomicAdd(&grad[e], s);
    }
    for (int o = 16; o > 0; o >>= 1) myloss += __shfl_xor_sync(0xffffffffu, myloss, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, (double)myloss);
}

// Adam on the FP32 master weights; refreshes the BF16 copy and clears the gradient.
__global__ void adam_kernel(float* master, __nv_bfloat16* Wb, float* grad, float* m1, float* m2, int nw, float lr,
                            float b1, float b2, float eps, float bc1, float bc2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
        const float g = grad[i];
        const float a = b1 * m1[i] + (1.f - b1) * g;
        const float v = b2 * m2[i] + (1.f - b2) * g * g;
        m1[i] = a;
        m2[i] = v;
        const float w = master[i] - lr * (a / bc1) / (sqrtf(v / bc2) + eps);
        master[i] = w;
        Wb[i] = __float2bfloat16(w);
        grad[i] = 0.f;
    }
}

template <int D>
size_t grad_smem_bytes() {
    using Md = MlpDims<D>;
    using Ly = MlpLayout<D>;
    return sizeof(float) * (((Ly::NW + 3) & ~3) + TB * (Md::NIN + 4 * Md::H + Md::NOUT));
}

template <int D>
int launch_grad(const __nv_bfloat16* Wb, const float* nrm, const float* X, const float* Y, const long long* idx,
                long long b0, int bsize, float scale, float* grad, double* loss, cudaStream_t s) {
    const size_t sm = grad_smem_bytes<D>();
    if (cudaFuncSetAttribute(mlp_grad_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
        return LELBM_E_CUDA;
    const int blocks = (bsize + TB - 1) / TB;
    mlp_grad_kernel<D><<<blocks, TB, sm, s>>>(Wb, nrm, X, Y, idx, b0, bsize, scale, grad, loss);
    return cudaGetLastError() == cudaSuccess ? LELBM_OK : LELBM_E_CUDA;
}

int sizes(int dims, int* nin, int* nout, long long* ntot, long long* nw) {
    if (dims == 1) {
        *nin = MlpDims<1>::NIN;
        *nout = MlpDims<1>::NOUT;
        *ntot = MlpLayout<1>::NTOT;
        *nw = MlpLayout<1>::NW;
    } else if (dims == 2) {
        *nin = MlpDims<2>::NIN;
        *nout = MlpDims<2>::NOUT;
        *ntot = MlpLayout<2>::NTOT;
        *nw = MlpLayout<2>::NW;
    } else {
        return LELBM_E_INVAL;
    }
    return LELBM_OK;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" int lelbm_mlp_size(int dims, int* n_in, int* n_out, long long* n_params, long long* n_weights) {
    int a, b;
    long long c, d;
    const int rc = sizes(dims, &a, &b, &c, &d);
    if (rc) return rc;
    if (n_in) *n_in = a;
    if (n_out) *n_out = b;
    if (n_params) *n_params = c;
    if (n_weights) *n_weights = d;
    return LELBM_OK;
}

extern "C" int lelbm_mlp_init(int dims, unsigned long long seed, const float* X, const float* Y, long long n,
                              float* params) {
    int nin, nout;
    long long ntot, nw;
    if (sizes(dims, &nin, &nout, &ntot, &nw) || !params || (n > 0 && (!X || !Y))) return LELBM_E_INVAL;
    std::vector<float> p(ntot, 0.f);
    std::mt19937_64 rng(seed);
    const int H = 64;
    auto fill = [&](int off, int rows, int cols, float gain) {
        const float lim = gain * std::sqrt(6.0f / (float)cols);
        std::uniform_real_distribution<float> U(-lim, lim);
        for (int i = 0; i < rows * cols; i++) p[off + i] = U(rng);
    };
    const int W1 = 0, B1 = W1 + H * nin, W2 = B1 + H, B2 = W2 + H * H, W3 = B2 + H;
    fill(W1, H, nin, 1.0f);
    fill(W2, H, H, 1.0f);
    fill(W3, nout, H, 0.1f);  // small output layer: training starts near the Maxwellian start
    std::vector<double> sx(2 * nin, 0.0), sy(2 * nout, 0.0);
    if (n > 0) {
        double* d = nullptr;
        if (cudaMalloc((void**)&d, sizeof(double) * 2 * (nin + nout)) != cudaSuccess) return LELBM_E_NOMEM;
        cudaMemset(d, 0, sizeof(double) * 2 * (nin + nout));
        column_stats_kernel<<<1024, 256>>>(X, n, nin, d);
        column_stats_kernel<<<1024, 256>>>(Y, n, nout, d + 2 * nin);
        cudaError_t e = cudaMemcpy(sx.data(), d, sizeof(double) * 2 * nin, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(sy.data(), d + 2 * nin, sizeof(double) * 2 * nout, cudaMemcpyDeviceToHost);
        cudaFree(d);
        if (e != cudaSuccess) return LELBM_E_CUDA;
    }
    auto stats = [&](const std::vector<double>& s, int cols, int mo, int so) {
        for (int c = 0; c < cols; c++) {
            const double mean = n > 0 ? s[c] / n : 0.0;
            const double var = n > 0 ? std::max(s[cols + c] / n - mean * mean, 0.0) : 1.0;
            const double sd = std::sqrt(var);
            p[mo + c] = (float)mean;
            p[so + c] = (float)(sd > 1e-6 * std::max(1.0, std::fabs(mean)) ? sd : 1.0);
        }
    };
    stats(sx, nin, (int)nw, (int)nw + nin);
    stats(sy, nout, (int)nw + 2 * nin, (int)nw + 2 * nin + nout);
    std::copy(p.begin(), p.end(), params);
    return LELBM_OK;
}

extern "C" int lelbm_mlp_loss_grad(int dims, const float* params, const float* X, const float* Y, long long n,
                                   float* grad, double* loss, void* stream) {
    int nin, nout;
    long long ntot, nw;
    if (sizes(dims, &nin, &nout, &ntot, &nw) || !params || !X || !Y || !grad || n < 1) return LELBM_E_INVAL;
    if (n > (1LL << 31) - TB) return LELBM_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    __nv_bfloat16* Wb = nullptr;
    double* dl = nullptr;
    if (cudaMalloc((void**)&Wb, sizeof(__nv_bfloat16) * nw) != cudaSuccess) return LELBM_E_NOMEM;
    if (cudaMalloc((void**)&dl, sizeof(double)) != cudaSuccess) {
        cudaFree(Wb);
        return LELBM_E_NOMEM;
    }
    cudaMemsetAsync(dl, 0, sizeof(double), s);
    cudaMemsetAsync(grad, 0, sizeof(float) * nw, s);
    to_bf16_kernel<<<64, 256, 0, s>>>(params, Wb, (int)nw);
    const float scale = 2.0f / (float)((double)n * nout);
    int rc = dims == 1 ? launch_grad<1>(Wb, params + nw, X, Y, nullptr, 0, (int)n, scale, grad, dl, s)
                       : launch_grad<2>(Wb, params + nw, X, Y, nullptr, 0, (int)n, scale, grad, dl, s);
    double h = 0.0;
    if (!rc && cudaMemcpyAsync(&h, dl, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = LELBM_E_CUDA;
    if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = LELBM_E_CUDA;
    cudaFree(Wb);
    cudaFree(dl);
    if (loss) *loss = h / ((double)n * nout);
    return rc;
}

extern "C" int lelbm_mlp_train(int dims, float* params, const float* X, const float* Y, long long n, int epochs,
                               int batch, float lr, unsigned long long seed, double* epoch_loss, void* stream) {
    int nin, nout;
    long long ntot, nw;
    if (sizes(dims, &nin, &nout, &ntot, &nw) || !params || !X || !Y || n < 1 || epochs < 1 || batch < 1 ||
        batch > (1 << 24) || !(lr > 0.f))
        return LELBM_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    __nv_bfloat16* Wb = nullptr;
    float *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    long long* idx = nullptr;
    double* dl = nullptr;
    int rc = LELBM_OK;
    if (cudaMalloc((void**)&Wb, sizeof(__nv_bfloat16) * nw) != cudaSuccess ||
        cudaMalloc((void**)&grad, sizeof(float) * nw) != cudaSuccess ||
        cudaMalloc((void**)&m1, sizeof(float) * nw) != cudaSuccess ||
        cudaMalloc((void**)&m2, sizeof(float) * nw) != cudaSuccess ||
        cudaMalloc((void**)&idx, sizeof(long long) * n) != cudaSuccess ||
        cudaMalloc((void**)&dl, sizeof(double) * epochs) != cudaSuccess)
        rc = LELBM_E_NOMEM;
    if (!rc) {
        cudaMemsetAsync(grad, 0, sizeof(float) * nw, s);
        cudaMemsetAsync(m1, 0, sizeof(float) * nw, s);
        cudaMemsetAsync(m2, 0, sizeof(float) * nw, s);
        cudaMemsetAsync(dl, 0, sizeof(double) * epochs, s);
        to_bf16_kernel<<<64, 256, 0, s>>>(params, Wb, (int)nw);
    }
    std::vector<long long> perm(n);
    std::iota(perm.begin(), perm.end(), 0LL);
    std::mt19937_64 rng(seed);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    long long tstep = 0;
    for (int ep = 0; ep < epochs && !rc; ep++) {
        std::shuffle(perm.begin(), perm.end(), rng);
        if (cudaMemcpyAsync(idx, perm.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            rc = LELBM_E_CUDA;
            break;
        }
        for (long long b0 = 0; b0 < n && !rc; b0 += batch) {
            const int bs = (int)std::min<long long>(batch, n - b0);
            const float scale = 2.0f / (float)((double)bs * nout);
            rc = dims == 1 ? launch_grad<1>(Wb, params + nw, X, Y, idx, b0, bs, scale, grad, dl + ep, s)
                           : launch_grad<2>(Wb, params + nw, X, Y, idx, b0, bs, scale, grad, dl + ep, s);
            tstep++;
            const float bc1 = 1.f - std::pow(b1, (float)tstep), bc2 = 1.f - std::pow(b2, (float)tstep);
            adam_kernel<<<(int)((nw + 255) / 256), 256, 0, s>>>(params, Wb, grad, m1, m2, (int)nw, lr, b1, b2, eps,
                                                              bc1, bc2);
            if (cudaGetLastError() != cudaSuccess) rc = LELBM_E_CUDA;
        }
        // the host permutation buffer is reused next epoch: wait for this epoch's copy
        if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = LELBM_E_CUDA;
    }
    if (!rc && epoch_loss) {
        std::vector<double> h(epochs);
        if (cudaMemcpy(h.data(), dl, sizeof(double) * epochs, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = LELBM_E_CUDA;
        for (int ep = 0; ep < epochs; ep++) epoch_loss[ep] = h[ep] / ((double)n * nout);
    }
    cudaFree(Wb);
    cudaFree(grad);
    cudaFree(m1);
    cudaFree(m2);
    cudaFree(idx);
    cudaFree(dl);
    return rc;
}
