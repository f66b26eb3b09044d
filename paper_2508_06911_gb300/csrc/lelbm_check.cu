// Check entry points of the double-float building blocks of the mixed path
// (lelbm_df.cuh): the table-driven 2^w and the double-float sum of products, run on
// caller data so a test can hold them against FP64.  The paper has no counterpart.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lelbm.h"
#include "lelbm_df.cuh"

namespace lbm {

// out[i] = the double-float 2^(w[i] 2^-54), widened to FP64 (h + l is exact in FP64).
__global__ void df_exp2_kernel(const long long* __restrict__ w, long long n, double* __restrict__ out) {
    __shared__ float2 tab[kExpTab];
    exp2_table_init(tab);
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float h, l;
        exp2_fix(w[i], tab, 0, h, l);
        out[i] = (double)h + (double)l;
    }
}

// out[r] = sum_t k[r][t] v[r][t] with v split into double-floats and accumulated by one
// thread in DFAcc, in index order (the way a streaming pass accumulates a row).
__global__ void df_dot_kernel(const float* __restrict__ k, const double* __restrict__ v, long long n_terms,
                              long long n_rows, double* __restrict__ out) {
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= n_rows) return;
    DFAcc acc;
    acc.zero();
    for (long long t = 0; t < n_terms; t++) {
        float vh, vl;
        df_split(v[r * n_terms + t], vh, vl);
        acc.add_scaled(k[r * n_terms + t], vh, vl);
    }
    out[r] = acc.value();
}

}  // namespace lbm

namespace {

// Copies host inputs to the device, runs launch(), copies n_out doubles back.
template <class F>
int run_check(const void* a, size_t a_bytes, const void* b, size_t b_bytes, double* out, size_t n_out, F launch) {
    void *da = nullptr, *db = nullptr, *dout = nullptr;
    int rc = LELBM_OK;
    if (cudaMalloc(&da, a_bytes ? a_bytes : 1) != cudaSuccess || cudaMalloc(&db, b_bytes ? b_bytes : 1) != cudaSuccess ||
        cudaMalloc(&dout, n_out * sizeof(double) + 1) != cudaSuccess) {
        rc = LELBM_E_NOMEM;
    } else if ((a_bytes && cudaMemcpy(da, a, a_bytes, cudaMemcpyHostToDevice) != cudaSuccess) ||
               (b_bytes && cudaMemcpy(db, b, b_bytes, cudaMemcpyHostToDevice) != cudaSuccess)) {
        rc = LELBM_E_CUDA;
    } else {
        launch(da, db, (double*)dout);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(out, dout, n_out * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = LELBM_E_CUDA;
    }
    cudaFree(da);
    cudaFree(db);
    cudaFree(dout);
    cudaGetLastError();
    return rc;
}

}  // namespace

extern "C" int lelbm_df_exp2(const long long* w, long long n, double* out) {
    if (n < 0 || (n > 0 && (!w || !out))) return LELBM_E_INVAL;
    if (n == 0) return LELBM_OK;
    for (long long i = 0; i < n; i++)
        if (w[i] > (long long)(200.0 * lbm::kFixOne) || w[i] < -(long long)(120.0 * lbm::kFixOne)) return LELBM_E_INVAL;
    return run_check(w, sizeof(long long) * (size_t)n, nullptr, 0, out, (size_t)n, [&](void* da, void*, double* dout) {
        lbm::df_exp2_kernel<<<(int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256>>>((const long long*)da, n, dout);
    });
}

extern "C" int lelbm_df_dot(const float* k, const double* v, long long n_terms, long long n_rows, double* out) {
    if (n_terms < 0 || n_rows < 0 || (n_terms * n_rows > 0 && (!k || !v)) || (n_rows > 0 && !out)) return LELBM_E_INVAL;
    if (n_rows == 0) return LELBM_OK;
    const size_t nt = (size_t)(n_terms * n_rows);
    return run_check(k, sizeof(float) * nt, v, sizeof(double) * nt, out, (size_t)n_rows,
                     [&](void* dk, void* dv, double* dout) {
                         lbm::df_dot_kernel<<<(int)((n_rows + 127) / 128), 128>>>((const float*)dk, (const double*)dv,
                                                                                  n_terms, n_rows, dout);
                     });
}
