// The persistent 1D batch kernel of one precision, selected at compile time by
// LBM_PREC (0 FP64, 1 mixed, 2 FP32); the build compiles this file once per precision.

#include "lelbm_step.cuh"

#if !defined(LBM_PREC)
#error "compile with -DLBM_PREC=<0|1|2>"
#endif

namespace lbm {

template <int PREC>
void BatchVariant<PREC>::launch(const Model& m, const Geometry& g, const double inlet[4], int bc_left_inflow,
                                 int bc_right_inflow, const uint8_t* type, double* A, double* B, DevStats* st,
                                 unsigned long long* work, const int* order, const long long* inst_first,
                                 const int* inst_pad, int* steps_left, int nsteps, int blocks, int threads,
                                 size_t smem, cudaStream_t s) {
    auto kern = batch_persistent_kernel<PREC>;
    if (smem) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, threads, smem, s>>>(m, g, inlet[0], inlet[1], inlet[3], bc_left_inflow, bc_right_inflow, type, A,
                                       B, st, work, order, inst_first, inst_pad, steps_left, nsteps);
}

template <int PREC>
int BatchVariant<PREC>::blocks_per_sm(int threads) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel<PREC>, threads, 0);
    return per_sm;
}

template struct BatchVariant<LBM_PREC>;

}  // namespace lbm
