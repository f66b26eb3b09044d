// The cell-update kernel of one (dimension, precision) variant, selected at compile
// time by LBM_D (1 or 2) and LBM_MIXED (0 or 1); the build compiles this file once
// per variant so the four compile in parallel.

#include "lelbm_step.cuh"

#if !defined(LBM_D) || !defined(LBM_MIXED)
#error "compile with -DLBM_D=<1|2> -DLBM_MIXED=<0|1>"
#endif

namespace lbm {

template <int D, bool MIXED>
void CellVariant<D, MIXED>::launch(const Model& m, const Geometry& g, const uint8_t* type, const double* Min,
                                   double* Mout, DevStats* st, unsigned long long* work, int blocks, size_t smem,
                                   cudaStream_t s) {
    auto kern = cell_update_kernel<D, MIXED>;
    if (smem) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, 128, smem, s>>>(m, g, type, Min, Mout, st, work);
}

template <int D, bool MIXED>
int CellVariant<D, MIXED>::blocks_per_sm() {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cell_update_kernel<D, MIXED>, 128, 0);
    return per_sm;
}

template struct CellVariant<LBM_D, (LBM_MIXED != 0)>;

}  // namespace lbm
