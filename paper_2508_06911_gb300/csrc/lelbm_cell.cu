// The cell-update kernel of one (dimension, precision) variant, selected at compile
// time by LBM_D (1 or 2) and LBM_PREC (0 FP64, 1 mixed, 2 FP32); the build compiles
// this file once per variant so the variants compile in parallel.

#include "lelbm_step.cuh"

#if !defined(LBM_D) || !defined(LBM_PREC)
#error "compile with -DLBM_D=<1|2> -DLBM_PREC=<0|1|2>"
#endif

namespace lbm {

template <int D, int PREC>
void CellVariant<D, PREC>::launch(const Model& m, const Geometry& g, const uint8_t* type, const double* Min,
                                   double* Mout, DevStats* st, unsigned long long* work, int blocks, size_t smem,
                                   cudaStream_t s) {
    auto kern = cell_update_kernel<D, PREC>;
    if (smem) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<blocks, cell_threads<PREC>(), smem, s>>>(m, g, type, Min, Mout, st, work);
}

template <int D, int PREC>
int CellVariant<D, PREC>::blocks_per_sm() {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cell_update_kernel<D, PREC>, cell_threads<PREC>(), 0);
    return per_sm;
}

template struct CellVariant<LBM_D, LBM_PREC>;

}  // namespace lbm
