// fluid_direct_b.cu -- direct fluid kernels of the tile shapes 1 x 8,
// 2 x 4 and 1 x 4 (cells per thread x rows per block).
#include "fluid_direct.cuh"

namespace lbib {

cudaError_t launch_fluid_direct_b(int prec, int cpt, int by, const FluidArgs& a, const Inst* one, int grid,
                                  cudaStream_t s, bool pdl) {
    if (cpt == 1 && by == 8) return launch_fluid_prec<1, 8>(prec, a, one, grid, s, pdl);
    if (cpt == 2 && by == 4) return launch_fluid_prec<2, 4>(prec, a, one, grid, s, pdl);
    if (cpt == 1 && by == 4) return launch_fluid_prec<1, 4>(prec, a, one, grid, s, pdl);
    return cudaErrorInvalidValue;
}

}  // namespace lbib
