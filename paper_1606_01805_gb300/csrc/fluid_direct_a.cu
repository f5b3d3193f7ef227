// fluid_direct_a.cu -- direct fluid kernels of the tile shapes 4 x 8,
// 4 x 4 and 2 x 8 (cells per thread x rows per block), and the tangent
// mode's one-cell tile.
#include "fluid_direct.cuh"

namespace lbib {

cudaError_t launch_fluid_direct_a(int prec, int cpt, int by, const FluidArgs& a, const Inst* one, int grid,
                                  cudaStream_t s, bool pdl) {
    if (prec == LBM_FP32_TANGENT)
        return cpt == 1 && by == 8 ? launch_fluid_shape<TF, TF, 1, 8>(a, one, grid, s, pdl) : cudaErrorInvalidValue;
    if (cpt == 4 && by == 8) return launch_fluid_prec<4, 8>(prec, a, one, grid, s, pdl);
    if (cpt == 4 && by == 4) return launch_fluid_prec<4, 4>(prec, a, one, grid, s, pdl);
    if (cpt == 2 && by == 8) return launch_fluid_prec<2, 8>(prec, a, one, grid, s, pdl);
    return cudaErrorInvalidValue;
}

}  // namespace lbib
