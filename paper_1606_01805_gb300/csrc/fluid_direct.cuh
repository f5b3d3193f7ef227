// fluid_direct.cuh -- the fused fluid kernels that read the streamed
// populations straight from global memory (vector loads and lane shuffles),
// one CTA per tile: over a batch's task list (k_fluid) or over one lattice's
// tile grid (k_fluid_one).  Instantiated per tile shape in
// fluid_direct_a.cu and fluid_direct_b.cu.
#pragma once

#include <type_traits>

#include "fluid_core.cuh"

namespace lbib {

namespace {

// resident blocks per SM the register budget is sized for: 1024 threads per
// SM for 4 FP32 / FP16 cells per thread, 512 for FP64 (two registers per
// value), 1280 (FP64: 768) for one cell per thread; 512 for one tangent-mode
// cell (four registers per value)
template <class S, int N, int BYt> struct FluidOccupancy {
    static constexpr int value =
        (sizeof(S) == 16 ? 2 : (N == 1 ? (sizeof(S) == 8 ? 3 : 5) : (sizeof(S) == 8 ? 2 : 4))) * 8 / BYt;
};

// fused fluid step over the task list (all instances): CTA b takes the
// TASKS_PER_CTA consecutive tasks from b * TASKS_PER_CTA, and further ones a
// grid apart if the grid is smaller.  A task record carries the geometry
// that addresses the tile's populations, so their loads follow the task's
// load directly; the instance descriptor (constants, flags, forces) is read
// beside them.
template <class S, class C, int N, int BYt>
__global__ void __launch_bounds__(32 * BYt, FluidOccupancy<S, N, BYt>::value) k_fluid(FluidArgs a) {
    const S* fin = static_cast<const S*>(a.fin);
    S* fout = static_cast<S*>(a.fout);
    ForceT<C>* flb = static_cast<ForceT<C>*>(a.flb);
    for (int t0 = blockIdx.x * TASKS_PER_CTA; t0 < a.ntasks; t0 += gridDim.x * TASKS_PER_CTA)
    for (int t = t0; t < min(t0 + TASKS_PER_CTA, a.ntasks); ++t) {
        const Task task = a.tasks[t];
        const Inst& I = a.insts[task.inst];
        const GlobalSrc<S, C, N> src{fin + task.f_off, (long long)task.pitch * task.ny, task.pitch, task.ny};
        fluid_tile<S, C, N>(src, I.G, fin + task.f_off, fout + task.f_off, flb + I.flb_off, a.flags + I.flags_off,
                            task.tx, task.ty * BYt + threadIdx.y, a.check, a.err, a.keep, NoWait{});
    }
}

// the same step for a context holding one lattice: its descriptor arrives
// by value (constant bank) and the grid is the tile grid itself, so no load
// stands in front of the population loads
template <class S, class C, int N, int BYt, bool PDL>
__global__ void __launch_bounds__(32 * BYt, FluidOccupancy<S, N, BYt>::value)
    k_fluid_one(FluidArgs a, Inst I) {
    const S* fin = static_cast<const S*>(a.fin) + I.f_off;
    using Wait = typename std::conditional<PDL, PdlWait, NoWait>::type;
    fluid_tile<S, C, N>(global_src<S, C, N>(fin, I.G), I.G, fin, static_cast<S*>(a.fout) + I.f_off,
                        static_cast<ForceT<C>*>(a.flb) + I.flb_off, a.flags + I.flags_off, blockIdx.x,
                        blockIdx.y * BYt + threadIdx.y, a.check, a.err, a.keep, Wait{});
}

template <class S, class C, int N, int BYt>
cudaError_t launch_fluid_shape(const FluidArgs& a, const Inst* one, int grid, cudaStream_t s, bool pdl) {
    if (one) {
        const dim3 g((one->G.nx + 32 * N - 1) / (32 * N), (one->G.ny + BYt - 1) / BYt);
        if (pdl) return launch_k(true, k_fluid_one<S, C, N, BYt, true>, g, dim3(32, BYt), s, a, *one);
        return launch_k(false, k_fluid_one<S, C, N, BYt, false>, g, dim3(32, BYt), s, a, *one);
    }
    // the task-list kernel of a batch is launched without PDL: its CTAs are
    // small and many, and the flags load is best issued with the populations
    return launch_k(false, k_fluid<S, C, N, BYt>, dim3(grid), dim3(32, BYt), s, a);
}

// the three population types of the direct kernels, one shape
template <int N, int BYt>
cudaError_t launch_fluid_prec(int prec, const FluidArgs& a, const Inst* one, int grid, cudaStream_t s, bool pdl) {
    if (prec == LBM_FP64) return launch_fluid_shape<double, double, N, BYt>(a, one, grid, s, pdl);
    if (prec == LBM_FP32) return launch_fluid_shape<float, float, N, BYt>(a, one, grid, s, pdl);
    if (prec == LBM_FP16_SHIFTED) return launch_fluid_shape<__half, float, N, BYt>(a, one, grid, s, pdl);
    return cudaErrorInvalidValue;
}

}  // namespace

}  // namespace lbib
