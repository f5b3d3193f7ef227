// particles.cu -- the immersed-boundary kernels of the LB-IB step (built
// from the device functions of ib_core.cuh): k_probes and k_markers (one warp
// per marker block), k_spread (one CTA per 32 x 16 tile of a particle's
// support box), and their launchers.
#include "ib_core.cuh"

namespace lbib {

namespace {

constexpr int SPREAD_TY = 16;  // rows of a spreading tile of the separate kernel

template <class S, class C, class R, bool ONE>
__global__ void __launch_bounds__(32) k_probes(ParticleArgs a) {
    probe_block<S, C, R, ONE, false>(a, a.blk_base + blockIdx.x, nullptr);
}

template <class S, class C, class R, bool ONE>
__global__ void __launch_bounds__(32) k_markers(ParticleArgs a) {
    marker_block<S, C, R, ONE, false>(a, a.blk_base + blockIdx.x, nullptr);
}

template <class C, class R, bool ONE>
__global__ void __launch_bounds__(TX * SPREAD_TY, sizeof(C) == 4 ? 2 : 1) k_spread(SpreadArgs a) {
    __shared__ SpreadSmem<C, SPREAD_TY> sm;
    const int p = a.p_base + blockIdx.y;
    const int4 pr = a.np_inline ? a.part_inline[p] : a.ptab[p];
    spread_tile<C, R, ONE, false, SPREAD_TY>(a, blockIdx.x, p, pr.w, sm);
}

}  // namespace

size_t rec_bytes(int prec) {
    if (prec == LBM_FP64) return sizeof(Rec<double>);
    if (prec == LBM_FP32_TANGENT) return sizeof(Rec<TF>);
    return sizeof(Rec<float>);
}
size_t real_bytes(int prec) { return prec == LBM_FP32_TANGENT ? sizeof(TD) : sizeof(double); }
size_t particle_bytes(int prec) {
    return prec == LBM_FP32_TANGENT ? sizeof(DParticleT<TD>) : sizeof(DParticleT<double>);
}
size_t pose_bytes(int prec) {
    if (prec == LBM_FP64) return sizeof(PoseC<double>);
    if (prec == LBM_FP32_TANGENT) return sizeof(PoseC<TF>);
    return sizeof(PoseC<float>);
}

// every IB kernel is launched with programmatic stream serialization: its
// prologue reads only what no kernel still running can write (pdl_wait)
template <bool ONE>
cudaError_t probes_t(int prec, const ParticleArgs& a, int nblocks, cudaStream_t s) {
    const dim3 g(nblocks), b(32);
    if (prec == LBM_FP64) return launch_k(true, k_probes<double, double, double, ONE>, g, b, s, a);
    if (prec == LBM_FP32) return launch_k(true, k_probes<float, float, double, ONE>, g, b, s, a);
    if (prec == LBM_FP16_SHIFTED) return launch_k(true, k_probes<__half, float, double, ONE>, g, b, s, a);
    return launch_k(true, k_probes<TF, TF, TD, ONE>, g, b, s, a);
}

template <bool ONE>
cudaError_t markers_t(int prec, const ParticleArgs& a, int nblocks, cudaStream_t s) {
    const dim3 g(nblocks), b(32);
    if (prec == LBM_FP64) return launch_k(true, k_markers<double, double, double, ONE>, g, b, s, a);
    if (prec == LBM_FP32) return launch_k(true, k_markers<float, float, double, ONE>, g, b, s, a);
    if (prec == LBM_FP16_SHIFTED) return launch_k(true, k_markers<__half, float, double, ONE>, g, b, s, a);
    return launch_k(true, k_markers<TF, TF, TD, ONE>, g, b, s, a);
}

template <bool ONE>
cudaError_t spread_t(int prec, const SpreadArgs& a, dim3 g, cudaStream_t s) {
    const dim3 b(TX * SPREAD_TY);
    if (prec == LBM_FP64) return launch_k(true, k_spread<double, double, ONE>, g, b, s, a);
    if (prec == LBM_FP32_TANGENT) return launch_k(true, k_spread<TF, TD, ONE>, g, b, s, a);
    return launch_k(true, k_spread<float, double, ONE>, g, b, s, a);
}

cudaError_t launch_probes(int prec, const ParticleArgs& a, int nblocks, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    return a.single ? probes_t<true>(prec, a, nblocks, s) : probes_t<false>(prec, a, nblocks, s);
}

cudaError_t launch_markers(int prec, const ParticleArgs& a, int nblocks, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    return a.single ? markers_t<true>(prec, a, nblocks, s) : markers_t<false>(prec, a, nblocks, s);
}

cudaError_t launch_spread(int prec, const SpreadArgs& a, int np, int tiles, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    const dim3 g(tiles, np);
    return a.single ? spread_t<true>(prec, a, g, s) : spread_t<false>(prec, a, g, s);
}

}  // namespace lbib
