// fluid.cu -- lattice kernels: initial field, the fused pull-stream /
// Zou-He / moments / forced-BGK collide step, and field extraction.
#include "fluid_core.cuh"

namespace lbib {

namespace {

constexpr int BY = 8;  // rows per block of the init and field kernels

// resident blocks per SM the register budget is sized for: 1024 threads per
// SM for 4 FP32 / FP16 cells per thread, 512 for FP64 (two registers per
// value), 1280 (FP64: 768) for one cell per thread; 512 for one tangent-mode
// cell (four registers per value)
template <class S, int N, int BYt> struct FluidOccupancy {
    static constexpr int value =
        (sizeof(S) == 16 ? 2 : (N == 1 ? (sizeof(S) == 8 ? 3 : 5) : (sizeof(S) == 8 ? 2 : 4))) * 8 / BYt;
};

// fused fluid step over the task list (all instances): CTA b takes the
// TASKS_PER_CTA consecutive tasks from b * TASKS_PER_CTA (mostly tiles of one
// lattice, whose task records and descriptor then come from L1 after the
// first), and further ones a grid apart if the grid is smaller
template <class S, class C, int N, int BYt>
__global__ void __launch_bounds__(32 * BYt, FluidOccupancy<S, N, BYt>::value) k_fluid(FluidArgs a) {
    const S* fin = static_cast<const S*>(a.fin);
    S* fout = static_cast<S*>(a.fout);
    C* flb = static_cast<C*>(a.flb);
    for (int t0 = blockIdx.x * TASKS_PER_CTA; t0 < a.ntasks; t0 += gridDim.x * TASKS_PER_CTA)
    for (int t = t0; t < min(t0 + TASKS_PER_CTA, a.ntasks); ++t) {
        const int4 task = a.tasks[t];
        const Inst& I = a.insts[task.x];
        fluid_tile<S, C, N, false>(global_src<S, C, N>(fin + I.f_off, I.G), I.G, fin + I.f_off,
                                   fout + I.f_off, flb + I.flb_off, a.flags + I.flags_off, task.y,
                                   task.z * BYt + threadIdx.y, a.check, a.err);
    }
}

// the same step for a context holding one lattice: its descriptor arrives
// by value (constant bank) and the grid is the tile grid itself, so no load
// stands in front of the population loads
template <class S, class C, int N, int BYt, bool PDL>
__global__ void __launch_bounds__(32 * BYt, FluidOccupancy<S, N, BYt>::value)
    k_fluid_one(FluidArgs a, Inst I) {
    const S* fin = static_cast<const S*>(a.fin) + I.f_off;
    fluid_tile<S, C, N, PDL>(global_src<S, C, N>(fin, I.G), I.G, fin, static_cast<S*>(a.fout) + I.f_off,
                             static_cast<C*>(a.flb) + I.flb_off, a.flags + I.flags_off, blockIdx.x,
                             blockIdx.y * BYt + threadIdx.y, a.check, a.err);
}

// initial post-collision field f* = f^eq(rho, u) (Eq. 2), shifted; R is the
// real type of the field (with tangents, the Couette profile carries the
// derivatives of the wall speeds)
template <class S, class C, class R>
__global__ void k_init(S* f, Geo G, int kind, double U0) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
    if (x >= G.nx || y >= G.ny) return;
    R rho = R(1.0), ux = R(0.0), uy = R(0.0);
    if (kind == LBM_INIT_COUETTE) {
        const R ub = geo_uw_r<R>(G, 2, 0), ut = geo_uw_r<R>(G, 3, 0);
        ux = ub + (ut - ub) * ((double)y / (double)(G.ny - 1));
    } else if (kind == LBM_INIT_TAYLOR_GREEN) {
        const double kx = 2.0 * M_PI / G.nx, ky = 2.0 * M_PI / G.ny;
        ux = R(-U0 * cos(kx * x) * sin(ky * y));
        uy = R(U0 * (kx / ky) * sin(kx * x) * cos(ky * y));
        rho = R(1.0 - 0.75 * U0 * U0 * (cos(2.0 * kx * x) + (kx * kx) / (ky * ky) * cos(2.0 * ky * y)));
    }
    const R usq = ux * ux + uy * uy;
    const long long c = (long long)y * G.pitch + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const R eu = (double)cx(i) * ux + (double)cy(i) * uy;
        const R feq = wt(i) * ((rho - 1.0) + rho * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq));
        st<S, C>(f + (long long)i * G.plane + c, (C)feq);
    }
}

// host-layout populations <-> stored shifted populations, a chunk of rows
// [y0, y0 + rows) at a time: h is [9][rows][nx] doubles of unshifted f_i;
// the storage holds f_i - w_i in S (the tangent mode: no derivative)
template <class S, class C>
__global__ void k_put_pops(const double* __restrict__ h, Geo G, int y0, int rows, S* __restrict__ f) {
    const int x = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * BY + threadIdx.y;
    if (x >= G.nx || r >= rows) return;
    const long long c = (long long)(y0 + r) * G.pitch + x, k = (long long)r * G.nx + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double v = h[(long long)i * rows * G.nx + k] - wt(i);
        st<S, C>(f + (long long)i * G.plane + c, C(static_cast<typename DualTraits<C>::value>(v)));
    }
}
template <class S, class C>
__global__ void k_get_pops(const S* __restrict__ f, Geo G, int y0, int rows, double* __restrict__ h) {
    const int x = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * BY + threadIdx.y;
    if (x >= G.nx || r >= rows) return;
    const long long c = (long long)(y0 + r) * G.pitch + x, k = (long long)r * G.nx + x;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        h[(long long)i * rows * G.nx + k] = (double)value_of(ld<S, C>(f + (long long)i * G.plane + c)) + wt(i);
}

__device__ __forceinline__ void put_tangents(double, double*, long long) {}
__device__ __forceinline__ void put_tangents(float, double*, long long) {}
__device__ __forceinline__ void put_tangents(const TF& v, double* out, long long stride) {
#pragma unroll
    for (int j = 0; j < KT; ++j) out[j * stride] = (double)v.d[j];
}

template <class S, class C>
__global__ void k_fields(FieldArgs a) {
    const int x = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * BY + threadIdx.y;
    if (x >= a.I.G.nx || r >= a.rows) return;
    C drho, ux, uy;
    node_fields<S, C>(static_cast<const S*>(a.f) + a.I.f_off, a.I.G, &a.I.G, x, a.y0 + r, drho, ux, uy);
    const C rho = C(1) + drho;
    const long long k = (long long)r * a.I.G.nx + x;
    a.rho[k] = (double)value_of(rho);
    a.ux[k] = (double)value_of(ux);
    a.uy[k] = (double)value_of(uy);
    if (a.tan) {  // tangent mode: d(rho, ux, uy)/dp_j as planes [3][K][rows][nx]
        const long long pl = (long long)a.rows * a.I.G.nx;
        put_tangents(rho, a.tan + k, pl);
        put_tangents(ux, a.tan + DualTraits<C>::K * pl + k, pl);
        put_tangents(uy, a.tan + 2 * DualTraits<C>::K * pl + k, pl);
    }
}

dim3 grid_for(int nx, int rows) { return dim3((nx + 31) / 32, (rows + BY - 1) / BY); }

template <class S, class C, int V>
cudaError_t launch_fluid_v(const FluidArgs& a, const Inst* one, int grid, cudaStream_t s, bool pdl) {
    constexpr int N = FLUID_VARIANTS[V].cpt, BYt = FLUID_VARIANTS[V].by;
    if (one) {
        const dim3 g((one->G.nx + 32 * N - 1) / (32 * N), (one->G.ny + BYt - 1) / BYt);
        if (pdl) return launch_k(true, k_fluid_one<S, C, N, BYt, true>, g, dim3(32, BYt), s, a, *one);
        return launch_k(false, k_fluid_one<S, C, N, BYt, false>, g, dim3(32, BYt), s, a, *one);
    }
    // the task-list kernel of a batch is launched without PDL: its CTAs are
    // small and many, and the flags load is best issued with the populations
    return launch_k(false, k_fluid<S, C, N, BYt>, dim3(grid), dim3(32, BYt), s, a);
}

template <class S, class C>
cudaError_t launch_fluid_t(int variant, const FluidArgs& a, const Inst* one, int grid, cudaStream_t s,
                           bool pdl) {
    switch (variant) {
        case 1: return launch_fluid_v<S, C, 1>(a, one, grid, s, pdl);
        case 2: return launch_fluid_v<S, C, 2>(a, one, grid, s, pdl);
        default: return launch_fluid_v<S, C, 0>(a, one, grid, s, pdl);
    }
}

template <class S, class C, int V>
int blocks_v() {
    constexpr int N = FLUID_VARIANTS[V].cpt, BYt = FLUID_VARIANTS[V].by;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fluid<S, C, N, BYt>, 32 * BYt, 0) != cudaSuccess)
        n = 1;
    return n > 0 ? n : 1;
}

template <class S, class C>
int blocks_t(int variant) {
    switch (variant) {
        case 1: return blocks_v<S, C, 1>();
        case 2: return blocks_v<S, C, 2>();
        default: return blocks_v<S, C, 0>();
    }
}

}  // namespace

size_t storage_bytes(int prec) {
    switch (prec) {
        case LBM_FP64: return sizeof(double);
        case LBM_FP32: return sizeof(float);
        case LBM_FP16_SHIFTED: return sizeof(__half);
        default: return sizeof(TF);
    }
}
size_t compute_bytes(int prec) {
    return prec == LBM_FP64 ? sizeof(double) : (prec == LBM_FP32_TANGENT ? sizeof(TF) : sizeof(float));
}

cudaError_t launch_init(int prec, void* fbuf, const Inst& I, int kind, double init_u, cudaStream_t s) {
    const dim3 b(32, BY), g = grid_for(I.G.nx, I.G.ny);
    if (prec == LBM_FP64)
        k_init<double, double, double><<<g, b, 0, s>>>((double*)fbuf + I.f_off, I.G, kind, init_u);
    else if (prec == LBM_FP32)
        k_init<float, float, double><<<g, b, 0, s>>>((float*)fbuf + I.f_off, I.G, kind, init_u);
    else if (prec == LBM_FP16_SHIFTED)
        k_init<__half, float, double><<<g, b, 0, s>>>((__half*)fbuf + I.f_off, I.G, kind, init_u);
    else
        k_init<TF, TF, TD><<<g, b, 0, s>>>((TF*)fbuf + I.f_off, I.G, kind, init_u);
    return cudaGetLastError();
}

// the tangent mode has the one-cell tile only (variant 2): a cell's 9
// populations with their derivatives already take 36 registers
cudaError_t launch_fluid(int prec, int variant, const FluidArgs& a, const Inst* one, int grid,
                         cudaStream_t s, bool pdl) {
    if (a.ntasks <= 0) return cudaSuccess;
    if (prec == LBM_FP64) return launch_fluid_t<double, double>(variant, a, one, grid, s, pdl);
    if (prec == LBM_FP32) return launch_fluid_t<float, float>(variant, a, one, grid, s, pdl);
    if (prec == LBM_FP16_SHIFTED) return launch_fluid_t<__half, float>(variant, a, one, grid, s, pdl);
    return launch_fluid_v<TF, TF, 2>(a, one, grid, s, pdl);
}

int fluid_blocks_per_sm(int prec, int variant) {
    if (prec == LBM_FP64) return blocks_t<double, double>(variant);
    if (prec == LBM_FP32) return blocks_t<float, float>(variant);
    if (prec == LBM_FP16_SHIFTED) return blocks_t<__half, float>(variant);
    return blocks_v<TF, TF, 2>();
}

cudaError_t launch_put_pops(int prec, const double* h, const Inst& I, int y0, int rows, void* fbuf,
                            cudaStream_t s) {
    const dim3 b(32, BY), g = grid_for(I.G.nx, rows);
    if (prec == LBM_FP64) k_put_pops<double, double><<<g, b, 0, s>>>(h, I.G, y0, rows, (double*)fbuf + I.f_off);
    else if (prec == LBM_FP32) k_put_pops<float, float><<<g, b, 0, s>>>(h, I.G, y0, rows, (float*)fbuf + I.f_off);
    else if (prec == LBM_FP16_SHIFTED)
        k_put_pops<__half, float><<<g, b, 0, s>>>(h, I.G, y0, rows, (__half*)fbuf + I.f_off);
    else k_put_pops<TF, TF><<<g, b, 0, s>>>(h, I.G, y0, rows, (TF*)fbuf + I.f_off);
    return cudaGetLastError();
}

cudaError_t launch_get_pops(int prec, const void* fbuf, const Inst& I, int y0, int rows, double* h,
                            cudaStream_t s) {
    const dim3 b(32, BY), g = grid_for(I.G.nx, rows);
    if (prec == LBM_FP64)
        k_get_pops<double, double><<<g, b, 0, s>>>((const double*)fbuf + I.f_off, I.G, y0, rows, h);
    else if (prec == LBM_FP32)
        k_get_pops<float, float><<<g, b, 0, s>>>((const float*)fbuf + I.f_off, I.G, y0, rows, h);
    else if (prec == LBM_FP16_SHIFTED)
        k_get_pops<__half, float><<<g, b, 0, s>>>((const __half*)fbuf + I.f_off, I.G, y0, rows, h);
    else k_get_pops<TF, TF><<<g, b, 0, s>>>((const TF*)fbuf + I.f_off, I.G, y0, rows, h);
    return cudaGetLastError();
}

__global__ void k_raise(unsigned* err, unsigned bits) { atomicOr(err, bits); }

cudaError_t launch_raise(unsigned* err, unsigned bits, cudaStream_t s) {
    k_raise<<<1, 1, 0, s>>>(err, bits);
    return cudaGetLastError();
}

cudaError_t launch_fields(int prec, const FieldArgs& a, cudaStream_t s) {
    const dim3 b(32, BY), g = grid_for(a.I.G.nx, a.rows);
    if (prec == LBM_FP64) k_fields<double, double><<<g, b, 0, s>>>(a);
    else if (prec == LBM_FP32) k_fields<float, float><<<g, b, 0, s>>>(a);
    else if (prec == LBM_FP16_SHIFTED) k_fields<__half, float><<<g, b, 0, s>>>(a);
    else k_fields<TF, TF><<<g, b, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbib
