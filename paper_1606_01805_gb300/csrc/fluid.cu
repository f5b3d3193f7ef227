// fluid.cu -- lattice kernels: initial field, the fused pull-stream /
// Zou-He / moments / forced-BGK collide step, and field extraction.
#include "fluid_core.cuh"

namespace lbib {

namespace {

constexpr int BY = 8;  // rows per block of the init and field kernels

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

}  // namespace

size_t storage_bytes(int prec) {
    switch (prec) {
        case LBM_FP64: return sizeof(double);
        case LBM_FP32: return sizeof(float);
        case LBM_FP16_SHIFTED: return sizeof(__half);
        default: return sizeof(TF);
    }
}
// bytes of one force-field value (the fixed point of ForceField for the
// FP32 compute type)
size_t force_bytes(int prec) {
    return prec == LBM_FP32 || prec == LBM_FP16_SHIFTED ? sizeof(long long) : compute_bytes(prec);
}

bool markers_spread(int prec) { return prec == LBM_FP32 || prec == LBM_FP16_SHIFTED; }

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

// Fused fluid step with tile variant `variant` (FLUID_VARIANTS): the direct
// kernels (fluid_direct.cuh) in two translation units, or the staged
// persistent kernel (fluid_staged.cu).  The tangent mode has the one-cell
// direct tile only (variant 2): a cell's 9 populations with their
// derivatives already take 36 registers.
cudaError_t launch_fluid(int prec, int variant, const FluidArgs& a, const Inst* one, int grid, int sms,
                         cudaStream_t s, bool pdl, long long wait_limit) {
    if (a.ntasks <= 0) return cudaSuccess;
    if (!variant_valid(prec, variant)) return cudaErrorInvalidValue;
    const FluidVariant& fv = FLUID_VARIANTS[variant];
    if (fv.stages) return launch_fluid_staged(prec, fv.cpt, fv.stages, a, one, sms, s, pdl, wait_limit);
    cudaError_t e = launch_fluid_direct_a(prec, fv.cpt, fv.by, a, one, grid, s, pdl);
    if (e == cudaErrorInvalidValue) e = launch_fluid_direct_b(prec, fv.cpt, fv.by, a, one, grid, s, pdl);
    return e;
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
