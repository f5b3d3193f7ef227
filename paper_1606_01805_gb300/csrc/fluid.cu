// fluid.cu -- lattice kernels: initial field, the fused pull-stream /
// Zou-He / moments / forced-BGK collide step, and field extraction.
#include "lbib_device.cuh"

namespace lbib {

namespace {

constexpr int BY = 8;  // rows per block; blockDim = (32, BY), one warp per row segment

// shifted equilibrium f~eq_i = f_eq_i - w_i (Eq. 2) and the Guo term (Eq. 5),
// then the BGK relaxation of Eq. 4, all in place on v
template <class C>
__device__ __forceinline__ void collide(C v[9], C drho, C ux, C uy, C Fx, C Fy, C omega) {
    const C rho = C(1) + drho;
    const C usq = ux * ux + uy * uy;
    const C cf = C(1) - C(0.5) * omega;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const C w = C(wt(i));
        const C eu = C(cx(i)) * ux + C(cy(i)) * uy;
        const C feq = w * (drho + rho * (C(3) * eu + C(4.5) * eu * eu - C(1.5) * usq));
        const C gi = cf * w *
                     ((C(3) * (C(cx(i)) - ux) + C(9) * eu * C(cx(i))) * Fx +
                      (C(3) * (C(cy(i)) - uy) + C(9) * eu * C(cy(i))) * Fy);
        v[i] = v[i] - omega * (v[i] - feq) + gi;
    }
}

template <class S, class C>
__global__ void __launch_bounds__(32 * BY) k_fluid(FluidArgs a) {
    const Geo& G = a.G;
    const S* __restrict__ fin = static_cast<const S*>(a.fin);
    S* __restrict__ fout = static_cast<S*>(a.fout);
    C* __restrict__ flb = static_cast<C*>(a.flb);
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * BY + threadIdx.y;
    if (y >= G.ny) return;  // whole warp
    const int seg = y * G.nseg + blockIdx.x;
    const bool forced = a.flags[seg] != 0;  // same address for the warp
    if (x < G.nx) {
        C v[9];
        const long long c = (long long)y * G.pitch + x;
        if (x > 0 && x < G.nx - 1 && y > 0 && y < G.ny - 1) {
#pragma unroll
            for (int i = 0; i < 9; ++i)
                v[i] = ld<S, C>(fin + (long long)i * G.plane + c - (long long)cy(i) * G.pitch - cx(i));
        } else {
            pull_general<S, C>(fin, G, x, y, v);
            complete_walls<S, C>(fin, G, x, y, v);
        }
        C drho, jx, jy;
        moments<C>(v, drho, jx, jy);
        C Fx = C(G.g[0]), Fy = C(G.g[1]);
        if (forced) {
            Fx += flb[c];
            Fy += flb[G.plane + c];
            flb[c] = C(0);
            flb[G.plane + c] = C(0);
        }
        const C rho = C(1) + drho;
        const C ux = (jx + C(0.5) * Fx) / rho, uy = (jy + C(0.5) * Fy) / rho;
        collide<C>(v, drho, ux, uy, Fx, Fy, C(1.0 / G.tau));
#pragma unroll
        for (int i = 0; i < 9; ++i) st<S, C>(fout + (long long)i * G.plane + c, v[i]);
    }
    __syncwarp();
    if (forced && threadIdx.x == 0) a.flags[seg] = 0;
}

// initial post-collision field f* = f^eq(rho, u) (Eq. 2), shifted
template <class S, class C>
__global__ void k_init(S* f, Geo G, int kind, double U0) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
    if (x >= G.nx || y >= G.ny) return;
    double rho = 1.0, ux = 0.0, uy = 0.0;
    if (kind == LBM_INIT_COUETTE) {
        const double ub = G.uw[2][0], ut = G.uw[3][0];
        ux = ub + (ut - ub) * (double)y / (double)(G.ny - 1);
    } else if (kind == LBM_INIT_TAYLOR_GREEN) {
        const double kx = 2.0 * M_PI / G.nx, ky = 2.0 * M_PI / G.ny;
        ux = -U0 * cos(kx * x) * sin(ky * y);
        uy = U0 * (kx / ky) * sin(kx * x) * cos(ky * y);
        rho = 1.0 - 0.75 * U0 * U0 * (cos(2.0 * kx * x) + (kx * kx) / (ky * ky) * cos(2.0 * ky * y));
    }
    const double usq = ux * ux + uy * uy;
    const long long c = (long long)y * G.pitch + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const double eu = cx(i) * ux + cy(i) * uy;
        const double feq = wt(i) * ((rho - 1.0) + rho * (3.0 * eu + 4.5 * eu * eu - 1.5 * usq));
        st<S, C>(f + (long long)i * G.plane + c, (C)feq);
    }
}

template <class S, class C>
__global__ void k_fields(FieldArgs a) {
    const int x = blockIdx.x * 32 + threadIdx.x, r = blockIdx.y * BY + threadIdx.y;
    if (x >= a.G.nx || r >= a.rows) return;
    double rho, ux, uy;
    node_fields<S, C>(static_cast<const S*>(a.f), a.G, x, a.y0 + r, rho, ux, uy);
    const long long k = (long long)r * a.G.nx + x;
    a.rho[k] = rho;
    a.ux[k] = ux;
    a.uy[k] = uy;
}

dim3 grid_for(int nx, int rows) { return dim3((nx + 31) / 32, (rows + BY - 1) / BY); }

}  // namespace

size_t storage_bytes(int prec) {
    return prec == LBM_FP64 ? sizeof(double) : (prec == LBM_FP32 ? sizeof(float) : sizeof(__half));
}
size_t compute_bytes(int prec) { return prec == LBM_FP64 ? sizeof(double) : sizeof(float); }

cudaError_t launch_init(int prec, void* f, const Geo& G, int kind, double init_u, cudaStream_t s) {
    const dim3 b(32, BY), g = grid_for(G.nx, G.ny);
    if (prec == LBM_FP64) k_init<double, double><<<g, b, 0, s>>>((double*)f, G, kind, init_u);
    else if (prec == LBM_FP32) k_init<float, float><<<g, b, 0, s>>>((float*)f, G, kind, init_u);
    else k_init<__half, float><<<g, b, 0, s>>>((__half*)f, G, kind, init_u);
    return cudaGetLastError();
}

cudaError_t launch_fluid(int prec, const FluidArgs& a, cudaStream_t s) {
    const dim3 b(32, BY), g = grid_for(a.G.nx, a.G.ny);
    if (prec == LBM_FP64) k_fluid<double, double><<<g, b, 0, s>>>(a);
    else if (prec == LBM_FP32) k_fluid<float, float><<<g, b, 0, s>>>(a);
    else k_fluid<__half, float><<<g, b, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fields(int prec, const FieldArgs& a, cudaStream_t s) {
    const dim3 b(32, BY), g = grid_for(a.G.nx, a.rows);
    if (prec == LBM_FP64) k_fields<double, double><<<g, b, 0, s>>>(a);
    else if (prec == LBM_FP32) k_fields<float, float><<<g, b, 0, s>>>(a);
    else k_fields<__half, float><<<g, b, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbib
