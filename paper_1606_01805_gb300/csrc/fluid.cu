// fluid.cu -- lattice kernels: initial field, the fused pull-stream /
// Zou-He / moments / forced-BGK collide step, and field extraction.
#include "lbib_device.cuh"

namespace lbib {

namespace {

constexpr int BY = 8;  // rows per block; blockDim = (32, BY), one warp per row segment

// BGK relaxation of Eq. 4 towards the shifted equilibrium f~eq_i = f_eq_i - w_i
// (Eq. 2), plus the Guo term (Eq. 5), in place on v.  Written over opposite
// velocity pairs (i, i'): with e_i' = -e_i, both terms split into a part even
// in e (shared) and a part odd in e (sign-flipped), so each pair costs one
// evaluation: f~eq = w (drho + rho (4.5 (e.u)^2 - 1.5 u.u)) +- 3 w rho e.u and
// G = (1 - omega/2) w [(9 (e.u)(e.F) - 3 u.F) +- 3 e.F].
template <class C>
__device__ __forceinline__ void collide(C v[9], C drho, C ux, C uy, C Fx, C Fy, C omega) {
    const C rho = C(1) + drho;
    const C usq = ux * ux + uy * uy;
    const C cf = C(1) - C(0.5) * omega;
    const C uF = ux * Fx + uy * Fy;
    {  // rest population
        const C w = C(4.0 / 9.0);
        const C feq = w * (drho - C(1.5) * rho * usq);
        v[0] = v[0] - omega * (v[0] - feq) - C(3) * cf * w * uF;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        // pairs (1,3), (2,4), (5,7), (6,8): i has e = (ex, ey), i' has -e
        const int i = p == 0 ? 1 : p == 1 ? 2 : p == 2 ? 5 : 6;
        const int j = p == 0 ? 3 : p == 1 ? 4 : p == 2 ? 7 : 8;
        const C w = C(wt(i));
        const C eu = C(cx(i)) * ux + C(cy(i)) * uy;
        const C eF = C(cx(i)) * Fx + C(cy(i)) * Fy;
        const C even = w * (drho + rho * (C(4.5) * eu * eu - C(1.5) * usq));
        const C odd = C(3) * w * rho * eu;
        const C geven = cf * w * (C(9) * eu * eF - C(3) * uF);
        const C godd = C(3) * cf * w * eF;
        v[i] = v[i] - omega * (v[i] - (even + odd)) + (geven + godd);
        v[j] = v[j] - omega * (v[j] - (even - odd)) + (geven - godd);
    }
}

// four consecutive storage elements starting at a 4-aligned index
template <class S, class C> struct Vec4;
template <> struct Vec4<float, float> {
    static __device__ __forceinline__ void load(const float* p, float v[4]) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    static __device__ __forceinline__ void store(float* p, const float v[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec4<double, double> {
    static __device__ __forceinline__ void load(const double* p, double v[4]) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void store(double* p, const double v[4]) {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
};
template <> struct Vec4<__half, float> {
    static __device__ __forceinline__ void load(const __half* p, float v[4]) {
        const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    static __device__ __forceinline__ void store(__half* p, const float v[4]) {
        const __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
        uint2 q;
        q.x = *reinterpret_cast<const unsigned*>(&a);
        q.y = *reinterpret_cast<const unsigned*>(&b);
        *reinterpret_cast<uint2*>(p) = q;
    }
};

// one cell: moments, IB force, forced BGK collision (Eqs. 2, 4-7)
template <class C>
__device__ __forceinline__ void cell_update(C v[9], const Geo& G, C fx_ib, C fy_ib) {
    C drho, jx, jy;
    moments<C>(v, drho, jx, jy);
    const C Fx = geo_g<C>(G, 0) + fx_ib, Fy = geo_g<C>(G, 1) + fy_ib;
    const C inv = C(1) / (C(1) + drho);
    const C ux = (jx + C(0.5) * Fx) * inv, uy = (jy + C(0.5) * Fy) * inv;
    collide<C>(v, drho, ux, uy, Fx, Fy, geo_omega<C>(G));
}

// Fused step, four consecutive cells (x0 .. x0+3, x0 = 4 * lane index) of
// one row per thread; a warp covers 128 cells of a row.  Populations move
// as 16-byte vectors: a pull along +-x is a one-lane shuffle of the
// neighbouring vector, with one extra element load at the warp's two ends.
// Cells on a wall or periodic edge take the per-cell general path.
// resident blocks per SM the register budget is sized for (FP64 values
// take two registers each)
template <class S> struct FluidOccupancy { static constexpr int value = 4; };
template <> struct FluidOccupancy<double> { static constexpr int value = 2; };

template <class S, class C>
__global__ void __launch_bounds__(32 * BY, FluidOccupancy<S>::value) k_fluid(FluidArgs a) {
    const Geo& G = a.G;
    const S* __restrict__ fin = static_cast<const S*>(a.fin);
    S* __restrict__ fout = static_cast<S*>(a.fout);
    C* __restrict__ flb = static_cast<C*>(a.flb);
    const int lane = threadIdx.x;
    const int x0 = (blockIdx.x * 32 + lane) * 4;
    const int y = blockIdx.y * BY + threadIdx.y;
    if (y >= G.ny) return;  // whole warp (one row)
    const long long row = (long long)y * G.pitch;
    // the vector values of cell x0 + k are its pulled populations whenever
    // the cell is interior (all 9 sources inside, none of them clamped)
    const bool rows_in = y >= 1 && y <= G.ny - 2;
    const bool any = x0 < G.nx;
    // force flags of the 32-cell segment of this thread (8 threads share one)
    const int seg = y * G.nseg + (x0 >> 5);
    const bool forced = any && a.flags[seg] != 0;

    C v[9][4];
    // vector loads for every lane (addresses clamped in-bounds), shuffles by all
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ys = min(max(y - cy(i), 0), G.ny - 1);
        const S* rp = fin + (long long)i * G.plane + (long long)ys * G.pitch;
        const int xa = min(x0, G.pitch - 4);
        C q[4];
        Vec4<S, C>::load(rp + xa, q);
        if (cx(i) == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[i][k] = q[k];
        } else if (cx(i) > 0) {  // source x - 1
            C left = __shfl_up_sync(0xffffffffu, q[3], 1);
            if (lane == 0) left = ld<S, C>(rp + max(xa - 1, 0));
            v[i][0] = left; v[i][1] = q[0]; v[i][2] = q[1]; v[i][3] = q[2];
        } else {  // source x + 1
            C right = __shfl_down_sync(0xffffffffu, q[0], 1);
            if (lane == 31) right = ld<S, C>(rp + min(xa + 4, G.pitch - 1));
            v[i][0] = q[1]; v[i][1] = q[2]; v[i][2] = q[3]; v[i][3] = right;
        }
    }
    if (any) {
        C fxi[4] = {C(0), C(0), C(0), C(0)}, fyi[4] = {C(0), C(0), C(0), C(0)};
        if (forced) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (x0 + k < G.nx) {
                    fxi[k] = flb[row + x0 + k];
                    fyi[k] = flb[G.plane + row + x0 + k];
                    flb[row + x0 + k] = C(0);
                    flb[G.plane + row + x0 + k] = C(0);
                }
        }
        // interior cells from the vector values
        unsigned edge = 0;  // bit k: cell x0 + k lies on an edge (and inside the lattice)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int xk = x0 + k;
            if (rows_in && xk >= 1 && xk <= G.nx - 2) {
                C c[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) c[i] = v[i][k];
                cell_update<C>(c, G, fxi[k], fyi[k]);
#pragma unroll
                for (int i = 0; i < 9; ++i) v[i][k] = c[i];
            } else if (xk < G.nx) {
                edge |= 1u << k;
            }
        }
        if (edge == 0 && x0 + 3 < G.nx) {
#pragma unroll
            for (int i = 0; i < 9; ++i) Vec4<S, C>::store(fout + (long long)i * G.plane + row + x0, v[i]);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (x0 + k < G.nx && !(edge >> k & 1u)) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) st<S, C>(fout + (long long)i * G.plane + row + x0 + k, v[i][k]);
                }
            // cells on a wall or periodic edge: general pull, wall completion,
            // collision, one at a time (emitted once, nothing else live)
#pragma unroll 1
            for (int k = 0; k < 4; ++k) {
                if (!(edge >> k & 1u)) continue;
                const int xk = x0 + k;
                C c[9];
                pull_general<S, C>(fin, G, xk, y, c);
                complete_walls<S, C>(fin, G, xk, y, c);
                C gx = C(0), gy = C(0);
                if (forced) {  // forces of this cell were read (and zeroed) above
                    gx = k == 0 ? fxi[0] : k == 1 ? fxi[1] : k == 2 ? fxi[2] : fxi[3];
                    gy = k == 0 ? fyi[0] : k == 1 ? fyi[1] : k == 2 ? fyi[2] : fyi[3];
                }
                cell_update<C>(c, G, gx, gy);
#pragma unroll
                for (int i = 0; i < 9; ++i) st<S, C>(fout + (long long)i * G.plane + row + xk, c[i]);
            }
        }
    }
    __syncwarp();
    if (forced && (lane & 7) == 0) a.flags[seg] = 0;
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
    C rho, ux, uy;
    node_fields<S, C>(static_cast<const S*>(a.f), a.G, x, a.y0 + r, rho, ux, uy);
    const long long k = (long long)r * a.G.nx + x;
    a.rho[k] = (double)rho;
    a.ux[k] = (double)ux;
    a.uy[k] = (double)uy;
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
    const dim3 b(32, BY), g((a.G.nx + 127) / 128, (a.G.ny + BY - 1) / BY);
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
