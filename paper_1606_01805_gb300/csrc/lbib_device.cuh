// lbib_device.cuh -- device building blocks of the LB-IB step: the D2Q9
// lattice, storage conversions, pull-streaming with Zou-He walls, moments,
// and the moving-least-squares transfer operator.
#pragma once

#include <cuda_fp16.h>

#include "lbib_internal.h"

namespace lbib {

// ------------------------------------------ programmatic dependent launch ----
// The four kernels of a step run back to back in one stream.  Each may be
// launched with programmatic stream serialization: it then starts while its
// predecessor still runs, does the part of its work that reads nothing the
// predecessor writes, and calls pdl_wait() before anything else (the
// predecessor has then completed and its writes are visible).  Each calls
// pdl_trigger() only after its own pdl_wait(), so when a kernel starts, every
// kernel before its immediate predecessor has completed.  Launched without
// the attribute, pdl_wait() returns at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
cudaError_t launch_k(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s,
                     Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ------------------------------------------------------------ force field ----
// The IB force field of Eq. 12.  With the FP32 compute type (FP32 and
// FP16-shifted storage) it is held in fixed point, units of 2^-40 in a
// 64-bit integer: every marker's contribution is rounded to that grid once
// and added with an integer atomic, so the sum is the same bits whatever
// the order of the additions (and whether markers add directly or a
// spreading tile gathers them first).  The other compute types keep the
// field in that type (their spreading tiles gather per cell in marker
// order and add one sum per cell and particle).
template <class C> struct ForceField {
    using T = C;
    static constexpr bool FIXED = false;
    __device__ __forceinline__ static C get(const T& v) { return v; }
};
template <> struct ForceField<float> {
    using T = long long;
    static constexpr bool FIXED = true;
    __device__ __forceinline__ static float get(long long v) { return (float)v * 0x1p-40f; }
    __device__ __forceinline__ static long long fix(float v) { return __float2ll_rn(v * 0x1p40f); }
    __device__ __forceinline__ static void add(long long* p, long long v) {
        atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
    }
};
template <class C> using ForceT = typename ForceField<C>::T;

// ---------------------------------------------------------------- D2Q9 ----
// Velocities of Eq. 3: e_0 rest, e_1..e_4 axes at angles (i-1) pi/2,
// e_5..e_8 diagonals at (2i-9) pi/4; weights 4/9, 1/9, 1/36.
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr double wt(int i) {
    return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}
// index of the velocity (ex, ey)
__host__ __device__ constexpr int dir(int ex, int ey) {
    return ex == 0 ? (ey == 0 ? 0 : (ey > 0 ? 2 : 4))
                   : (ex > 0 ? (ey == 0 ? 1 : (ey > 0 ? 5 : 8)) : (ey == 0 ? 3 : (ey > 0 ? 6 : 7)));
}

// ------------------------------------------------------ storage types ----
template <class S, class C> __device__ __forceinline__ C ld(const S* p);
template <> __device__ __forceinline__ double ld<double, double>(const double* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld<float, float>(const float* p) { return __ldg(p); }
template <> __device__ __forceinline__ float ld<__half, float>(const __half* p) {
    return __half2float(__ldg(p));
}
template <> __device__ __forceinline__ TF ld<TF, TF>(const TF* p) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    TF r;
    r.v = q.x;
    r.d[0] = q.y;
    r.d[1] = q.z;
    r.d[2] = q.w;
    return r;
}
template <class S, class C> __device__ __forceinline__ void st(S* p, C v);
template <> __device__ __forceinline__ void st<TF, TF>(TF* p, TF v) {
    *reinterpret_cast<float4*>(p) = make_float4(v.v, v.d[0], v.d[1], v.d[2]);
}
template <> __device__ __forceinline__ void st<double, double>(double* p, double v) { *p = v; }
template <> __device__ __forceinline__ void st<float, float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void st<__half, float>(__half* p, float v) {
    *p = __float2half_rn(v);
}

// ------------------------------------------- constants in precision C ----
template <class C> __device__ __forceinline__ C geo_g(const Geo& G, int k);
template <> __device__ __forceinline__ double geo_g<double>(const Geo& G, int k) { return G.g[k]; }
template <> __device__ __forceinline__ float geo_g<float>(const Geo& G, int k) { return G.gf[k]; }
template <class C> __device__ __forceinline__ C geo_uw(const Geo& G, int s, int k);
template <> __device__ __forceinline__ double geo_uw<double>(const Geo& G, int s, int k) { return G.uw[s][k]; }
template <> __device__ __forceinline__ float geo_uw<float>(const Geo& G, int s, int k) { return G.uwf[s][k]; }
template <class C> __device__ __forceinline__ C geo_omega(const Geo& G);
template <> __device__ __forceinline__ double geo_omega<double>(const Geo& G) { return G.omega; }
template <> __device__ __forceinline__ float geo_omega<float>(const Geo& G) { return G.omegaf; }
// tangent mode: the body force and relaxation rate carry no derivative, the
// wall velocities carry the seeds of lbm_set_wall_tangents
template <> __device__ __forceinline__ TF geo_g<TF>(const Geo& G, int k) { return TF(G.gf[k]); }
template <> __device__ __forceinline__ TF geo_omega<TF>(const Geo& G) { return TF(G.omegaf); }
template <> __device__ __forceinline__ TF geo_uw<TF>(const Geo& G, int s, int k) {
    TF r(G.uwf[s][k]);
    for (int j = 0; j < KT; ++j) r.d[j] = G.uwdf[s][k][j];
    return r;
}
// the same in the particle real type
template <class R> __device__ __forceinline__ R geo_uw_r(const Geo& G, int s, int k);
template <> __device__ __forceinline__ double geo_uw_r<double>(const Geo& G, int s, int k) { return G.uw[s][k]; }
template <> __device__ __forceinline__ TD geo_uw_r<TD>(const Geo& G, int s, int k) {
    TD r(G.uw[s][k]);
    for (int j = 0; j < KT; ++j) r.d[j] = G.uwd[s][k][j];
    return r;
}

// ------------------------------------------------- streaming + walls ----
// Pull the populations arriving at (x, y) (Eq. 4 in pull form).  Sources
// across a wall side are unknown and left at 0; periodic sides wrap.
template <class S, class C>
__device__ __forceinline__ void pull_general(const S* __restrict__ f, const Geo& G, int x, int y,
                                             C v[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sx = x - cx(i), sy = y - cy(i);
        bool ok = true;
        if (sx < 0) {
            if (G.px) sx += G.nx; else ok = false;
        } else if (sx >= G.nx) {
            if (G.px) sx -= G.nx; else ok = false;
        }
        if (sy < 0) {
            if (G.py) sy += G.ny; else ok = false;
        } else if (sy >= G.ny) {
            if (G.py) sy -= G.ny; else ok = false;
        }
        v[i] = ok ? ld<S, C>(f + (long long)i * G.plane + (long long)sy * G.pitch + sx) : C(0);
    }
}

// Zou-He completion on a straight wall with inward normal (NX, NY): the
// three populations pointing into the fluid follow from the known ones
// and the target momentum J = rho u_w - g/2 (so that the forced velocity
// of Eq. 7 equals the wall's).  Works on shifted populations: the weights
// of the known set sum so that rho - 1 needs only the shifted values.
template <int NX, int NY, class C>
__device__ __forceinline__ void zou_he_edge(C v[9], C uwx, C uwy, C gx, C gy) {
    constexpr int TX = NY != 0 ? 1 : 0, TY = NX != 0 ? 1 : 0;  // wall tangent
    constexpr int iN = dir(NX, NY), iNo = dir(-NX, -NY);
    constexpr int iT = dir(TX, TY), iTo = dir(-TX, -TY);
    constexpr int iNpT = dir(NX + TX, NY + TY), iNmT = dir(NX - TX, NY - TY);
    constexpr int iOmT = dir(-NX - TX, -NY - TY), iOpT = dir(-NX + TX, -NY + TY);
    const C un = uwx * C(NX) + uwy * C(NY), ut = uwx * C(TX) + uwy * C(TY);
    const C gn = gx * C(NX) + gy * C(NY), gt = gx * C(TX) + gy * C(TY);
    const C k0 = v[0] + v[iT] + v[iTo];
    const C ko = v[iNo] + v[iOpT] + v[iOmT];
    const C drho = (k0 + C(2) * ko - C(0.5) * gn + un) / (C(1) - un);
    const C rho = C(1) + drho;
    const C Jn = rho * un - C(0.5) * gn, Jt = rho * ut - C(0.5) * gt;
    const C dt = C(0.5) * (v[iT] - v[iTo]);
    v[iN] = v[iNo] + C(2.0 / 3.0) * Jn;
    v[iNpT] = v[iOmT] - dt + C(0.5) * Jt + Jn * C(1.0 / 6.0);
    v[iNmT] = v[iOpT] + dt - C(0.5) * Jt + Jn * C(1.0 / 6.0);
}

// Corner between two walls, inward diagonal (SX, SY): density from the
// diagonal interior neighbour (drho_nb, shifted), axis and inward-diagonal
// unknowns by non-equilibrium bounce-back, the two buried diagonals share
// the remaining mass so that both momentum components are met.
template <int SX, int SY, class C>
__device__ __forceinline__ void zou_he_corner(C v[9], C drho_nb, C uwx, C uwy, C gx, C gy) {
    constexpr int ax = dir(SX, 0), axo = dir(-SX, 0), ay = dir(0, SY), ayo = dir(0, -SY);
    constexpr int dg = dir(SX, SY), dgo = dir(-SX, -SY), ba = dir(-SX, SY), bb = dir(SX, -SY);
    const C rho = C(1) + drho_nb;
    const C Jx = rho * uwx - C(0.5) * gx, Jy = rho * uwy - C(0.5) * gy;
    v[ax] = v[axo] + C(2.0 / 3.0) * C(SX) * Jx;
    v[ay] = v[ayo] + C(2.0 / 3.0) * C(SY) * Jy;
    v[dg] = v[dgo] + (C(SX) * Jx + C(SY) * Jy) * C(1.0 / 6.0);
    C rest = drho_nb;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        if (i != ba && i != bb) rest -= v[i];
    const C diff = (C(SX) * Jx - C(SY) * Jy) * C(1.0 / 6.0);
    v[ba] = C(0.5) * (rest - diff);
    v[bb] = C(0.5) * (rest + diff);
}

// Apply the wall completion at (x, y) if it is a wall node.
template <class S, class C>
__device__ __forceinline__ void complete_walls(const S* __restrict__ f, const Geo& G, int x, int y,
                                               C v[9]) {
    const bool bot = !G.py && y == 0, top = !G.py && y == G.ny - 1;
    const bool lef = !G.px && x == 0, rig = !G.px && x == G.nx - 1;
    const C gx = geo_g<C>(G, 0), gy = geo_g<C>(G, 1);
    if ((bot || top) && (lef || rig)) {
        const int sx = lef ? 1 : -1, sy = bot ? 1 : -1;
        C nbv[9];
        pull_general<S, C>(f, G, x + sx, y + sy, nbv);
        C d = C(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) d += nbv[i];
        const int side = bot ? 2 : 3;  // corners move with the wall along y
        const C ux = geo_uw<C>(G, side, 0), uy = geo_uw<C>(G, side, 1);
        if (bot && lef) zou_he_corner<1, 1, C>(v, d, ux, uy, gx, gy);
        else if (bot) zou_he_corner<-1, 1, C>(v, d, ux, uy, gx, gy);
        else if (lef) zou_he_corner<1, -1, C>(v, d, ux, uy, gx, gy);
        else zou_he_corner<-1, -1, C>(v, d, ux, uy, gx, gy);
    } else if (bot) {
        zou_he_edge<0, 1, C>(v, geo_uw<C>(G, 2, 0), geo_uw<C>(G, 2, 1), gx, gy);
    } else if (top) {
        zou_he_edge<0, -1, C>(v, geo_uw<C>(G, 3, 0), geo_uw<C>(G, 3, 1), gx, gy);
    } else if (lef) {
        zou_he_edge<1, 0, C>(v, geo_uw<C>(G, 0, 0), geo_uw<C>(G, 0, 1), gx, gy);
    } else if (rig) {
        zou_he_edge<-1, 0, C>(v, geo_uw<C>(G, 1, 0), geo_uw<C>(G, 1, 1), gx, gy);
    }
}

// Moments (Eqs. 6-7) of shifted populations: rho - 1 and the bare momentum.
template <class C>
__device__ __forceinline__ void moments(const C v[9], C& drho, C& jx, C& jy) {
    drho = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
    jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
    jy = (v[2] - v[4]) + (v[5] - v[8]) + (v[6] - v[7]);
}

// Density deviation drho = rho - 1 and velocity u* (constant force with its
// half step, no IB force) in the compute precision C, from shifted
// populations v.  drho is the sum of the shifted values themselves, so it
// carries no rounding of the 1 (FP32 would hold rho - 1 only to 6e-8).
template <class C>
__device__ __forceinline__ void fields_of(const C v[9], const Geo& G, C& drho, C& ux, C& uy) {
    C jx, jy;
    moments<C>(v, drho, jx, jy);
    const C inv = C(1) / (C(1) + drho);
    ux = (jx + C(0.5) * geo_g<C>(G, 0)) * inv;
    uy = (jy + C(0.5) * geo_g<C>(G, 1)) * inv;
}

// wrap / wall path of node_fields, kept out of line so the unrolled gathers
// of the marker kernels stay small
template <class S, class C>
__device__ __noinline__ bool node_fields_general(const S* __restrict__ f, const Geo& G, int ix,
                                                 int iy, C& drho, C& ux, C& uy) {
    if (ix < 0 || ix >= G.nx) {
        if (!G.px) return false;
        ix = ((ix % G.nx) + G.nx) % G.nx;
    }
    if (iy < 0 || iy >= G.ny) {
        if (!G.py) return false;
        iy = ((iy % G.ny) + G.ny) % G.ny;
    }
    C v[9];
    pull_general<S, C>(f, G, ix, iy, v);
    complete_walls<S, C>(f, G, ix, iy, v);
    fields_of<C>(v, G, drho, ux, uy);
    return true;
}

// rho - 1, u* at the unwrapped node (ix, iy); false if it lies across a wall.
// Gg is the same geometry in global memory, for the out-of-line wrap / wall
// path (G itself may live in the kernel's parameters).
template <class S, class C>
__device__ __forceinline__ bool node_fields(const S* __restrict__ f, const Geo& G, const Geo* Gg, int ix,
                                            int iy, C& drho, C& ux, C& uy) {
    if (ix > 0 && ix < G.nx - 1 && iy > 0 && iy < G.ny - 1) {
        C v[9];
        const long long c = (long long)iy * G.pitch + ix;
#pragma unroll
        for (int i = 0; i < 9; ++i)
            v[i] = ld<S, C>(f + (long long)i * G.plane + c - (long long)cy(i) * G.pitch - cx(i));
        fields_of<C>(v, G, drho, ux, uy);
        return true;
    }
    return node_fields_general<S, C>(f, *Gg, ix, iy, drho, ux, uy);
}

// --------------------------------------------------------------- MLS ----
// Weight functions of Eq. 10 (exponential, alpha = 0.3) and Eqs. 17-20,
// argument r = |x - x_k| / r_w with r_w = 2.6.  The polynomial weight is
// read as the 4-point kernel in q = 2 r (as printed its second branch takes
// the root of a negative number).
template <class W>
__device__ __forceinline__ W mls_weight(int kind, W r) {
    if (r > W(1)) return W(0);
    switch (kind) {
        case LBM_W_CUBIC: return W(2.0 / 3.0) - W(4) * r * r + W(4) * r * r * r;
        case LBM_W_QUARTIC: return W(1) + r * r * (W(-6) + r * (W(8) - W(3) * r));
        case LBM_W_COSINE: return W(0.25) * (W(1) + cospi(W(0.5) * r));
        case LBM_W_POLY: {
            const W q = W(2) * r;
            return q <= W(1) ? W(0.125) * (W(3) - W(2) * q + sqrt(W(1) + W(4) * q - W(4) * q * q))
                             : W(0.125) * (W(5) - W(2) * q - sqrt(W(-7) + W(12) * q - W(4) * q * q));
        }
        default: {
            const W s = r * W(1.0 / 0.3);
            return exp(-s * s);
        }
    }
}

}  // namespace lbib
