// lbib_device.cuh -- device building blocks of the LB-IB step: the D2Q9
// lattice, storage conversions, pull-streaming with Zou-He walls, moments,
// and the moving-least-squares transfer operator.
#pragma once

#include <cuda_fp16.h>

#include "lbib_internal.h"

namespace lbib {

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
template <class S, class C> __device__ __forceinline__ void st(S* p, C v);
template <> __device__ __forceinline__ void st<double, double>(double* p, double v) { *p = v; }
template <> __device__ __forceinline__ void st<float, float>(float* p, float v) { *p = v; }
template <> __device__ __forceinline__ void st<__half, float>(__half* p, float v) {
    *p = __float2half_rn(v);
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
    const C gx = C(G.g[0]), gy = C(G.g[1]);
    if ((bot || top) && (lef || rig)) {
        const int sx = lef ? 1 : -1, sy = bot ? 1 : -1;
        C nbv[9];
        pull_general<S, C>(f, G, x + sx, y + sy, nbv);
        C d = C(0);
#pragma unroll
        for (int i = 0; i < 9; ++i) d += nbv[i];
        const int side = bot ? 2 : 3;  // corners move with the wall along y
        const C ux = C(G.uw[side][0]), uy = C(G.uw[side][1]);
        if (bot && lef) zou_he_corner<1, 1, C>(v, d, ux, uy, gx, gy);
        else if (bot) zou_he_corner<-1, 1, C>(v, d, ux, uy, gx, gy);
        else if (lef) zou_he_corner<1, -1, C>(v, d, ux, uy, gx, gy);
        else zou_he_corner<-1, -1, C>(v, d, ux, uy, gx, gy);
    } else if (bot) {
        zou_he_edge<0, 1, C>(v, C(G.uw[2][0]), C(G.uw[2][1]), gx, gy);
    } else if (top) {
        zou_he_edge<0, -1, C>(v, C(G.uw[3][0]), C(G.uw[3][1]), gx, gy);
    } else if (lef) {
        zou_he_edge<1, 0, C>(v, C(G.uw[0][0]), C(G.uw[0][1]), gx, gy);
    } else if (rig) {
        zou_he_edge<-1, 0, C>(v, C(G.uw[1][0]), C(G.uw[1][1]), gx, gy);
    }
}

// Moments (Eqs. 6-7) of shifted populations: rho - 1 and the bare momentum.
template <class C>
__device__ __forceinline__ void moments(const C v[9], C& drho, C& jx, C& jy) {
    drho = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
    jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
    jy = (v[2] - v[4]) + (v[5] - v[8]) + (v[6] - v[7]);
}

// Density and velocity u* (constant force with its half step, no IB force)
// at the unwrapped node (ix, iy); false if the node lies across a wall.
template <class S, class C>
__device__ __forceinline__ bool node_fields(const S* __restrict__ f, const Geo& G, int ix, int iy,
                                            double& rho, double& ux, double& uy) {
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
    C d, jx, jy;
    moments<C>(v, d, jx, jy);
    rho = 1.0 + (double)d;
    ux = ((double)jx + 0.5 * G.g[0]) / rho;
    uy = ((double)jy + 0.5 * G.g[1]) / rho;
    return true;
}

// --------------------------------------------------------------- MLS ----
// Weight functions of Eq. 10 (exponential, alpha = 0.3) and Eqs. 17-20,
// argument r = |x - x_k| / r_w with r_w = 2.6.  The polynomial weight is
// read as the 4-point kernel in q = 2 r (as printed its second branch takes
// the root of a negative number).
__device__ __forceinline__ double mls_weight(int kind, double r) {
    if (r > 1.0) return 0.0;
    switch (kind) {
        case LBM_W_CUBIC: return 2.0 / 3.0 - 4.0 * r * r + 4.0 * r * r * r;
        case LBM_W_QUARTIC: return 1.0 + r * r * (-6.0 + r * (8.0 - 3.0 * r));
        case LBM_W_COSINE: return 0.25 * (1.0 + cospi(0.5 * r));
        case LBM_W_POLY: {
            const double q = 2.0 * r;
            return q <= 1.0 ? 0.125 * (3.0 - 2.0 * q + sqrt(1.0 + 4.0 * q - 4.0 * q * q))
                            : 0.125 * (5.0 - 2.0 * q - sqrt(-7.0 + 12.0 * q - 4.0 * q * q));
        }
        default: {
            const double s = r * (1.0 / 0.3);
            return exp(-s * s);
        }
    }
}

// MLS operator at (px, py) over the 3x3 nodes around the nearest node:
// phi (Eq. 8 weights) and, if D, the weights of the two linear
// coefficients (the x and y derivatives of the fit).  Linear basis in
// coordinates relative to the point; the 3x3 moment matrix A = sum W p p^T
// is inverted in FP64 by its adjugate.  (i0, j0) = lower-left node.
template <bool D>
__device__ __forceinline__ void mls(int kind, double px, double py, int& i0, int& j0, double phi[9],
                                    double dphx[9], double dphy[9]) {
    const int ic = (int)floor(px + 0.5), jc = (int)floor(py + 0.5);
    i0 = ic - 1;
    j0 = jc - 1;
    double W[9], DX[9], DY[9];
    double a00 = 0, a01 = 0, a02 = 0, a11 = 0, a12 = 0, a22 = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double dx = (double)(i0 + k % 3) - px, dy = (double)(j0 + k / 3) - py;
        const double w = mls_weight(kind, sqrt(dx * dx + dy * dy) * (1.0 / 2.6));
        W[k] = w;
        DX[k] = dx;
        DY[k] = dy;
        a00 += w;
        a01 += w * dx;
        a02 += w * dy;
        a11 += w * dx * dx;
        a12 += w * dx * dy;
        a22 += w * dy * dy;
    }
    // adjugate of the symmetric matrix
    const double c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
    const double det = a00 * c00 + a01 * c01 + a02 * c02;
    const double id = 1.0 / det;
    const double i00 = c00 * id, i01 = c01 * id, i02 = c02 * id;
#pragma unroll
    for (int k = 0; k < 9; ++k) phi[k] = W[k] * (i00 + i01 * DX[k] + i02 * DY[k]);
    if (D) {
        const double i11 = (a00 * a22 - a02 * a02) * id, i12 = (a01 * a02 - a00 * a12) * id;
        const double i22 = (a00 * a11 - a01 * a01) * id;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            dphx[k] = W[k] * (i01 + i11 * DX[k] + i12 * DY[k]);
            dphy[k] = W[k] * (i02 + i12 * DX[k] + i22 * DY[k]);
        }
    }
}

}  // namespace lbib
