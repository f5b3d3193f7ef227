// adjoint.cu -- reverse-mode (adjoint) kernels of the LB-IB step, FP32
// populations with FP64 particle work.
//
// One reverse step carries the adjoint of the post-collision populations
// lambda(f*(n+1)) and of the particle state lambda(P(n+1)) back to level n,
// for two outputs at once.  The step's forward quantities are recomputed
// from the stored f*(n), P(n) (the host reruns the step's immersed-boundary
// kernels, which leave the force field f_lb(n), its flags and P(n+1)).  In
// order:
//  k_adj_cells   per cell: the collision of Eqs. 2, 4-7 reversed (hand
//                written) -> lambda of the streamed populations g(x) and of
//                the force F(x) (kept where the force field is flagged);
//  k_adj_markers per marker: the spreading of Eq. 12, the direct forcing of
//                Eq. 11 and the MLS interpolation of Eq. 8 reversed ->
//                lambda of the updated pose, of the node velocities (added
//                to lambda(g) through the moments of Eqs. 6-7) and of the
//                marker geometry;
//  k_adj_rigid   per particle: the two-level update of Eqs. 15-16 reversed
//                -> lambda of the old state, of F and M;
//  k_adj_probes  per marker: the probe stress and surface integrals of
//                Eqs. 13-14 reversed -> lambda of the node density and
//                velocities at the probe supports, of the old pose and of
//                the marker geometry;
//  k_adj_walls   per wall node: lambda of the wall velocity (Zou-He);
//  k_adj_stream  per cell: streaming (Eq. 4, pull) reversed, with the
//                Zou-He completion's transpose at wall nodes ->
//                lambda(f*(n)).
// The per-marker Jacobians (of the MLS shape functions and everything that
// follows from the pose and the marker geometry) come from forward-mode
// dual numbers in FP64 inside each marker's thread; the node-value
// dependence, which is linear through the MLS fits, is reversed by hand.
#include "lbib_device.cuh"

namespace lbib {

namespace {

constexpr double ACS2 = 1.0 / 3.0;
constexpr double APROBE = 1.2;
constexpr int AB = 8;  // rows per block of the cell kernels

// lambda accumulators of a particle state, per output: level 0 and level 1
// of X (2), theta, U (2), W, then the sum of omega
enum { LX0 = 0, LY0, LT0, LU0, LV0, LW0, LX1, LY1, LT1, LU1, LV1, LW1, LWS, LP_N };
// per-marker geometry adjoint: rb (2), nb (2), S
enum { LG_RX = 0, LG_RY, LG_NX, LG_NY, LG_S, LG_N };
// per-particle mass-property adjoint: 1/m, 1/I, area, rho_s
enum { LS_INVM = 0, LS_INVI, LS_AREA, LS_RHO, LS_N };

__device__ __forceinline__ long long cell_index(const Inst& I, int i, int x, int y) {
    return I.f_off + (long long)i * I.G.plane + (long long)y * I.G.pitch + x;
}

// streamed (and wall-completed) shifted populations at (x, y) from f*
__device__ __forceinline__ void pulled(const float* f, const Inst& I, int x, int y, float g[9]) {
    pull_general<float, float>(f + I.f_off, I.G, x, y, g);
    complete_walls<float, float>(f + I.f_off, I.G, x, y, g);
}

// The collision of Eqs. 2, 4, 5, 7 reversed at one cell: given lam (the
// adjoint of the shifted post-collision populations), the streamed shifted
// populations g and the total force F, add the adjoint of g to lg and
// return that of F.
__device__ __forceinline__ void collide_adjoint(const float g[9], float Fx, float Fy, float omega,
                                                const float lam[9], float lg[9], float& lFx, float& lFy) {
    float drho = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        drho += g[i];
        jx += g[i] * cx(i);
        jy += g[i] * cy(i);
    }
    const float rho = 1.f + drho, inv = 1.f / rho;
    const float ux = (jx + 0.5f * Fx) * inv, uy = (jy + 0.5f * Fy) * inv;
    const float uu = ux * ux + uy * uy, cf = 1.f - 0.5f * omega;
    float rb = 0.f, ubx = 0.f, uby = 0.f, fbx = 0.f, fby = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float w = (float)wt(i), ex = (float)cx(i), ey = (float)cy(i);
        const float eu = ex * ux + ey * uy, eF = ex * Fx + ey * Fy;
        const float l = lam[i];
        lg[i] += (1.f - omega) * l;
        rb += l * omega * w * (1.f + 3.f * eu + 4.5f * eu * eu - 1.5f * uu);
        // d feq_i / d u (times omega) and d G_i / d u
        ubx += l * (omega * w * rho * (3.f * ex + 9.f * eu * ex - 3.f * ux) + cf * w * (-3.f * Fx + 9.f * eF * ex));
        uby += l * (omega * w * rho * (3.f * ey + 9.f * eu * ey - 3.f * uy) + cf * w * (-3.f * Fy + 9.f * eF * ey));
        // d G_i / d F
        fbx += l * cf * w * (3.f * (ex - ux) + 9.f * eu * ex);
        fby += l * cf * w * (3.f * (ey - uy) + 9.f * eu * ey);
    }
    // u = (j + F/2) / rho
    const float jbx = ubx * inv, jby = uby * inv;
    fbx += 0.5f * jbx;
    fby += 0.5f * jby;
    rb -= (ubx * ux + uby * uy) * inv;
#pragma unroll
    for (int i = 0; i < 9; ++i) lg[i] += rb + jbx * cx(i) + jby * cy(i);
    lFx = fbx;
    lFy = fby;
}

// the moments of Eqs. 6-7 (rho - 1 and u* = (j + g_f/2)/rho) reversed at a
// node: lambda of (rho - 1, u*) into lambda of the node's streamed
// populations (atomically: several markers may share a node)
__device__ __forceinline__ void scatter_moments(float* lg, const Inst& I, int x, int y, float ldr, float lux,
                                                float luy, float rho, float ux, float uy) {
    const float inv = 1.f / rho;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float v = ldr + (lux * (cx(i) - ux) + luy * (cy(i) - uy)) * inv;
        atomicAdd(lg + cell_index(I, i, x, y), v);
    }
}

__global__ void k_adj_cells(AdjArgs a, int inst) {
    const Inst& I = a.insts[inst];
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * AB + threadIdx.y;
    if (x >= I.G.nx || y >= I.G.ny) return;
    float g[9];
    pulled(a.f, I, x, y, g);
    const int seg = y * I.G.nseg + (x >> 5);
    const long long c = (long long)y * I.G.pitch + x;
    const bool forced = a.flags[I.flags_off + seg] != 0;
    float Fx = I.G.gf[0], Fy = I.G.gf[1];
    if (forced) {
        Fx += a.flb[I.flb_off + c];
        Fy += a.flb[I.flb_off + I.G.plane + c];
    }
#pragma unroll
    for (int o = 0; o < 2; ++o) {
        const float* lin = a.lam_in + o * a.pop_elems;
        float lam[9], lg[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            lam[i] = lin[cell_index(I, i, x, y)];
            lg[i] = 0.f;
        }
        float lFx, lFy;
        collide_adjoint(g, Fx, Fy, I.G.omegaf, lam, lg, lFx, lFy);
        float* lgo = a.lam_g + o * a.pop_elems;
#pragma unroll
        for (int i = 0; i < 9; ++i) lgo[cell_index(I, i, x, y)] = lg[i];
        if (forced) {
            a.lam_F[(2 * o) * a.flb_elems + I.flb_off + c] = lFx;
            a.lam_F[(2 * o + 1) * a.flb_elems + I.flb_off + c] = lFy;
        }
    }
}

// after every reader of the step's force field and flags: clear them for
// the next recompute (the forward fluid kernel's job in a normal step)
__global__ void k_adj_clear_forces(AdjArgs a, int inst) {
    const Inst& I = a.insts[inst];
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * AB + threadIdx.y;
    // a warp is one 32-cell row segment; no lane leaves before the warp
    // has read the segment's flag
    const bool in = x < I.G.nx && y < I.G.ny;
    const int seg = y * I.G.nseg + (x >> 5);
    const bool fl = in && a.flags[I.flags_off + seg] != 0;
    if (fl) {
        const long long c = (long long)y * I.G.pitch + x;
        a.flb[I.flb_off + c] = 0.f;
        a.flb[I.flb_off + I.G.plane + c] = 0.f;
    }
    __syncwarp();
    if (fl && (x & 31) == 0) a.flags[I.flags_off + seg] = 0;
}

// MLS of Eqs. 8-10 at the point (x, y) in a real type T (double or a dual):
// the 3x3 support around the nearest node (lower-left node (i0, j0)), the
// shape functions phi and, if D, the diffuse derivatives dpx, dpy
template <class T, bool D>
__device__ __forceinline__ void mls_point(int kind, const T& x, const T& y, int& i0, int& j0, T phi[9], T dpx[9],
                                          T dpy[9]) {
    i0 = (int)floor_value(x + 0.5) - 1;
    j0 = (int)floor_value(y + 0.5) - 1;
    T W[9], DX[9], DY[9];
    T a00 = T(0.0), a01 = T(0.0), a02 = T(0.0), a11 = T(0.0), a12 = T(0.0), a22 = T(0.0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        DX[k] = T((double)(i0 + k % 3)) - x;
        DY[k] = T((double)(j0 + k / 3)) - y;
        W[k] = mls_weight<T>(kind, sqrt(DX[k] * DX[k] + DY[k] * DY[k]) * (1.0 / 2.6));
        const T wx = W[k] * DX[k], wy = W[k] * DY[k];
        a00 += W[k];
        a01 += wx;
        a02 += wy;
        a11 += wx * DX[k];
        a12 += wx * DY[k];
        a22 += wy * DY[k];
    }
    const T c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
    const T id = T(1.0) / (a00 * c00 + a01 * c01 + a02 * c02);
    const T i00 = c00 * id, i01 = c01 * id, i02 = c02 * id;
    T i11 = T(0.0), i12 = T(0.0), i22 = T(0.0);
    if (D) {
        i11 = (a00 * a22 - a02 * a02) * id;
        i12 = (a01 * a02 - a00 * a12) * id;
        i22 = (a00 * a11 - a01 * a01) * id;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        phi[k] = W[k] * (i00 + i01 * DX[k] + i02 * DY[k]);
        if (D) {
            dpx[k] = W[k] * (i01 + i11 * DX[k] + i12 * DY[k]);
            dpy[k] = W[k] * (i02 + i12 * DX[k] + i22 * DY[k]);
        }
    }
}

// node (x, y) of lattice I, periodic sides wrapped; false across a wall
__device__ __forceinline__ bool wrap_node(const Geo& G, int& x, int& y) {
    if (x < 0 || x >= G.nx) {
        if (!G.px) return false;
        x = ((x % G.nx) + G.nx) % G.nx;
    }
    if (y < 0 || y >= G.ny) {
        if (!G.py) return false;
        y = ((y % G.ny) + G.ny) % G.ny;
    }
    return true;
}

// density - 1 and velocity u* at a node from the streamed populations
__device__ __forceinline__ void node_moments(const float* f, const Inst& I, int x, int y, float& drho, float& ux,
                                             float& uy) {
    float g[9];
    pulled(f, I, x, y, g);
    fields_of<float>(g, I.G, drho, ux, uy);
}

using D9 = Dual<double, 9>;
using D15 = Dual<double, 15>;
using D5 = Dual<double, 5>;

template <int K>
__device__ __forceinline__ Dual<double, K> seed(double v, int k) {
    Dual<double, K> r(v);
    r.d[k] = 1.0;
    return r;
}

// k_adj_markers: one thread per marker of the step's markers (the body at
// level n+1, the fluid at level n)
__global__ void k_adj_markers(AdjArgs a) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.nmark) return;
    const int p = a.marker_particle[l];
    const int4 pr = a.ptab[p];
    const Inst& I = a.insts[pr.z];
    const DParticle& Q = a.Pn1[p];  // after the update
    const double* mg = a.mgeo + 5 * (long long)l;
    // duals over (X, Y, theta, U, V, W of the new level, rbx, rby, S)
    const D9 X = seed<9>(Q.X[0][0], 0), Y = seed<9>(Q.X[0][1], 1), T = seed<9>(Q.th[0], 2);
    const D9 U = seed<9>(Q.U[0][0], 3), V = seed<9>(Q.U[0][1], 4), Wb = seed<9>(Q.W[0], 5);
    const D9 rbx = seed<9>(mg[0], 6), rby = seed<9>(mg[1], 7), S = seed<9>(mg[4], 8);
    const D9 c = cos(T), s = sin(T);
    const D9 rx = c * rbx - s * rby, ry = s * rbx + c * rby;
    const D9 px = X + rx, py = Y + ry;
    int i0, j0;
    D9 phi[9], dum[9];
    mls_point<D9, false>(a.weight, px, py, i0, j0, phi, dum, dum);
    // node velocities (fixed in this pass) and the force adjoint at the nodes
    float nu[9], nv[9], nr[9];
    double lc[2][9][2];
    int nxk[9], nyk[9];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        int xk = i0 + k % 3, yk = j0 + k / 3;
        ok = ok && wrap_node(I.G, xk, yk) && yk > 0 && yk < I.G.ny - 1;
        nxk[k] = xk;
        nyk[k] = yk;
        float dr = 0.f, ux = 0.f, uy = 0.f;
        if (ok) node_moments(a.f, I, xk, yk, dr, ux, uy);
        nr[k] = 1.f + dr;
        nu[k] = ux;
        nv[k] = uy;
        const long long cc = (long long)yk * I.G.pitch + xk;
        for (int o = 0; o < 2; ++o) {
            lc[o][k][0] = ok ? (double)a.lam_F[(2 * o) * a.flb_elems + I.flb_off + cc] : 0.0;
            lc[o][k][1] = ok ? (double)a.lam_F[(2 * o + 1) * a.flb_elems + I.flb_off + cc] : 0.0;
        }
    }
    if (!ok) {
        atomicOr(a.err, ERR_DOMAIN);
        return;
    }
    D9 Ux = D9(0.0), Uy = D9(0.0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        Ux += phi[k] * (double)nu[k];
        Uy += phi[k] * (double)nv[k];
    }
    const D9 Fx = (U - Wb * ry) - Ux, Fy = (V + Wb * rx) - Uy;  // Eq. 11
    for (int o = 0; o < 2; ++o) {
        // L = sum_k lambda_F(x_k) . (phi_k S F_l)  (Eq. 12)
        D9 L = D9(0.0);
        double sx = 0.0, sy = 0.0;  // sum_k phi_k lambda_F(x_k) (values)
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            L += phi[k] * S * (Fx * lc[o][k][0] + Fy * lc[o][k][1]);
            sx += phi[k].v * lc[o][k][0];
            sy += phi[k].v * lc[o][k][1];
        }
        double* lp = a.lamP_new + ((long long)p * 2 + o) * LP_N;
        atomicAdd(lp + LX0, L.d[0]);
        atomicAdd(lp + LY0, L.d[1]);
        atomicAdd(lp + LT0, L.d[2]);
        atomicAdd(lp + LU0, L.d[3]);
        atomicAdd(lp + LV0, L.d[4]);
        atomicAdd(lp + LW0, L.d[5]);
        double* lgm = a.lam_mgeo + ((long long)l * 2 + o) * LG_N;
        lgm[LG_RX] += L.d[6];
        lgm[LG_RY] += L.d[7];
        lgm[LG_S] += L.d[8];
        // node velocities: d L / d u_j = -S phi_j sum_k phi_k lambda_F(x_k)
        float* lg = a.lam_g + o * a.pop_elems;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const double cj = -S.v * phi[j].v;
            scatter_moments(lg, I, nxk[j], nyk[j], 0.f, (float)(cj * sx), (float)(cj * sy), nr[j], nu[j], nv[j]);
        }
    }
}

// k_adj_rigid: one thread per particle; the update from P(n) to P(n+1)
// (Eqs. 15-16 and the same two-level form for position and angle; the
// first update is u1 = u0 + a, x1 = x0 + u1)
__global__ void k_adj_rigid(AdjArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const DParticle& P = a.Pn[p];
    const DParticle& Q = a.Pn1[p];
    const int inst = a.ptab[p].z;
    const Geo& G = a.insts[inst].G;
    const double k = 2.0 / 3.0;
    const bool first = P.nupd == 0;
    const double buoy = (P.rho_s - 1.0) * P.area;
    for (int o = 0; o < 2; ++o) {
        double* ln = a.lamP_new + ((long long)p * 2 + o) * LP_N;
        double* lo = a.lamP_old + ((long long)p * 2 + o) * LP_N;
        double* fm = a.lamFM + ((long long)p * 2 + o) * 3;
        double* ls = a.lam_shape + ((long long)p * 2 + o) * LS_N;
        lo[LWS] += ln[LWS];  // the sum of omega is carried; its new term is W0 of P(n+1)
        for (int c = 0; c < 3; ++c) {
            const int ip0 = c == 0 ? LX0 : c == 1 ? LY0 : LT0, ip1 = ip0 + 6;
            const int iv0 = c == 0 ? LU0 : c == 1 ? LV0 : LW0, iv1 = iv0 + 6;
            double lvn = ln[iv0] + (c == 2 ? ln[LWS] : 0.0);
            const double lpn = ln[ip0];
            lvn += (first ? 1.0 : k) * lpn;
            lo[ip0] += ln[ip1] + (first ? 1.0 : 2.0 * k) * lpn;
            lo[ip1] += first ? 0.0 : -0.5 * k * lpn;
            lo[iv0] += ln[iv1] + (first ? 1.0 : 2.0 * k) * lvn;
            lo[iv1] += first ? 0.0 : -0.5 * k * lvn;
            const double la = (first ? 1.0 : k) * lvn;  // adjoint of the acceleration
            if (c < 2) {
                const double F = c == 0 ? Q.F[0] : Q.F[1], gc = G.grav[c];
                fm[c] = la * P.inv_mass;
                ls[LS_INVM] += la * (F + buoy * gc);
                ls[LS_AREA] += la * P.inv_mass * (P.rho_s - 1.0) * gc;
                ls[LS_RHO] += la * P.inv_mass * P.area * gc;
            } else {
                fm[2] = la * P.inv_inertia;
                ls[LS_INVI] += la * Q.M;
            }
        }
    }
}

// traction of a marker (Section 2.3) and its force / torque contributions,
// in a real type T
template <class T>
__device__ __forceinline__ void traction(const T& dr, const T& uxx, const T& uxy, const T& uyx, const T& uyy,
                                         const T& nx, const T& ny, const T& rx, const T& ry, const T& dvx,
                                         const T& dvy, const T& S, double tau, T& Fx, T& Fy, T& M) {
    const T r = T(1.0) + dr;
    const T p = ACS2 * dr + r * APROBE * (dvx * nx + dvy * ny);
    const T mu = r * (ACS2 * (tau - 0.5));
    const T txx = 2.0 * mu * uxx, tyy = 2.0 * mu * uyy, txy = mu * (uxy + uyx);
    const T tx = txx * nx + txy * ny - p * nx, ty = txy * nx + tyy * ny - p * ny;
    Fx = tx * S;
    Fy = ty * S;
    M = (rx * ty - ry * tx) * S;
}

// k_adj_probes: one thread per marker; the probes of the step (the body at
// level n with its previous level, the fluid at level n)
__global__ void k_adj_probes(AdjArgs a) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.nmark) return;
    const int p = a.marker_particle[l];
    const int4 pr = a.ptab[p];
    const Inst& I = a.insts[pr.z];
    const DParticle& P = a.Pn[p];
    const double* mg = a.mgeo + 5 * (long long)l;
    // duals over (X0, Y0, th0, th1, U0, V0, U1, V1, W0, W1, rbx, rby, nbx, nby, S)
    const D15 X0 = seed<15>(P.X[0][0], 0), Y0 = seed<15>(P.X[0][1], 1);
    const D15 T0 = seed<15>(P.th[0], 2), T1 = seed<15>(P.th[1], 3);
    const D15 U0 = seed<15>(P.U[0][0], 4), V0 = seed<15>(P.U[0][1], 5);
    const D15 U1 = seed<15>(P.U[1][0], 6), V1 = seed<15>(P.U[1][1], 7);
    const D15 W0 = seed<15>(P.W[0], 8), W1 = seed<15>(P.W[1], 9);
    const D15 rbx = seed<15>(mg[0], 10), rby = seed<15>(mg[1], 11);
    const D15 nbx = seed<15>(mg[2], 12), nby = seed<15>(mg[3], 13), S = seed<15>(mg[4], 14);
    const D15 c0 = cos(T0), s0 = sin(T0), c1 = cos(T1), s1 = sin(T1);
    const D15 rx = c0 * rbx - s0 * rby, ry = s0 * rbx + c0 * rby;
    const D15 nx = c0 * nbx - s0 * nby, ny = s0 * nbx + c0 * nby;
    const D15 r1x = c1 * rbx - s1 * rby, r1y = s1 * rbx + c1 * rby;
    const D15 qx = X0 + rx + APROBE * nx, qy = Y0 + ry + APROBE * ny;
    int i0, j0;
    D15 phi[9], dpx[9], dpy[9];
    mls_point<D15, true>(a.weight, qx, qy, i0, j0, phi, dpx, dpy);
    float nd[9], nu[9], nv[9];
    int nxk[9], nyk[9];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        int xk = i0 + k % 3, yk = j0 + k / 3;
        ok = ok && wrap_node(I.G, xk, yk) && yk > 0 && yk < I.G.ny - 1;
        nxk[k] = xk;
        nyk[k] = yk;
        float dr = 0.f, ux = 0.f, uy = 0.f;
        if (ok) node_moments(a.f, I, xk, yk, dr, ux, uy);
        nd[k] = dr;
        nu[k] = ux;
        nv[k] = uy;
    }
    if (!ok) {
        atomicOr(a.err, ERR_DOMAIN);
        return;
    }
    D15 dr = D15(0.0), uxx = D15(0.0), uxy = D15(0.0), uyx = D15(0.0), uyy = D15(0.0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        dr += phi[k] * (double)nd[k];
        uxx += dpx[k] * (double)nu[k];
        uxy += dpy[k] * (double)nu[k];
        uyx += dpx[k] * (double)nv[k];
        uyy += dpy[k] * (double)nv[k];
    }
    // change of the marker's rigid velocity between the two stored levels
    const D15 drx = rx - r1x, dry = ry - r1y, dW = W0 - W1;
    const D15 dvx = (U0 - U1) - (dW * ry + W1 * dry), dvy = (V0 - V1) + (dW * rx + W1 * drx);
    D15 Fx, Fy, M;
    traction<D15>(dr, uxx, uxy, uyx, uyy, nx, ny, rx, ry, dvx, dvy, S, I.G.tau, Fx, Fy, M);
    // the same with the five fits as the directions (everything else fixed)
    D5 f5[5] = {D5(dr.v), D5(uxx.v), D5(uxy.v), D5(uyx.v), D5(uyy.v)};
    for (int q = 0; q < 5; ++q) f5[q].d[q] = 1.0;
    D5 Gx, Gy, GM;
    traction<D5>(f5[0], f5[1], f5[2], f5[3], f5[4], D5(nx.v), D5(ny.v), D5(rx.v), D5(ry.v), D5(dvx.v), D5(dvy.v),
                 D5(S.v), I.G.tau, Gx, Gy, GM);
    for (int o = 0; o < 2; ++o) {
        const double* fm = a.lamFM + ((long long)p * 2 + o) * 3;
        const D15 L = fm[0] * Fx + fm[1] * Fy + fm[2] * M;
        double* lp = a.lamP_old + ((long long)p * 2 + o) * LP_N;
        atomicAdd(lp + LX0, L.d[0]);
        atomicAdd(lp + LY0, L.d[1]);
        atomicAdd(lp + LT0, L.d[2]);
        atomicAdd(lp + LT1, L.d[3]);
        atomicAdd(lp + LU0, L.d[4]);
        atomicAdd(lp + LV0, L.d[5]);
        atomicAdd(lp + LU1, L.d[6]);
        atomicAdd(lp + LV1, L.d[7]);
        atomicAdd(lp + LW0, L.d[8]);
        atomicAdd(lp + LW1, L.d[9]);
        double* lgm = a.lam_mgeo + ((long long)l * 2 + o) * LG_N;
        lgm[LG_RX] += L.d[10];
        lgm[LG_RY] += L.d[11];
        lgm[LG_NX] += L.d[12];
        lgm[LG_NY] += L.d[13];
        lgm[LG_S] += L.d[14];
        // the node values through the fits (linear in them)
        double lf[5];
        for (int q = 0; q < 5; ++q) lf[q] = fm[0] * Gx.d[q] + fm[1] * Gy.d[q] + fm[2] * GM.d[q];
        float* lg = a.lam_g + o * a.pop_elems;
#pragma unroll
        for (int kk = 0; kk < 9; ++kk) {
            const double ldr = phi[kk].v * lf[0];
            const double lu = dpx[kk].v * lf[1] + dpy[kk].v * lf[2];
            const double lv = dpx[kk].v * lf[3] + dpy[kk].v * lf[4];
            scatter_moments(lg, I, nxk[kk], nyk[kk], (float)ldr, (float)lu, (float)lv, 1.f + nd[kk], nu[kk], nv[kk]);
        }
    }
}

// the Zou-He completion of wall side `side` (y- = 2, y+ = 3) reversed: the
// three unknowns are affine in the six knowns with constant coefficients
// (the target density is linear in the knowns): A[u][j] = ZH_u(e_j) - ZH_u(0)
template <int NY>
__device__ __forceinline__ void zh_matrix(const Geo& G, int side, float A[9][9]) {
    float z[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) z[i] = 0.f;
    zou_he_edge<0, NY, float>(z, G.uwf[side][0], G.uwf[side][1], G.gf[0], G.gf[1]);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        float e[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) e[i] = i == j ? 1.f : 0.f;
        zou_he_edge<0, NY, float>(e, G.uwf[side][0], G.uwf[side][1], G.gf[0], G.gf[1]);
#pragma unroll
        for (int u = 0; u < 9; ++u) A[u][j] = e[u] - z[u] - (u == j ? 1.f : 0.f);
    }
}

// lambda of the streamed value of population i at node (x, y): the cell's
// lambda(g) plus, at a wall node, what the Zou-He unknowns owe it
__device__ __forceinline__ float lam_streamed(const float* lg, const Inst& I, int i, int x, int y) {
    float v = lg[cell_index(I, i, x, y)];
    const bool bot = !I.G.py && y == 0, top = !I.G.py && y == I.G.ny - 1;
    if (bot || top) {
        float A[9][9];
        if (bot) zh_matrix<1>(I.G, 2, A);
        else zh_matrix<-1>(I.G, 3, A);
#pragma unroll
        for (int u = 0; u < 9; ++u)
            if (A[u][i] != 0.f) v += A[u][i] * lg[cell_index(I, u, x, y)];
    }
    return v;
}

// streaming (pull, Eq. 4) reversed: f*_i(y) went to node y + e_i
__global__ void k_adj_stream(AdjArgs a, int inst) {
    const Inst& I = a.insts[inst];
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * AB + threadIdx.y;
    if (x >= I.G.nx || y >= I.G.ny) return;
    for (int o = 0; o < 2; ++o) {
        const float* lg = a.lam_g + o * a.pop_elems;
        float* lo = a.lam_out + o * a.pop_elems;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            int xd = x + cx(i), yd = y + cy(i);
            float v = 0.f;
            if (wrap_node(I.G, xd, yd)) v = lam_streamed(lg, I, i, xd, yd);
            lo[cell_index(I, i, x, y)] = v;
        }
    }
}

// lambda of the wall velocities: d(Zou-He unknowns)/d(u_w) at each wall node
__global__ void k_adj_walls(AdjArgs a, int inst) {
    const Inst& I = a.insts[inst];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (I.G.py || x >= I.G.nx) return;
    using D2 = Dual<float, 2>;
    for (int w = 0; w < 2; ++w) {
        const int y = w == 0 ? 0 : I.G.ny - 1, side = w == 0 ? 2 : 3;
        float g[9];
        pull_general<float, float>(a.f + I.f_off, I.G, x, y, g);
        D2 v[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) v[i] = D2(g[i]);
        D2 ux(I.G.uwf[side][0]), uy(I.G.uwf[side][1]);
        ux.d[0] = 1.f;
        uy.d[1] = 1.f;
        if (w == 0) zou_he_edge<0, 1, D2>(v, ux, uy, D2(I.G.gf[0]), D2(I.G.gf[1]));
        else zou_he_edge<0, -1, D2>(v, ux, uy, D2(I.G.gf[0]), D2(I.G.gf[1]));
        for (int o = 0; o < 2; ++o) {
            const float* lg = a.lam_g + o * a.pop_elems;
            double s0 = 0.0, s1 = 0.0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const double l = lg[cell_index(I, i, x, y)];
                s0 += l * v[i].d[0];
                s1 += l * v[i].d[1];
            }
            double* lw = a.lam_wall + ((long long)inst * 2 + o) * 8 + side * 2;
            atomicAdd(lw, s0);
            atomicAdd(lw + 1, s1);
        }
    }
}

// the initial field f* = f^eq(1, u(y)) of the planar Couette profile
// u(y) = ub + (ut - ub) y / H reversed: lambda of the two wall speeds
__global__ void k_adj_init(AdjArgs a, int inst) {
    const Inst& I = a.insts[inst];
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * AB + threadIdx.y;
    if (x >= I.G.nx || y >= I.G.ny) return;
    const double ub = I.G.uw[2][0], ut = I.G.uw[3][0], t = (double)y / (double)(I.G.ny - 1);
    const double ux = ub + (ut - ub) * t;
    for (int o = 0; o < 2; ++o) {
        const float* lin = a.lam_in + o * a.pop_elems;
        double d = 0.0;  // sum_i lambda_i d feq_i / d ux at rho = 1, uy = 0
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double ex = cx(i);
            d += lin[cell_index(I, i, x, y)] * wt(i) * (3.0 * ex + 9.0 * ex * ex * ux - 3.0 * ux);
        }
        double* lw = a.lam_wall + ((long long)inst * 2 + o) * 8;
        atomicAdd(lw + 2 * 2 + 0, d * (1.0 - t));
        atomicAdd(lw + 3 * 2 + 0, d * t);
    }
}

dim3 cell_grid(const Inst& I) { return dim3((I.G.nx + 31) / 32, (I.G.ny + AB - 1) / AB); }

}  // namespace

cudaError_t launch_adjoint_step(const AdjArgs& a, const std::vector<Inst>& insts, cudaStream_t s) {
    const dim3 b(32, AB);
    for (int i = 0; i < (int)insts.size(); ++i) k_adj_cells<<<cell_grid(insts[i]), b, 0, s>>>(a, i);
    if (a.nmark > 0) k_adj_markers<<<(a.nmark + 63) / 64, 64, 0, s>>>(a);
    if (a.np > 0) k_adj_rigid<<<(a.np + 63) / 64, 64, 0, s>>>(a);
    if (a.nmark > 0) k_adj_probes<<<(a.nmark + 63) / 64, 64, 0, s>>>(a);
    for (int i = 0; i < (int)insts.size(); ++i) {
        k_adj_walls<<<(insts[i].G.nx + 127) / 128, 128, 0, s>>>(a, i);
        k_adj_stream<<<cell_grid(insts[i]), b, 0, s>>>(a, i);
        k_adj_clear_forces<<<cell_grid(insts[i]), b, 0, s>>>(a, i);
    }
    return cudaGetLastError();
}

cudaError_t launch_adjoint_init(const AdjArgs& a, const std::vector<Inst>& insts, const std::vector<int>& init_couette,
                                cudaStream_t s) {
    const dim3 b(32, AB);
    for (int i = 0; i < (int)insts.size(); ++i)
        if (init_couette[i]) k_adj_init<<<cell_grid(insts[i]), b, 0, s>>>(a, i);
    return cudaGetLastError();
}

}  // namespace lbib
