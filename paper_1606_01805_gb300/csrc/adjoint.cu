// adjoint.cu -- reverse-mode (adjoint) kernels of the LB-IB step, FP32
// populations with FP64 particle work.
//
// One reverse step carries the adjoint of the post-collision populations
// lambda(f*(n+1)) and of the particle state lambda(P(n+1)) back to level n,
// for two outputs at once.  The step's forward quantities are recomputed
// from the stored f*(n), P(n) (the host reruns the step's immersed-boundary
// kernels, which leave the force field f_lb(n), its flags and P(n+1)).  In
// order:
//  k_adj_cells   per cell: streaming (Eq. 4, pull) reversed, with the
//                Zou-He completion's transpose at wall nodes, turns the next
//                level's lambda(g) into lambda(f*(n+1)); then the collision
//                of Eqs. 2, 4-7 reversed (hand written) -> lambda of the
//                streamed populations g(x) and of the force F(x) (kept where
//                the force field is flagged); on the wall rows also lambda of
//                the wall velocities;
//  k_adj_markers per marker: the spreading of Eq. 12, the direct forcing of
//                Eq. 11 and the MLS interpolation of Eq. 8 reversed ->
//                lambda of the updated pose, of the node velocities (added
//                to lambda(g) through the moments of Eqs. 6-7) and of the
//                marker geometry;
//  k_adj_rigid   per particle: the two-level update of Eqs. 15-16 reversed
//                -> lambda of the old state, of F and M;
//  k_adj_probes_pre / _fin  per marker: the probe stress and surface
//                integrals of Eqs. 13-14 reversed -> lambda of the node
//                density and velocities at the probe supports, of the old
//                pose and of the marker geometry.  Their Jacobians do not
//                depend on any adjoint: _pre forms them (on a second stream,
//                beside the kernels above), _fin contracts them with the
//                force and torque adjoint of k_adj_rigid;
// The markers' and probes' shares of lambda(g(n)) are added before the
// next (earlier) level's k_adj_cells reads it.  The cell kernels walk one
// list of blocks over all instances of a batch.
// The per-marker Jacobians (of everything that follows from the pose and
// the marker geometry) come from forward-mode dual numbers in FP32 inside
// each marker's thread, with positions relative to the node at or below
// the particle's centre; the MLS shape functions enter through their
// gradient in the point (a dual over its two coordinates), and the
// node-value dependence, linear through the MLS fits, is reversed by hand.
// Accumulations across markers and steps are FP64.
#include "lbib_device.cuh"

namespace lbib {

namespace {

constexpr double ACS2 = 1.0 / 3.0;
constexpr double APROBE = 1.2;
constexpr int AB = 8;  // rows per block of the cell kernels

using F2 = Dual<float, 2>;
using F5 = Dual<float, 5>;
using F9 = Dual<float, 9>;
using F15 = Dual<float, 15>;

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

// density, velocity of Eq. 7 and total force at a cell, from its streamed
// shifted populations g and the force F
struct CellState {
    float rho, inv, ux, uy, Fx, Fy;
};
__device__ __forceinline__ CellState cell_state(const float g[9], float Fx, float Fy) {
    float drho = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        drho += g[i];
        if (cx(i) != 0) jx += cx(i) > 0 ? g[i] : -g[i];
        if (cy(i) != 0) jy += cy(i) > 0 ? g[i] : -g[i];
    }
    const float rho = 1.f + drho, inv = 1.f / rho;
    return CellState{rho, inv, (jx + 0.5f * Fx) * inv, (jy + 0.5f * Fy) * inv, Fx, Fy};
}

// The collision of Eqs. 2, 4, 5, 7 reversed at one cell: given lam (the
// adjoint of the shifted post-collision populations), add the adjoint of
// the streamed populations to lg and return that of the force.  Every sum
// over the velocities that the equilibrium and the Guo term need is a
// weighted moment of lam (M0 = sum w lam, Ma = sum w lam e_a, Mab = sum w
// lam e_a e_b), so the populations enter only through those six moments.
__device__ __forceinline__ void collide_adjoint(const CellState& c, float omega, const float lam[9], float lg[9],
                                                float& lFx, float& lFy) {
    float M0 = 0.f, Mx = 0.f, My = 0.f, Mxx = 0.f, Mxy = 0.f, Myy = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const float wl = (float)wt(i) * lam[i];
        M0 += wl;
        if (cx(i) != 0) {
            Mx += cx(i) > 0 ? wl : -wl;
            Mxx += wl;
        }
        if (cy(i) != 0) {
            My += cy(i) > 0 ? wl : -wl;
            Myy += wl;
        }
        if (cx(i) != 0 && cy(i) != 0) Mxy += cx(i) * cy(i) > 0 ? wl : -wl;
    }
    const float ux = c.ux, uy = c.uy, uu = ux * ux + uy * uy, cf = 1.f - 0.5f * omega;
    const float Sx = ux * Mxx + uy * Mxy, Sy = ux * Mxy + uy * Myy;  // sum w lam (e.u) e
    // d/d rho of sum lam feq (times omega), and d/du of sum lam (omega feq + cf G)
    const float rb = omega * (M0 * (1.f - 1.5f * uu) + 3.f * (ux * Mx + uy * My) + 4.5f * (ux * Sx + uy * Sy));
    const float ubx = omega * c.rho * (3.f * Mx + 9.f * Sx - 3.f * ux * M0) +
                      cf * (9.f * (c.Fx * Mxx + c.Fy * Mxy) - 3.f * c.Fx * M0);
    const float uby = omega * c.rho * (3.f * My + 9.f * Sy - 3.f * uy * M0) +
                      cf * (9.f * (c.Fx * Mxy + c.Fy * Myy) - 3.f * c.Fy * M0);
    // u = (j + F/2) / rho
    const float jbx = ubx * c.inv, jby = uby * c.inv;
    const float rt = rb - (ubx * ux + uby * uy) * c.inv;
#pragma unroll
    for (int i = 0; i < 9; ++i) lg[i] += (1.f - omega) * lam[i] + rt + jbx * cx(i) + jby * cy(i);
    // d/dF of sum lam cf G, and through u
    lFx = cf * (3.f * (Mx - ux * M0) + 9.f * Sx) + 0.5f * jbx;
    lFy = cf * (3.f * (My - uy * M0) + 9.f * Sy) + 0.5f * jby;
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

// the cell kernels walk a list of 32 x AB blocks over all instances
// (instance, block x, block y, Couette-initialised flag)
struct CellPos {
    const Inst* I;
    int inst, x, y, flags;
};
__device__ __forceinline__ CellPos cell_pos(const AdjArgs& a) {
    const int4 b = a.cblk[blockIdx.x];
    return CellPos{a.insts + b.x, b.x, b.y * 32 + (int)threadIdx.x, b.z * AB + (int)threadIdx.y, b.w};
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

// lambda(f*_i) at (x, y) for both outputs, from the next level's lambda(g):
// streaming (pull, Eq. 4) reversed, f*_i(x) went to node x + e_i; at a y
// wall node also what the Zou-He unknowns owe the known populations (the
// transposes of k_adj_zh)
__device__ __forceinline__ void lam_post(const AdjArgs& a, const Inst& I, int inst, int x, int y, float lam[2][9]) {
    const Geo& G = I.G;
    const int xm = x > 0 ? x - 1 : (G.px ? G.nx - 1 : -1), xp = x < G.nx - 1 ? x + 1 : (G.px ? 0 : -1);
    const int ym = y > 0 ? y - 1 : (G.py ? G.ny - 1 : -1), yp = y < G.ny - 1 ? y + 1 : (G.py ? 0 : -1);
    const float* __restrict__ l0 = a.lam_gp + I.f_off;
    const float* __restrict__ l1 = l0 + a.pop_elems;
    int xs[9], ys[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        xs[i] = cx(i) == 0 ? x : (cx(i) > 0 ? xp : xm);
        ys[i] = cy(i) == 0 ? y : (cy(i) > 0 ? yp : ym);
        const bool ok = xs[i] >= 0 && ys[i] >= 0;
        const long long e = (long long)i * G.plane + (long long)ys[i] * G.pitch + xs[i];
        lam[0][i] = ok ? l0[e] : 0.f;
        lam[1][i] = ok ? l1[e] : 0.f;
    }
    if (!G.py && (y <= 1 || y >= G.ny - 2)) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const bool bot = ys[i] == 0, top = ys[i] == G.ny - 1;
            if (xs[i] < 0 || ys[i] < 0 || !(bot || top)) continue;
            const float* A = a.zh + ((long long)inst * 2 + (top ? 1 : 0)) * 81;
            const long long e = (long long)ys[i] * G.pitch + xs[i];
            for (int u = 0; u < 9; ++u) {
                const float c = A[u * 9 + i];
                if (c != 0.f) {
                    lam[0][i] += c * l0[u * G.plane + e];
                    lam[1][i] += c * l1[u * G.plane + e];
                }
            }
        }
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One cell of level n: lambda(f*(n)) from the next level's lambda(g)
// (streaming reversed), then the collision of Eqs. 2, 4-7 reversed ->
// lambda(g(n)) and, in flagged segments, lambda of the IB force.  On the y
// wall rows also lambda of the wall velocities (the derivative of the
// Zou-He unknowns by u_w against the row's own lambda(g): no marker support
// reaches a wall row); and the step's force field and flags are cleared for
// the next recompute (the forward fluid kernel's job in a normal step; this
// kernel is their last reader).  A warp is one 32-cell row segment; no lane
// leaves early.
__global__ void __launch_bounds__(32 * AB, 4) k_adj_cells(AdjArgs a) {
    const CellPos q = cell_pos(a);
    const Inst& I = *q.I;
    // the lattice's geometry in registers; element offsets within one
    // instance fit 32 bits (lbm_adjoint checks)
    const int nx = I.G.nx, ny = I.G.ny, pitch = I.G.pitch, plane = (int)I.G.plane;
    const bool px = I.G.px != 0, py = I.G.py != 0;
    const int x = q.x, y = q.y;
    const bool in = x < nx && y < ny;
    const int seg = y * I.G.nseg + (x >> 5);
    const int c = y * pitch + x;
    const bool wall = !py && y < ny && (y == 0 || y == ny - 1);  // the same for the whole warp
    const int side = y == 0 ? 2 : 3;
    const float* __restrict__ f = a.f + I.f_off;
    const float* __restrict__ lp0 = a.lam_gp + I.f_off;
    const float* __restrict__ lp1 = lp0 + a.pop_elems;
    bool forced = false;
    float lg[2][9], g0[9];
    if (in) {
        // neighbour columns and rows (periodic wrap; -1 across a wall)
        const int xm = x > 0 ? x - 1 : (px ? nx - 1 : -1), xp = x < nx - 1 ? x + 1 : (px ? 0 : -1);
        const int ym = y > 0 ? y - 1 : (py ? ny - 1 : -1), yp = y < ny - 1 ? y + 1 : (py ? 0 : -1);
        // every load first: the streamed populations (pull from x - e_i),
        // the force, both outputs' lambda(g) of the next level at x + e_i
        int ts[9];
        float lam[2][9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sx = cx(i) == 0 ? x : (cx(i) > 0 ? xm : xp), sy = cy(i) == 0 ? y : (cy(i) > 0 ? ym : yp);
            g0[i] = sx >= 0 && sy >= 0 ? f[i * plane + sy * pitch + sx] : 0.f;
            const int tx = cx(i) == 0 ? x : (cx(i) > 0 ? xp : xm), ty = cy(i) == 0 ? y : (cy(i) > 0 ? yp : ym);
            ts[i] = tx >= 0 && ty >= 0 ? ty * pitch + tx : -1;
            lam[0][i] = ts[i] >= 0 ? lp0[i * plane + ts[i]] : 0.f;
            lam[1][i] = ts[i] >= 0 ? lp1[i * plane + ts[i]] : 0.f;
        }
        forced = a.flags[I.flags_off + seg] != 0;
        float Fx = I.G.gf[0], Fy = I.G.gf[1];
        if (forced) {
            Fx += ForceField<float>::get(a.flb[I.flb_off + c]);
            Fy += ForceField<float>::get(a.flb[I.flb_off + plane + c]);
        }
        // at a y wall node x + e_i, what the Zou-He unknowns owe the known
        // populations (the transposes of k_adj_zh)
        if (!py && (y <= 1 || y >= ny - 2)) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                if (ts[i] < 0) continue;
                const int ty = cy(i) == 0 ? y : (cy(i) > 0 ? yp : ym);
                if (ty != 0 && ty != ny - 1) continue;
                const float* A = a.zh + ((long long)q.inst * 2 + (ty == 0 ? 0 : 1)) * 81;
                for (int u = 0; u < 9; ++u) {
                    const float w = A[u * 9 + i];
                    if (w != 0.f) {
                        lam[0][i] += w * lp0[u * plane + ts[i]];
                        lam[1][i] += w * lp1[u * plane + ts[i]];
                    }
                }
            }
        }
        float g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = g0[i];
        complete_walls<float, float>(f, I.G, x, y, g);
        const CellState cs = cell_state(g, Fx, Fy);
        const float omega = I.G.omegaf;
#pragma unroll
        for (int o = 0; o < 2; ++o) {
#pragma unroll
            for (int i = 0; i < 9; ++i) lg[o][i] = 0.f;
            float lFx, lFy;
            collide_adjoint(cs, omega, lam[o], lg[o], lFx, lFy);
            float* __restrict__ lgo = a.lam_g + o * a.pop_elems + I.f_off;
#pragma unroll
            for (int i = 0; i < 9; ++i) lgo[i * plane + c] = lg[o][i];
            if (forced) {
                a.lam_F[(2 * o) * a.flb_elems + I.flb_off + c] = lFx;
                a.lam_F[(2 * o + 1) * a.flb_elems + I.flb_off + c] = lFy;
            }
        }
    }
    if (wall) {
        using D2 = Dual<float, 2>;
        double s[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
        if (in) {
            D2 v[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) v[i] = D2(g0[i]);
            D2 ux(I.G.uwf[side][0]), uy(I.G.uwf[side][1]);
            ux.d[0] = 1.f;
            uy.d[1] = 1.f;
            if (side == 2) zou_he_edge<0, 1, D2>(v, ux, uy, D2(I.G.gf[0]), D2(I.G.gf[1]));
            else zou_he_edge<0, -1, D2>(v, ux, uy, D2(I.G.gf[0]), D2(I.G.gf[1]));
#pragma unroll
            for (int o = 0; o < 2; ++o)
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    s[o][0] += (double)lg[o][i] * v[i].d[0];
                    s[o][1] += (double)lg[o][i] * v[i].d[1];
                }
        }
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            const double s0 = warp_sum(s[o][0]), s1 = warp_sum(s[o][1]);
            if (threadIdx.x == 0) {
                double* lw = a.lam_wall + ((long long)q.inst * 2 + o) * 8 + side * 2;
                atomicAdd(lw, s0);
                atomicAdd(lw + 1, s1);
            }
        }
    }
    if (forced) {
        a.flb[I.flb_off + c] = 0;
        a.flb[I.flb_off + plane + c] = 0;
    }
    __syncwarp();  // every lane has read the segment's flag
    if (forced && (x & 31) == 0) a.flags[I.flags_off + seg] = 0;
}

// MLS of Eqs. 8-10 at the point (x, y), given relative to some lattice node
// (so that FP32 holds it closely): the 3x3 support around the nearest node
// (lower-left node (i0, j0), relative to the same node), the shape functions
// phi and, if D, the diffuse derivatives dpx, dpy; T is a dual over the
// point's two coordinates, so every output carries its gradient with
// respect to the point
template <bool D>
__device__ __forceinline__ void mls_point(int kind, float x, float y, int& i0, int& j0, F2 phi[9], F2 dpx[9],
                                          F2 dpy[9]) {
    i0 = (int)floorf(x + 0.5f) - 1;
    j0 = (int)floorf(y + 0.5f) - 1;
    F2 px(x), py(y);
    px.d[0] = 1.f;
    py.d[1] = 1.f;
    F2 W[9], DX[9], DY[9];
    F2 a00(0.f), a01(0.f), a02(0.f), a11(0.f), a12(0.f), a22(0.f);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        DX[k] = F2((float)(i0 + k % 3)) - px;
        DY[k] = F2((float)(j0 + k / 3)) - py;
        W[k] = mls_weight<F2>(kind, sqrt(DX[k] * DX[k] + DY[k] * DY[k]) * (1.f / 2.6f));
        const F2 wx = W[k] * DX[k], wy = W[k] * DY[k];
        a00 += W[k];
        a01 += wx;
        a02 += wy;
        a11 += wx * DX[k];
        a12 += wx * DY[k];
        a22 += wy * DY[k];
    }
    const F2 c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
    const F2 id = F2(1.f) / (a00 * c00 + a01 * c01 + a02 * c02);
    const F2 i00 = c00 * id, i01 = c01 * id, i02 = c02 * id;
    F2 i11(0.f), i12(0.f), i22(0.f);
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

// density - 1 and velocity u* at a node from the streamed populations
__device__ __forceinline__ void node_moments(const float* f, const Inst& I, int x, int y, float& drho, float& ux,
                                             float& uy) {
    float g[9];
    pulled(f, I, x, y, g);
    fields_of<float>(g, I.G, drho, ux, uy);
}

template <int K>
__device__ __forceinline__ Dual<float, K> seed(float v, int k) {
    Dual<float, K> r(v);
    r.d[k] = 1.f;
    return r;
}

// cos and sin of an angle (FP64 value) as duals along input k
template <int K>
__device__ __forceinline__ void cos_sin(double th, int k, Dual<float, K>& c, Dual<float, K>& s) {
    double sv, cv;
    sincos(th, &sv, &cv);
    c = Dual<float, K>((float)cv);
    s = Dual<float, K>((float)sv);
    c.d[k] = (float)-sv;
    s.d[k] = (float)cv;
}

// a(q), known with its gradient in the point q = (qx, qy), as a dual over
// the K inputs that q depends on (chain rule through q)
template <int K>
__device__ __forceinline__ Dual<float, K> lift(const F2& a, const Dual<float, K>& qx, const Dual<float, K>& qy) {
    Dual<float, K> r(a.v);
#pragma unroll
    for (int k = 0; k < K; ++k) r.d[k] = a.d[0] * qx.d[k] + a.d[1] * qy.d[k];
    return r;
}

// sum_k w_k v_k as v_ref + sum_k w_k (v_k - v_ref) (the weights sum to 1,
// or to 0 for the diffuse derivatives, whose sum drops v_ref): the
// differences keep FP32 rounding relative to the field's variation
__device__ __forceinline__ F2 fit(const F2 w[9], const float v[9], bool unit) {
    const float r = v[4];
    F2 s(unit ? r : 0.f);
#pragma unroll
    for (int k = 0; k < 9; ++k) s += w[k] * (v[k] - r);
    return s;
}

// k_adj_markers: one thread per marker of the step's markers (the body at
// level n+1, the fluid at level n).  Positions are relative to the node at
// or below the particle's centre; duals over (X, Y, theta, U, V, W of the
// new level, rbx, rby, S) in FP32, the MLS part through its gradient in the
// marker position.
__global__ void __launch_bounds__(64) k_adj_markers(AdjArgs a) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.nmark) return;
    const int p = a.marker_particle[l];
    const int4 pr = a.ptab[p];
    const Inst& I = a.insts[pr.z];
    const DParticle& Q = a.Pn1[p];  // after the update
    const double* mg = a.mgeo + 5 * (long long)l;
    const double bxd = floor(Q.X[0][0]), byd = floor(Q.X[0][1]);
    const F9 X = seed<9>((float)(Q.X[0][0] - bxd), 0), Y = seed<9>((float)(Q.X[0][1] - byd), 1);
    F9 c, s;
    cos_sin<9>(Q.th[0], 2, c, s);
    const F9 U = seed<9>((float)Q.U[0][0], 3), V = seed<9>((float)Q.U[0][1], 4), Wb = seed<9>((float)Q.W[0], 5);
    const F9 rbx = seed<9>((float)mg[0], 6), rby = seed<9>((float)mg[1], 7), S = seed<9>((float)mg[4], 8);
    const F9 rx = c * rbx - s * rby, ry = s * rbx + c * rby;
    const F9 px = X + rx, py = Y + ry;
    int i0, j0;
    F2 phi[9];
    mls_point<false>(a.weight, px.v, py.v, i0, j0, phi, nullptr, nullptr);
    i0 += (int)bxd;
    j0 += (int)byd;
    // node velocities (fixed in this pass) and the force adjoint at the nodes
    float nu[9], nv[9], nr[9], lcx[2][9], lcy[2][9];
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
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            lcx[o][k] = ok ? a.lam_F[(2 * o) * a.flb_elems + I.flb_off + cc] : 0.f;
            lcy[o][k] = ok ? a.lam_F[(2 * o + 1) * a.flb_elems + I.flb_off + cc] : 0.f;
        }
    }
    if (!ok) {
        atomicOr(a.err, ERR_DOMAIN);
        return;
    }
    const F9 Ux = lift<9>(fit(phi, nu, true), px, py), Uy = lift<9>(fit(phi, nv, true), px, py);
    const F9 Fx = (U - Wb * ry) - Ux, Fy = (V + Wb * rx) - Uy;  // Eq. 11
#pragma unroll
    for (int o = 0; o < 2; ++o) {
        // L = sum_k lambda_F(x_k) . (phi_k S F_l) = S (F_x s_x + F_y s_y)  (Eq. 12)
        F2 sx2(0.f), sy2(0.f);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            sx2 += phi[k] * lcx[o][k];
            sy2 += phi[k] * lcy[o][k];
        }
        const F9 sx = lift<9>(sx2, px, py), sy = lift<9>(sy2, px, py);
        const F9 L = S * (Fx * sx + Fy * sy);
        double* lp = a.lamP_new + ((long long)p * 2 + o) * LP_N;
        atomicAdd(lp + LX0, (double)L.d[0]);
        atomicAdd(lp + LY0, (double)L.d[1]);
        atomicAdd(lp + LT0, (double)L.d[2]);
        atomicAdd(lp + LU0, (double)L.d[3]);
        atomicAdd(lp + LV0, (double)L.d[4]);
        atomicAdd(lp + LW0, (double)L.d[5]);
        double* lgm = a.lam_mgeo + ((long long)l * 2 + o) * LG_N;
        lgm[LG_RX] += L.d[6];
        lgm[LG_RY] += L.d[7];
        lgm[LG_S] += L.d[8];
        // node velocities: d L / d u_j = -S phi_j s_x (and s_y)
        float* lg = a.lam_g + o * a.pop_elems;
#pragma unroll 1
        for (int j = 0; j < 9; ++j) {  // (atomics: nothing to wait for; a loop keeps the code small)
            const float cj = -S.v * phi[j].v;
            scatter_moments(lg, I, nxk[j], nyk[j], 0.f, cj * sx.v, cj * sy.v, nr[j], nu[j], nv[j]);
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
// in a real type T over FP32
template <class T>
__device__ __forceinline__ void traction(const T& dr, const T& uxx, const T& uxy, const T& uyx, const T& uyy,
                                         const T& nx, const T& ny, const T& rx, const T& ry, const T& dvx,
                                         const T& dvy, const T& S, float tau, T& Fx, T& Fy, T& M) {
    const T r = T(1.f) + dr;
    const T p = (float)ACS2 * dr + r * (float)APROBE * (dvx * nx + dvy * ny);
    const T mu = r * (float)(ACS2 * (tau - 0.5));
    const T txx = 2.f * mu * uxx, tyy = 2.f * mu * uyy, txy = mu * (uxy + uyx);
    const T tx = txx * nx + txy * ny - p * nx, ty = txy * nx + tyy * ny - p * ny;
    Fx = tx * S;
    Fy = ty * S;
    M = (rx * ty - ry * tx) * S;
}

// k_adj_probes_pre: one thread per marker; the probes of the step (the body at
// level n with its previous level, the fluid at level n).  Positions are
// relative to the node at or below the centre; duals over (X0, Y0, th0,
// th1, U0, V0, U1, V1, W0, W1, rbx, rby, nbx, nby, S) in FP32, the MLS fits
// through their gradients in the probe position.
__global__ void __launch_bounds__(64) k_adj_probes_pre(AdjArgs a) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.nmark) return;
    const int p = a.marker_particle[l];
    const int4 pr = a.ptab[p];
    const Inst& I = a.insts[pr.z];
    const DParticle& P = a.Pn[p];
    const double* mg = a.mgeo + 5 * (long long)l;
    const double bxd = floor(P.X[0][0]), byd = floor(P.X[0][1]);
    const F15 X0 = seed<15>((float)(P.X[0][0] - bxd), 0), Y0 = seed<15>((float)(P.X[0][1] - byd), 1);
    F15 c0, s0, c1, s1;
    cos_sin<15>(P.th[0], 2, c0, s0);
    cos_sin<15>(P.th[1], 3, c1, s1);
    const F15 U0 = seed<15>((float)P.U[0][0], 4), V0 = seed<15>((float)P.U[0][1], 5);
    const F15 U1 = seed<15>((float)P.U[1][0], 6), V1 = seed<15>((float)P.U[1][1], 7);
    const F15 W0 = seed<15>((float)P.W[0], 8), W1 = seed<15>((float)P.W[1], 9);
    const F15 rbx = seed<15>((float)mg[0], 10), rby = seed<15>((float)mg[1], 11);
    const F15 nbx = seed<15>((float)mg[2], 12), nby = seed<15>((float)mg[3], 13), S = seed<15>((float)mg[4], 14);
    const F15 rx = c0 * rbx - s0 * rby, ry = s0 * rbx + c0 * rby;
    const F15 nx = c0 * nbx - s0 * nby, ny = s0 * nbx + c0 * nby;
    const F15 r1x = c1 * rbx - s1 * rby, r1y = s1 * rbx + c1 * rby;
    const F15 qx = X0 + rx + (float)APROBE * nx, qy = Y0 + ry + (float)APROBE * ny;
    int i0, j0;
    F2 phi[9], dpx[9], dpy[9];
    mls_point<true>(a.weight, qx.v, qy.v, i0, j0, phi, dpx, dpy);
    i0 += (int)bxd;
    j0 += (int)byd;
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
    ProbePre& pp = a.ppre[l];
    pp.ok = ok ? 1 : 0;
    if (!ok) {
        atomicOr(a.err, ERR_DOMAIN);
        return;
    }
    const F15 dr = lift<15>(fit(phi, nd, true), qx, qy);
    const F15 uxx = lift<15>(fit(dpx, nu, false), qx, qy), uxy = lift<15>(fit(dpy, nu, false), qx, qy);
    const F15 uyx = lift<15>(fit(dpx, nv, false), qx, qy), uyy = lift<15>(fit(dpy, nv, false), qx, qy);
    // change of the marker's rigid velocity between the two stored levels
    const F15 drx = rx - r1x, dry = ry - r1y, dW = W0 - W1;
    const F15 dvx = (U0 - U1) - (dW * ry + W1 * dry), dvy = (V0 - V1) + (dW * rx + W1 * drx);
    const float tau = (float)I.G.tau;
    F15 Fx, Fy, M;
    traction<F15>(dr, uxx, uxy, uyx, uyy, nx, ny, rx, ry, dvx, dvy, S, tau, Fx, Fy, M);
    // the same with the five fits as the directions (everything else fixed)
    F5 f5[5] = {F5(dr.v), F5(uxx.v), F5(uxy.v), F5(uyx.v), F5(uyy.v)};
#pragma unroll
    for (int q = 0; q < 5; ++q) f5[q].d[q] = 1.f;
    F5 Gx, Gy, GM;
    traction<F5>(f5[0], f5[1], f5[2], f5[3], f5[4], F5(nx.v), F5(ny.v), F5(rx.v), F5(ry.v), F5(dvx.v), F5(dvy.v),
                 F5(S.v), tau, Gx, Gy, GM);
    // what the finishing kernel needs, none of it depending on the adjoint
#pragma unroll
    for (int k = 0; k < 15; ++k) {
        pp.jF[0][k] = Fx.d[k];
        pp.jF[1][k] = Fy.d[k];
        pp.jF[2][k] = M.d[k];
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        pp.jG[0][q] = Gx.d[q];
        pp.jG[1][q] = Gy.d[q];
        pp.jG[2][q] = GM.d[q];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        pp.w[0][k] = phi[k].v;
        pp.w[1][k] = dpx[k].v;
        pp.w[2][k] = dpy[k].v;
        pp.nf[0][k] = nd[k];
        pp.nf[1][k] = nu[k];
        pp.nf[2][k] = nv[k];
        pp.node[0][k] = nxk[k];
        pp.node[1][k] = nyk[k];
    }
}

// k_adj_probes_fin: one thread per marker, after k_adj_rigid: the probe
// Jacobians of k_adj_probes_pre contracted with the adjoint of the force
// and torque -> lambda of the old pose, of the marker geometry and, through
// the fits, of the node density and velocities
__global__ void __launch_bounds__(64) k_adj_probes_fin(AdjArgs a) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.nmark) return;
    const ProbePre& pp = a.ppre[l];
    if (!pp.ok) return;
    const int p = a.marker_particle[l];
    const Inst& I = a.insts[a.ptab[p].z];
#pragma unroll
    for (int o = 0; o < 2; ++o) {
        const double* fm = a.lamFM + ((long long)p * 2 + o) * 3;
        const float f0 = (float)fm[0], f1 = (float)fm[1], f2 = (float)fm[2];
        float L[15];
#pragma unroll
        for (int k = 0; k < 15; ++k) L[k] = f0 * pp.jF[0][k] + f1 * pp.jF[1][k] + f2 * pp.jF[2][k];
        double* lp = a.lamP_old + ((long long)p * 2 + o) * LP_N;
        atomicAdd(lp + LX0, (double)L[0]);
        atomicAdd(lp + LY0, (double)L[1]);
        atomicAdd(lp + LT0, (double)L[2]);
        atomicAdd(lp + LT1, (double)L[3]);
        atomicAdd(lp + LU0, (double)L[4]);
        atomicAdd(lp + LV0, (double)L[5]);
        atomicAdd(lp + LU1, (double)L[6]);
        atomicAdd(lp + LV1, (double)L[7]);
        atomicAdd(lp + LW0, (double)L[8]);
        atomicAdd(lp + LW1, (double)L[9]);
        double* lgm = a.lam_mgeo + ((long long)l * 2 + o) * LG_N;
        lgm[LG_RX] += L[10];
        lgm[LG_RY] += L[11];
        lgm[LG_NX] += L[12];
        lgm[LG_NY] += L[13];
        lgm[LG_S] += L[14];
        // the node values through the fits (linear in them)
        float lf[5];
#pragma unroll
        for (int q = 0; q < 5; ++q) lf[q] = f0 * pp.jG[0][q] + f1 * pp.jG[1][q] + f2 * pp.jG[2][q];
        float* lg = a.lam_g + o * a.pop_elems;
#pragma unroll 1
        for (int kk = 0; kk < 9; ++kk) {  // (atomics: nothing to wait for; a loop keeps the code small)
            const float ldr = pp.w[0][kk] * lf[0];
            const float lu = pp.w[1][kk] * lf[1] + pp.w[2][kk] * lf[2];
            const float lv = pp.w[1][kk] * lf[3] + pp.w[2][kk] * lf[4];
            scatter_moments(lg, I, pp.node[0][kk], pp.node[1][kk], ldr, lu, lv, 1.f + pp.nf[0][kk], pp.nf[1][kk],
                            pp.nf[2][kk]);
        }
    }
}

// the Zou-He completion of wall side `side` (y- = 2, y+ = 3) reversed: the
// three unknowns are affine in the six knowns with constant coefficients
// (the target density is linear in the knowns): A[u][j] = ZH_u(e_j) - ZH_u(0)
// - delta_uj, one 9 x 9 table per wall of each instance
template <int NY>
__device__ __forceinline__ void zh_matrix(const Geo& G, int side, float* A) {
    float z[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) z[i] = 0.f;
    zou_he_edge<0, NY, float>(z, G.uwf[side][0], G.uwf[side][1], G.gf[0], G.gf[1]);
    for (int j = 0; j < 9; ++j) {
        float e[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) e[i] = i == j ? 1.f : 0.f;
        zou_he_edge<0, NY, float>(e, G.uwf[side][0], G.uwf[side][1], G.gf[0], G.gf[1]);
#pragma unroll
        for (int u = 0; u < 9; ++u) A[u * 9 + j] = e[u] - z[u] - (u == j ? 1.f : 0.f);
    }
}

__global__ void k_adj_zh(AdjArgs a, int ninst) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * ninst) return;
    const Geo& G = a.insts[t >> 1].G;
    float* A = a.zh + (long long)t * 81;
    if (t & 1) zh_matrix<-1>(G, 3, A);
    else zh_matrix<1>(G, 2, A);
}

// the initial field f* = f^eq(1, u(y)) of the planar Couette profile
// u(y) = ub + (ut - ub) y / H reversed: lambda of the two wall speeds
// (instances whose blocks carry the Couette flag), with lambda(f*(0)) from
// level 0's lambda(g) (streaming reversed); summed per warp, then per
// block, one atomic per block and value
__global__ void k_adj_init(AdjArgs a) {
    __shared__ double part[AB][4];
    const CellPos q = cell_pos(a);
    if (!(q.flags & 1)) return;  // the same for the whole block
    const Inst& I = *q.I;
    const int x = q.x, y = q.y;
    const bool in = x < I.G.nx && y < I.G.ny;
    // per cell in FP32 (this part's FP64 rate is a small fraction of its
    // FP32 rate); the sums over cells in FP64
    const float ub = I.G.uwf[2][0], ut = I.G.uwf[3][0], t = (float)y / (float)(I.G.ny - 1);
    const float ux = ub + (ut - ub) * t;
    float lam[2][9];
    if (in) lam_post(a, I, q.inst, x, y, lam);
#pragma unroll
    for (int o = 0; o < 2; ++o) {
        float d = 0.f;  // sum_i lambda_i d feq_i / d ux at rho = 1, uy = 0
        if (in) {
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float ex = (float)cx(i);
                d += lam[o][i] * (float)wt(i) * (3.f * ex + 9.f * ex * ex * ux - 3.f * ux);
            }
        }
        const double db = warp_sum((double)(d * (1.f - t))), dt = warp_sum((double)(d * t));
        if (threadIdx.x == 0) {
            part[threadIdx.y][2 * o] = db;
            part[threadIdx.y][2 * o + 1] = dt;
        }
    }
    __syncthreads();
    if (threadIdx.y == 0 && threadIdx.x < 4) {
        double v = 0.0;
        for (int w = 0; w < AB; ++w) v += part[w][threadIdx.x];
        const int o = threadIdx.x >> 1, side = (threadIdx.x & 1) ? 3 : 2;
        atomicAdd(a.lam_wall + ((long long)q.inst * 2 + o) * 8 + side * 2 + 0, v);
    }
}

}  // namespace

int adjoint_block_rows() { return AB; }

cudaError_t launch_adjoint_setup(const AdjArgs& a, int ninst, cudaStream_t s) {
    k_adj_zh<<<(2 * ninst + 63) / 64, 64, 0, s>>>(a, ninst);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_step(const AdjArgs& a, cudaStream_t s) {
    k_adj_cells<<<a.ncblk, dim3(32, AB), 0, s>>>(a);
    if (a.nmark > 0) k_adj_markers<<<(a.nmark + 63) / 64, 64, 0, s>>>(a);
    if (a.np > 0) k_adj_rigid<<<(a.np + 63) / 64, 64, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_probes_pre(const AdjArgs& a, cudaStream_t s) {
    if (a.nmark > 0) k_adj_probes_pre<<<(a.nmark + 63) / 64, 64, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_probes_fin(const AdjArgs& a, cudaStream_t s) {
    if (a.nmark > 0) k_adj_probes_fin<<<(a.nmark + 63) / 64, 64, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_init(const AdjArgs& a, cudaStream_t s) {
    k_adj_init<<<a.ncblk, dim3(32, AB), 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbib
