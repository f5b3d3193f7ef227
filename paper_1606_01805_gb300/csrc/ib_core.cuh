// ib_core.cuh -- the immersed-boundary work of a step as device functions:
// probe stress, force/torque block sums and the rigid-body update of one
// marker block (probe_block), MLS interpolation, direct forcing and
// spreading records of one marker block (marker_block), and one spreading
// tile (spread_tile).  The separate IB kernels (particles.cu) and the fused
// persistent step (step_fused.cu) are built from them.
//
// The markers of all particles are cut into blocks of MB = 8 (one warp per
// block, four lanes per marker), so the FP64 work spreads over many SMs and
// each lane's dependency chain covers only 2-3 of the 9 support nodes.
// probe_block: probe 1.2 dx along the outward normal of each marker of the
//   body at its latest level, MLS fit of density and velocity there,
//   surface traction; warp sums of force and torque per block (Eqs. 13-14,
//   FP64).  The last block of a particle to finish (a completion counter;
//   nothing waits) adds the block sums (fixed lane assignment and shuffle
//   tree, so deterministic) and applies the two-level rigid-body update
//   (Eqs. 15-16, FP64), once per particle, into the other state buffer, with
//   the new pose in the compute type C (PoseC) beside it.
// marker_block: the markers at the new level: MLS interpolation (Eq. 8),
//   direct-forcing force (Eq. 11), the per-marker spreading record
//   S_l phi_k F_l of Eq. 12 and the particle's support box.
// spread_tile (one CTA per 32 x TY tile of a particle's box): gathers, cell
//   by cell and in marker order, the records whose support covers the cell,
//   then adds the particle's sum into f_lb (the only atomic: one add per
//   cell and particle, contended only where particles overlap) and flags the
//   32-cell row segments the fluid kernel must read.
// Marker and probe geometry runs in C, relative to the node at or below
// the particle's centre; FP64 (the type R) is kept for the 3x3 MLS solve,
// the force/torque sums and the rigid-body update.
// Each function is a template on the population storage type S, the compute
// type C and the particle real type R: (double, double, double) in FP64,
// (float or half, float, double) in FP32 / FP16, and in the tangent mode
// (TF, TF, TD), where every value carries its derivatives along K input
// directions and the same code propagates them.
#pragma once

#include <climits>

#include "lbib_device.cuh"

namespace lbib {

namespace {


constexpr int TX = 32;  // spreading tile width (cells; one thread per cell); the height is a parameter
constexpr double CS2 = 1.0 / 3.0;
constexpr double PROBE = 1.2;

__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// load through L2 of a value another block of the running kernel wrote
__device__ __forceinline__ double ldcg_r(const double* p) { return __ldcg(p); }
__device__ __forceinline__ TD ldcg_r(const TD* p) {
    TD r;
    r.v = __ldcg(&p->v);
#pragma unroll
    for (int k = 0; k < KT; ++k) r.d[k] = __ldcg(&p->d[k]);
    return r;
}

// 1 / x, correctly rounded (with its derivatives for a dual)
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }
__device__ __forceinline__ TD recip(const TD& x) { return TD(1.0) / x; }

constexpr int LPM = 4;  // lanes per marker: lane q gathers support nodes q, q + 4, q + 8

template <class T>
__device__ __forceinline__ T quad_sum(T v) {  // sum over the 4 lanes of a marker
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return v;
}

// The MLS operator of Eqs. 8-10 split over the 4 lanes of a marker: lane q
// holds support nodes k = q, q + 4, q + 8 (k < 9) of the 3x3 block around
// the nearest node of the point.  The point is given in C relative to a
// reference node (ix, iy) of the particle (lx, ly: under the particle's
// size plus two cells).  Weights and the moment matrix A = sum W p p^T in
// precision C (reduced across the lanes); A is inverted (adjugate) in the
// particle type R.  On return the lane has, for its nodes, the first (phi)
// and, if D, second/third rows of A^-1 [W p].
template <bool D, class C, class R>
struct QuadMLS {
    int i0, j0;      // lower-left node of the support
    int li, lj;      // the same relative to the reference node
    int nk;          // nodes held by this lane (3 or 2)
    int qd;          // the lane's place in its quad
    int kk[3];
    C phi[3], dpx[3], dpy[3];

    // support of (ix + lx, iy + ly) and the nodes of lane q; the choice of
    // support is piecewise constant in the position and carries no derivative
    __device__ __forceinline__ void support(int ix, int iy, const C& lx, const C& ly, int q) {
        li = (int)floor_value(lx + C(0.5)) - 1;
        lj = (int)floor_value(ly + C(0.5)) - 1;
        i0 = ix + li;
        j0 = iy + lj;
        nk = q == 0 ? 3 : 2;
        qd = q;
#pragma unroll
        for (int j = 0; j < 3; ++j) kk[j] = q + 4 * j;
    }

    // weights and moment matrix in precision C, the 3x3 solve in R
    // (after support(), the same lx, ly)
    __device__ __forceinline__ void build(int kind, const C& lx, const C& ly, bool active) {
        C W[3], DX[3], DY[3];
        C b00 = C(0), b01 = C(0), b02 = C(0), b11 = C(0), b12 = C(0), b22 = C(0);
        // offsets from the support's lower-left node (a small integer
        // minus the point: no rounding beyond that of lx, ly)
        const C ox = C(li) - lx, oy = C(lj) - ly;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int k = kk[j];
            W[j] = C(0);
            DX[j] = C(0);
            DY[j] = C(0);
            if (j < nk && active) {
                const C dxw = ox + C(k % 3), dyw = oy + C(k / 3);
                W[j] = mls_weight<C>(kind, sqrt(dxw * dxw + dyw * dyw) * C(1.0 / 2.6));
                DX[j] = dxw;
                DY[j] = dyw;
                const C w = W[j], wx = w * dxw, wy = w * dyw;
                b00 += w;
                b01 += wx;
                b02 += wy;
                b11 += wx * dxw;
                b12 += wx * dyw;
                b22 += wy * dyw;
            }
        }
        R a00 = (R)quad_sum(b00), a01 = (R)quad_sum(b01), a02 = (R)quad_sum(b02);
        R a11 = (R)quad_sum(b11), a12 = (R)quad_sum(b12), a22 = (R)quad_sum(b22);
        if (!active) a00 = a11 = a22 = R(1.0);  // keep idle lanes finite
        // The adjugate split over the marker's lanes (the FP64 unit takes a
        // warp instruction whatever its lanes do): lane q forms cofactor
        // c0q of the first row and, if D, c11 / c12 / c22 (q = 0 / 1 / 2;
        // lane 3 repeats lane 0); the determinant and the rows of A^-1 then
        // come from the quad by shuffles.
        const int base = (threadIdx.x & 31) & ~(LPM - 1);
        const R x = qd == 1 ? a02 : qd == 2 ? a01 : a11, y = qd == 1 || qd == 2 ? a12 : a22;
        const R z = qd == 1 ? a01 : qd == 2 ? a02 : a12, w = qd == 1 ? a22 : qd == 2 ? a11 : a12;
        const R cf = x * y - z * w;  // c00, c01, c02
        const R c00 = __shfl_sync(0xffffffffu, cf, base), c01 = __shfl_sync(0xffffffffu, cf, base + 1);
        const R c02 = __shfl_sync(0xffffffffu, cf, base + 2);
        const R id = recip(a00 * c00 + a01 * c01 + a02 * c02);
        const C ir = (C)(cf * id);
        const C i00 = __shfl_sync(0xffffffffu, ir, base), i01 = __shfl_sync(0xffffffffu, ir, base + 1);
        const C i02 = __shfl_sync(0xffffffffu, ir, base + 2);
        C i11 = C(0), i12 = C(0), i22 = C(0);
        if (D) {
            const R xs = qd == 1 ? a01 : a00, ys = qd == 1 ? a02 : qd == 2 ? a11 : a22;
            const R zs = qd == 1 ? a00 : qd == 2 ? a01 : a02, ws = qd == 1 ? a12 : qd == 2 ? a01 : a02;
            const C is = (C)((xs * ys - zs * ws) * id);  // c11, c12, c22 over det
            i11 = __shfl_sync(0xffffffffu, is, base);
            i12 = __shfl_sync(0xffffffffu, is, base + 1);
            i22 = __shfl_sync(0xffffffffu, is, base + 2);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            phi[j] = W[j] * (i00 + i01 * DX[j] + i02 * DY[j]);
            if (D) {
                dpx[j] = W[j] * (i01 + i11 * DX[j] + i12 * DY[j]);
                dpy[j] = W[j] * (i02 + i12 * DX[j] + i22 * DY[j]);
            }
        }
    }
};

// Sum of the block force/torque sums of particle P and its rigid-body update
// (Eqs. 15-16), computed identically by every lane.
template <class R>
struct Body {
    R X, Y, T, U, V, W, c, s, F0, F1, M;
};
template <class R>
__device__ __forceinline__ Body<R> update_body(const DParticleT<R>* P, const R* partial,
                                               const double gravity[2], int lane) {
    // lane l sums component j = l % 4 (< 3) of the blocks g, g + 8, g + 16,
    // ... (g = l / 4) in that order, eight loads issued together (L2: other
    // blocks wrote them); a butterfly over the 8 groups then leaves every
    // group with the totals, so one FP64 add per block and tree level
    // serves all three components
    const int j = lane & 3, g = lane >> 2;
    const int b0 = P->b0, nb = P->nblk;
    R acc = R(0.0);
    for (int base = 0; base < nb; base += 64) {
        R q[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int b = base + 8 * u + g;
            q[u] = j < 3 && b < nb ? ldcg_r(partial + 3 * (long long)(b0 + b) + j) : R(0.0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (base + 8 * u + g < nb) acc += q[u];
    }
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const R F0 = __shfl_sync(0xffffffffu, acc, 0), F1 = __shfl_sync(0xffffffffu, acc, 1);
    const R Mt = __shfl_sync(0xffffffffu, acc, 2);
    const R th0 = P->th[0];
    const R buoy = (P->rho_s - 1.0) * P->area;
    // lane c = 0, 1, 2 integrates x, y, the angle (the FP64 unit takes a
    // warp instruction whatever its lanes do); the others repeat lane 0
    const int c = lane < 3 ? lane : 0;
    const R fc = c == 0 ? F0 : c == 1 ? F1 : Mt;
    const R gc = R(c == 1 ? gravity[1] : gravity[0]);
    const R inv = c == 2 ? P->inv_inertia : P->inv_mass;
    const R fg = fc + buoy * gc;
    const R ac = (c == 2 ? fc : fg) * inv;  // a_x, a_y, alpha
    const R v0 = c == 0 ? P->U[0][0] : c == 1 ? P->U[0][1] : P->W[0];
    const R p0 = c == 0 ? P->X[0][0] : c == 1 ? P->X[0][1] : th0;
    R vn, pn;
    if (P->nupd == 0) {  // one stored level: u1 = u0 + a, x1 = x0 + u1
        vn = v0 + ac;
        pn = p0 + vn;
    } else {  // Eqs. 15-16 and the same two-level form for position and angle
        const double k = 2.0 / 3.0;
        const R v1 = c == 0 ? P->U[1][0] : c == 1 ? P->U[1][1] : P->W[1];
        const R p1 = c == 0 ? P->X[1][0] : c == 1 ? P->X[1][1] : P->th[1];
        vn = k * (2.0 * v0 - 0.5 * v1 + ac);
        pn = k * (2.0 * p0 - 0.5 * p1 + vn);
    }
    Body<R> B;
    B.U = __shfl_sync(0xffffffffu, vn, 0);
    B.V = __shfl_sync(0xffffffffu, vn, 1);
    B.W = __shfl_sync(0xffffffffu, vn, 2);
    B.X = __shfl_sync(0xffffffffu, pn, 0);
    B.Y = __shfl_sync(0xffffffffu, pn, 1);
    B.T = __shfl_sync(0xffffffffu, pn, 2);
    // (cos, sin) of the new angle: the stored pair of the old one turned by
    // the increment d, with cos d and sin d from their Taylor series: for
    // |d| < 1e-4 to d^4 / d^3 (the next terms below 1.4e-27 and 8.3e-19 |d|),
    // for |d| < 1e-2 to d^8 / d^9 (below 1e-26), both far under half an
    // FP64 ulp; a larger increment takes sincos
    const R d = B.T - th0;
    const double ad = fabs(value_of(d));
    if (ad < 1e-4) {
        const R d2 = d * d;
        const R cd = 1.0 + d2 * (-1.0 / 2 + d2 * (1.0 / 24));
        const R sd = d + (d * d2) * (-1.0 / 6);
        const R c0 = P->cs[0][0], s0 = P->cs[0][1];
        B.c = c0 * cd - s0 * sd;
        B.s = s0 * cd + c0 * sd;
    } else if (ad < 1e-2) {
        const R d2 = d * d;
        const R cd = 1.0 + d2 * (-1.0 / 2 + d2 * (1.0 / 24 + d2 * (-1.0 / 720 + d2 * (1.0 / 40320))));
        const R sd = d * (1.0 + d2 * (-1.0 / 6 + d2 * (1.0 / 120 + d2 * (-1.0 / 5040 + d2 * (1.0 / 362880)))));
        const R c0 = P->cs[0][0], s0 = P->cs[0][1];
        B.c = c0 * cd - s0 * sd;
        B.s = s0 * cd + c0 * sd;
    } else {
        sincos(B.T, &B.s, &B.c);
    }
    B.F0 = F0;
    B.F1 = F1;
    B.M = Mt;
    return B;
}

// The pose of the updated body B in C (PoseC), over the lanes: lane k
// forms entry k as hi - lo in R (lo: the node at or below the centre, or
// the previous level's value for a change) and converts it once, so the
// whole conversion is a few FP64 warp instructions.
template <class C, class R>
__device__ __forceinline__ void publish_pose(PoseC<C>* out, const Body<R>& B, const DParticleT<R>* P,
                                             int lane) {
    const R zero = R(0.0);
    const R hi[PC_N] = {B.X, B.Y, B.c, B.s, B.U, B.V, B.W, B.U, B.V, B.W, P->W[0], B.c, B.s};
    const R lo[PC_N] = {zero, zero, zero, zero, zero, zero, zero,
                        P->U[0][0], P->U[0][1], P->W[0], zero, P->cs[0][0], P->cs[0][1]};
    R h = zero, l = zero;
#pragma unroll
    for (int k = 0; k < PC_N; ++k)
        if (lane == k) {
            h = hi[k];
            l = lo[k];
        }
    const double fl = floor(value_of(h));  // used by lanes PC_XF, PC_YF
    if (lane == PC_XF || lane == PC_YF) {
        l = R(fl);
        (&out->ix)[lane - PC_XF] = (int)fl;
    }
    if (lane < PC_N) out->v[lane] = (C)(h - l);
}

// The lattice of a marker block or particle: for a context of one lattice
// its descriptor travels in the kernel parameters (ONE), else it is loaded.
template <bool ONE, class A>
__device__ __forceinline__ const Inst& inst_of(const A& a, int w) {
    if (ONE) return a.one;
    return a.insts[w];
}

// Probe stress of marker block `blk` (one warp, 4 lanes per marker), its
// block sums of force and torque, and, in the particle's last block to
// finish, the rigid-body update.  FUSED: inside the persistent step (no
// programmatic-launch waits; the update then releases *upd = 1).
template <class S, class C, class R, bool ONE, bool FUSED>
__device__ __forceinline__ void probe_block(const ParticleArgs& a, int blk, unsigned* upd) {
    const int4 bk = a.nblk_inline ? a.blk_inline[blk] : a.blk[blk];
    const DParticleT<R>* P = static_cast<const DParticleT<R>*>(a.pin) + bk.x;
    const Inst& I = inst_of<ONE>(a, bk.w);
    const Geo& G = I.G;
    const Geo* Gg = &a.insts[ONE ? 0 : bk.w].G;
    const S* __restrict__ f = static_cast<const S*>(a.f) + I.f_off;
    R* partial = static_cast<R*>(a.partial);
    const int lane = threadIdx.x & 31, q = lane & (LPM - 1);
    const int ml = lane / LPM, m = bk.y + ml;  // marker (absolute index)
    const bool active = ml < bk.z;
    unsigned err = 0;
    // body at its latest level (written by this kernel a step ago), in C
    const PoseC<C>& pc = static_cast<const PoseC<C>*>(a.pcin)[bk.x];
    MGeo<C> g{C(0), C(0), C(1), C(0)};
    if (active) g = static_cast<const MGeo<C>*>(a.mg)[m];
    const C c0 = pc.v[PC_C], s0 = pc.v[PC_S];
    const C rx = c0 * g.rx - s0 * g.ry, ry = s0 * g.rx + c0 * g.ry;  // x_l - X_c
    const C nx = c0 * g.nx - s0 * g.ny, ny = s0 * g.nx + c0 * g.ny;
    // the probe x_l + 1.2 n_l relative to the node (ix, iy)
    const C lx = pc.v[PC_XF] + rx + C(PROBE) * nx, ly = pc.v[PC_YF] + ry + C(PROBE) * ny;
    QuadMLS<true, C, R> M;
    M.support(pc.ix, pc.iy, lx, ly, q);
    if (!FUSED) {
        pdl_wait();  // the populations come from the fluid kernel before this one
        pdl_trigger();
    }
    if (lane == 0 && bk.y == P->m0)  // the particle's first block resets its box
        a.boxes[bk.x] = make_int4(INT_MAX, INT_MAX, INT_MIN, INT_MIN);
    // node fields first (their loads overlap the FP64 work of the solve);
    // the density as rho - 1, whose fit at the probe then needs no
    // cancellation against 1 (partition of unity: rho_P - 1 = sum phi (rho - 1))
    C rk[3], uk[3], vk[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        rk[j] = C(0); uk[j] = C(0); vk[j] = C(0);
        if (j < M.nk && active) {
            const int k = M.kk[j];
            if (!node_fields<S, C>(f, G, Gg, M.i0 + k % 3, M.j0 + k / 3, rk[j], uk[j], vk[j])) {
                err |= ERR_DOMAIN;
                rk[j] = C(0); uk[j] = C(0); vk[j] = C(0);
            }
        }
    }
    M.build(a.weight, lx, ly, active);
    // MLS fit of rho - 1 and grad u at the probe (Section 2.3)
    C dr = C(0), uxx = C(0), uxy = C(0), uyx = C(0), uyy = C(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        if (j < M.nk && active) {
            dr += M.phi[j] * rk[j];
            uxx += M.dpx[j] * uk[j];
            uxy += M.dpy[j] * uk[j];
            uyx += M.dpx[j] * vk[j];
            uyy += M.dpy[j] * vk[j];
        }
    }
    dr = quad_sum(dr); uxx = quad_sum(uxx); uxy = quad_sum(uxy); uyx = quad_sum(uyx); uyy = quad_sum(uyy);
    const C r = C(1) + dr;  // rho_P
    C cF[3] = {C(0), C(0), C(0)};  // this marker's force and torque (quad leader)
    if (active && q == 0) {
        // change of the marker's rigid velocity u + omega z x r between the
        // two stored levels, from the changes of u, omega and r (r - r1 =
        // (R(th) - R(th1)) r_b), free of cancellation
        const C dc = pc.v[PC_DC], ds = pc.v[PC_DS], dw = pc.v[PC_DW], w1 = pc.v[PC_W1];
        const C drx = dc * g.rx - ds * g.ry, dry = ds * g.rx + dc * g.ry;
        const C dvx = pc.v[PC_DU] - (dw * ry + w1 * dry);
        const C dvy = pc.v[PC_DV] + (dw * rx + w1 * drx);
        const C p = C(CS2) * dr + r * C(PROBE) * (dvx * nx + dvy * ny);
        const C mu = r * C(CS2 * (G.tau - 0.5));
        const C txx = C(2) * mu * uxx, tyy = C(2) * mu * uyy, txy = mu * (uxy + uyx);
        const C tx = txx * nx + txy * ny - p * nx;
        const C ty = txy * nx + tyy * ny - p * ny;
        const C Sl = static_cast<const C*>(a.S)[m];
        // the marker's force and torque in C, their sums (Eqs. 13-14) in R
        cF[0] = tx * Sl;
        cF[1] = ty * Sl;
        cF[2] = (rx * ty - ry * tx) * Sl;
    }
    // lane q < 3 of each quad takes component q of its leader's values, so
    // one FP64 conversion and one FP64 add per tree level sum all three
    // (the same tree over the 8 quads for each component: lanes 0, 1, 2
    // end with the block's F_x, F_y, M)
    C mine = cF[0];
#pragma unroll
    for (int j = 1; j < 3; ++j) {
        const C v = __shfl_sync(0xffffffffu, cF[j], lane & ~(LPM - 1));
        if (q == j) mine = v;
    }
    R acc = q < 3 ? (R)mine : R(0.0);
#pragma unroll
    for (int o = 16; o >= LPM; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    const R Fy = __shfl_sync(0xffffffffu, acc, 1), Mz = __shfl_sync(0xffffffffu, acc, 2);
    if (err) atomicOr(a.err, err);
    unsigned done = 0;
    if (lane == 0) {
        R* part = partial + 3 * (long long)blk;
        part[0] = acc;
        part[1] = Fy;
        part[2] = Mz;
        __threadfence();  // the block sums are visible before the count says so
        done = atomicAdd(a.count + bk.x, 1u);
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    if (done != (unsigned)P->nblk - 1) return;  // not the last block (whole warp)
    __threadfence();
    const Body<R> B = update_body<R>(P, partial, G.grav, lane);
    publish_pose<C, R>(static_cast<PoseC<C>*>(a.pcout) + bk.x, B, P, lane);
    if (lane == 0) {
        DParticleT<R>* Q = static_cast<DParticleT<R>*>(a.pout) + bk.x;
        *Q = *P;
        Q->X[1][0] = P->X[0][0]; Q->X[1][1] = P->X[0][1]; Q->th[1] = P->th[0];
        Q->U[1][0] = P->U[0][0]; Q->U[1][1] = P->U[0][1]; Q->W[1] = P->W[0];
        Q->cs[1][0] = P->cs[0][0]; Q->cs[1][1] = P->cs[0][1];
        Q->X[0][0] = B.X; Q->X[0][1] = B.Y; Q->th[0] = B.T;
        Q->U[0][0] = B.U; Q->U[0][1] = B.V; Q->W[0] = B.W;
        Q->cs[0][0] = B.c; Q->cs[0][1] = B.s;
        Q->F[0] = B.F0; Q->F[1] = B.F1; Q->M = B.M;
        Q->wsum = P->wsum + B.W;
        Q->nupd = P->nupd + 1;
        if (!isfinite(B.X) || !isfinite(B.Y) || !isfinite(B.T) || !isfinite(B.U) || !isfinite(B.W))
            atomicOr(a.err, ERR_NONFINITE);
        a.count[bk.x] = 0;
    }
    if (FUSED) {  // the new pose and state are visible before the flag says so
        __syncwarp();
        __threadfence();
        if (lane == 0) atomicExch(upd + bk.x, 1u);
    }
}

// MLS interpolation, direct forcing and spreading records of marker block
// `blk` (one warp), and its part of the particle's support box.  FUSED: the
// caller waited for the particle's update; the block then counts itself
// done in *mdone (per particle) after its records and box are visible.
template <class S, class C, class R, bool ONE, bool FUSED>
__device__ __forceinline__ void marker_block(const ParticleArgs& a, int blk, unsigned* mdone) {
    const int4 bk = a.nblk_inline ? a.blk_inline[blk] : a.blk[blk];
    const PoseC<C>* Q = static_cast<const PoseC<C>*>(a.pcout) + bk.x;  // after the update, in C
    const Inst& I = inst_of<ONE>(a, bk.w);
    const Geo& G = I.G;
    const Geo* Gg = &a.insts[ONE ? 0 : bk.w].G;
    const S* __restrict__ f = static_cast<const S*>(a.f) + I.f_off;
    Rec<C>* recs = static_cast<Rec<C>*>(a.recs);
    const int lane = threadIdx.x & 31, q = lane & (LPM - 1);
    const int ml = lane / LPM, m = bk.y + ml;  // marker (absolute index)
    const bool active = ml < bk.z;
    unsigned err = 0;
    MGeo<C> g{C(0), C(0), C(1), C(0)};
    if (active) g = static_cast<const MGeo<C>*>(a.mg)[m];
    if (!FUSED) {
        pdl_wait();  // the updated body comes from the probe kernel
        pdl_trigger();
    }
    const C cn = Q->v[PC_C], sn = Q->v[PC_S];
    const C BU = Q->v[PC_U], BV = Q->v[PC_V], BW = Q->v[PC_W];
    const C rx = cn * g.rx - sn * g.ry, ry = sn * g.rx + cn * g.ry;
    const C lx = Q->v[PC_XF] + rx, ly = Q->v[PC_YF] + ry;  // relative to (ix, iy)
    QuadMLS<false, C, R> M;
    M.support(Q->ix, Q->iy, lx, ly, q);
    C uk[3], vk[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        uk[j] = C(0); vk[j] = C(0);
        if (j < M.nk && active) {
            const int k = M.kk[j];
            C rk;
            if (!node_fields<S, C>(f, G, Gg, M.i0 + k % 3, M.j0 + k / 3, rk, uk[j], vk[j])) {
                err |= ERR_DOMAIN;
                uk[j] = C(0); vk[j] = C(0);
            }
        }
    }
    M.build(a.weight, lx, ly, active);
    C ux = C(0), uy = C(0);
#pragma unroll
    for (int j = 0; j < 3; ++j)
        if (j < M.nk && active) {
            ux += M.phi[j] * uk[j];
            uy += M.phi[j] * vk[j];
        }
    ux = quad_sum(ux);  // Eq. 8: U(x_l)
    uy = quad_sum(uy);
    int bx0 = INT_MAX, by0 = INT_MAX, bx1 = INT_MIN, by1 = INT_MIN;
    if (active) {
        // Eq. 11 with dt = 1, times the arc length c_l = S_l of Eq. 12
        const C Sl = static_cast<const C*>(a.S)[m];
        const C sx = Sl * ((BU - BW * ry) - ux);
        const C sy = Sl * ((BV + BW * rx) - uy);
        if constexpr (!FUSED && ForceField<C>::FIXED) {
            // Eq. 12 added straight into the fixed-point force field: each
            // lane its support nodes (no records, no spreading kernel)
            using FF = ForceField<C>;
            ForceT<C>* flb = static_cast<ForceT<C>*>(a.flb) + I.flb_off;
            uint8_t* flags = a.flags + I.flags_off;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j < M.nk) {
                    const int k = M.kk[j];
                    int gx = M.i0 + k % 3, gy = M.j0 + k / 3;
                    bool in = true;
                    if (gx < 0 || gx >= G.nx) {
                        if (G.px) gx = ((gx % G.nx) + G.nx) % G.nx;
                        else in = false;
                    }
                    if (gy < 0 || gy >= G.ny) {
                        if (G.py) gy = ((gy % G.ny) + G.ny) % G.ny;
                        else in = false;
                    }
                    if (in) {
                        const long long c = (long long)gy * G.pitch + gx;
                        FF::add(flb + c, FF::fix(M.phi[j] * sx));
                        FF::add(flb + G.plane + c, FF::fix(M.phi[j] * sy));
                        flags[gy * G.nseg + (gx >> 5)] = 1;
                    }
                }
        } else {
            Rec<C>* rc = recs + m;
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (j < M.nk) {
                    rc->cx[M.kk[j]] = M.phi[j] * sx;
                    rc->cy[M.kk[j]] = M.phi[j] * sy;
                }
            if (q == 0) {
                rc->i0 = M.i0;
                rc->j0 = M.j0;
            }
        }
        if (q == 0) {
            bx0 = M.i0;
            by0 = M.j0;
            bx1 = M.i0 + 2;
            by1 = M.j0 + 2;
        }
    }
    if (err) atomicOr(a.err, err);
    bx0 = warp_min(bx0);
    by0 = warp_min(by0);
    bx1 = warp_max(bx1);
    by1 = warp_max(by1);
    if (lane == 0) {
        int4* b = a.boxes + bk.x;
        atomicMin(&b->x, bx0);
        atomicMin(&b->y, by0);
        atomicMax(&b->z, bx1);
        atomicMax(&b->w, by1);
    }
    if (FUSED) {  // records and box visible before the count says so
        __syncwarp();
        __threadfence();
        if (lane == 0) atomicAdd(mdone + bk.x, 1u);
    }
}

// records examined per round of a spreading tile of 32 x TYt cells: as
// many as fit the list (48 KB less the warp counts), at most two per thread
template <class C, int TYt>
constexpr int spread_cap() {
    const int c = (int)((48 * 1024 - 256) / sizeof(Rec<C>));
    return c < 2 * TX * TYt ? c : 2 * TX * TYt;
}

// shared memory of a spreading tile: the compacted records and the warps' counts
template <class C, int TYt>
struct SpreadSmem {
    Rec<C> list[spread_cap<C, TYt>()];
    int wcount[2][TX * TYt / 32];
};

// Spreading tile `tile` (32 x TYt cells, one thread each, the CTA) of
// particle p's support box: gathers, cell by cell and in marker order, the
// records that cover the cell and adds the particle's sum into f_lb with one
// atomic per cell, flagging the 32-cell row segment.  tiles: the tile bound
// of the particle's box for this tile height.  FUSED: the caller waited for
// the particle's marker blocks (no programmatic-launch waits).
template <class C, class R, bool ONE, bool FUSED, int TYt>
__device__ __forceinline__ void spread_tile(const SpreadArgs& a, int tile, int p, int tiles,
                                            SpreadSmem<C, TYt>& sm) {
    constexpr int CAP = spread_cap<C, TYt>();
    constexpr int TY = TYt;
    // the particle's markers and lattice (fixed when it was added)
    const int4 pr = a.np_inline ? a.part_inline[p] : a.ptab[p];
    const int m0 = pr.x, nm = pr.y;
    if (tile >= tiles) return;  // beyond this particle's box (whole CTA)
    const Inst& I = inst_of<ONE>(a, pr.z);
    const Geo& G = I.G;
    const Rec<C>* recs = static_cast<const Rec<C>*>(a.recs);
    using FF = ForceField<C>;
    ForceT<C>* flb = static_cast<ForceT<C>*>(a.flb) + I.flb_off;
    uint8_t* flags = a.flags + I.flags_off;
    constexpr int NW = TX * TY / 32;
    Rec<C>* list = sm.list;
    auto& wcount = sm.wcount;
    if (!FUSED) {
        pdl_wait();  // boxes and records come from the marker kernel
        pdl_trigger();
    }
    const int4 box = a.boxes[p];
    if (box.x > box.z) return;
    const int ntx = (box.z - box.x + TX) / TX, nty = (box.w - box.y + TY) / TY;
    if (tile == 0 && threadIdx.x == 0 && ntx * nty > tiles) atomicOr(a.err, ERR_DOMAIN);
    if (tile >= ntx * nty) return;  // whole CTA
    const int x0 = box.x + (tile % ntx) * TX, y0 = box.y + (tile / ntx) * TY;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int cxl = x0 + t % TX, cyl = y0 + t / TX;  // this thread's (unwrapped) cell
    ForceT<C> ax = ForceT<C>(0), ay = ForceT<C>(0);  // (fixed point: each contribution rounded, then summed)
    bool touched = false;
    for (int base = 0; base < nm; base += CAP) {
        // thread t examines records base + t (slot 0) and base + TX TY + t
        // (slot 1); the relevant ones are compacted in marker order: all of
        // slot 0 in thread order, then all of slot 1
        bool rel[2] = {false, false};
        Rec<C> r[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = h * TX * TY + t, l = base + k;
            if (k < CAP && l < nm) {
                // the support origin first (one 16-byte load, the record's
                // first sector); the whole record only if it is relevant
                const int4 head = *reinterpret_cast<const int4*>(recs + m0 + l);
                rel[h] = head.x <= x0 + TX - 1 && head.x + 2 >= x0 && head.y <= y0 + TY - 1 && head.y + 2 >= y0;
                if (rel[h]) r[h] = recs[m0 + l];
            }
        }
        const unsigned bal0 = __ballot_sync(0xffffffffu, rel[0]), bal1 = __ballot_sync(0xffffffffu, rel[1]);
        if (lane == 0) {
            wcount[0][wid] = __popc(bal0);
            wcount[1][wid] = __popc(bal1);
        }
        __syncthreads();
        int off0 = 0, off1 = 0, total0 = 0, total1 = 0;
        for (int w = 0; w < NW; ++w) {
            off0 += (w < wid) ? wcount[0][w] : 0;
            off1 += (w < wid) ? wcount[1][w] : 0;
            total0 += wcount[0][w];
            total1 += wcount[1][w];
        }
        const unsigned below = (1u << lane) - 1u;
        if (rel[0]) list[off0 + __popc(bal0 & below)] = r[0];
        if (rel[1]) list[total0 + off1 + __popc(bal1 & below)] = r[1];
        const int total = total0 + total1;
        __syncthreads();
        // warp wid holds tile row cyl: it picks, 32 at a time, the records
        // whose support has that row (one ballot), then every lane adds
        // those that cover its cell, in list (marker) order
        for (int b0 = 0; b0 < total; b0 += 32) {
            const int m = b0 + lane;
            bool row = false;
            if (m < total) {
                const int db = cyl - list[m].j0;
                row = db >= 0 && db < 3;
            }
            unsigned bits = __ballot_sync(0xffffffffu, row);
            while (bits) {
                const Rec<C>& rc = list[b0 + __ffs(bits) - 1];
                bits &= bits - 1u;
                const int da = cxl - rc.i0, db = cyl - rc.j0;
                if (da >= 0 && da < 3) {
                    if constexpr (FF::FIXED) {
                        ax += FF::fix(rc.cx[db * 3 + da]);
                        ay += FF::fix(rc.cy[db * 3 + da]);
                    } else {
                        ax += rc.cx[db * 3 + da];
                        ay += rc.cy[db * 3 + da];
                    }
                    touched = true;
                }
            }
        }
        __syncthreads();
    }
    if (!touched || cxl > box.z || cyl > box.w) return;
    int gx = cxl, gy = cyl;
    if (gx < 0 || gx >= G.nx) {
        if (!G.px) return;
        gx = ((gx % G.nx) + G.nx) % G.nx;
    }
    if (gy < 0 || gy >= G.ny) {
        if (!G.py) return;
        gy = ((gy % G.ny) + G.ny) % G.ny;
    }
    const long long c = (long long)gy * G.pitch + gx;
    if constexpr (FF::FIXED) {
        FF::add(flb + c, ax);
        FF::add(flb + G.plane + c, ay);
    } else {
        atomicAdd(flb + c, ax);
        atomicAdd(flb + G.plane + c, ay);
    }
    flags[gy * G.nseg + (gx >> 5)] = 1;
}

}  // namespace

}  // namespace lbib
