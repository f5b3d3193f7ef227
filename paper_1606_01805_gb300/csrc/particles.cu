// particles.cu -- immersed-boundary kernels of the LB-IB step.
//
// k_particles (one CTA per particle, FP64):
//   probes 1.2 dx along the outward normals of the body at its latest level,
//   MLS fit of density and velocity there, surface traction, block reduction
//   of force and torque (Eqs. 13-14), two-level rigid-body update (Eqs.
//   15-16), then the markers at the new level: MLS interpolation (Eq. 8),
//   direct-forcing force (Eq. 11) and the per-marker spreading record
//   S_l phi_k F_l of Eq. 12, plus the particle's support box.
// k_spread (one CTA per 16x16 tile of a particle's box): gathers, cell by
//   cell and in marker order, the records whose support covers the cell,
//   then adds the particle's sum into f_lb (the only atomic: one add per
//   cell and particle, contended only where particles overlap) and flags the
//   32-cell row segments the fluid kernel must read.
#include <climits>

#include "lbib_device.cuh"

namespace lbib {

namespace {

constexpr int PT = 256;    // threads per particle CTA
constexpr int TILE = 16;   // spreading tile edge
constexpr double CS2 = 1.0 / 3.0;
constexpr double PROBE = 1.2;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
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

template <class S, class C>
__global__ void __launch_bounds__(PT) k_particles(ParticleArgs a) {
    const S* __restrict__ f = static_cast<const S*>(a.f);
    const Geo& G = a.G;
    DParticle* P = a.parts + blockIdx.x;
    Rec<C>* recs = static_cast<Rec<C>*>(a.recs);
    __shared__ double red[3][PT / 32];
    __shared__ int ired[4][PT / 32];
    __shared__ double st_new[6];  // X, Y, theta, U, V, W at the new level
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int m0 = P->m0, nm = P->nm;
    const double X0 = P->X[0][0], Y0 = P->X[0][1], th0 = P->th[0];
    const double U0 = P->U[0][0], V0 = P->U[0][1], W0 = P->W[0];
    const double th1 = P->th[1], U1 = P->U[1][0], V1 = P->U[1][1], W1 = P->W[1];
    const double nu = CS2 * (G.tau - 0.5);
    double c0, s0, c1, s1;
    sincos(th0, &s0, &c0);
    sincos(th1, &s1, &c1);
    unsigned err = 0;

    // ---- probes on the body at the latest level -> F, M (Eqs. 13-14)
    double Fx = 0, Fy = 0, Mz = 0;
    for (int l = threadIdx.x; l < nm; l += PT) {
        const double2 rb = a.rb[m0 + l], nb = a.nb[m0 + l];
        const double Sl = a.S[m0 + l];
        const double rx = c0 * rb.x - s0 * rb.y, ry = s0 * rb.x + c0 * rb.y;  // x_l - X_c
        const double nx = c0 * nb.x - s0 * nb.y, ny = s0 * nb.x + c0 * nb.y;
        const double px = X0 + rx + PROBE * nx, py = Y0 + ry + PROBE * ny;
        int i0, j0;
        double phi[9], dpx[9], dpy[9];
        mls<true>(a.weight, px, py, i0, j0, phi, dpx, dpy);
        double r = 0, uxx = 0, uxy = 0, uyx = 0, uyy = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double rk, uk, vk;
            if (!node_fields<S, C>(f, G, i0 + k % 3, j0 + k / 3, rk, uk, vk)) {
                err |= ERR_DOMAIN;
                rk = 1.0; uk = 0.0; vk = 0.0;
            }
            r += phi[k] * rk;
            uxx += dpx[k] * uk;
            uxy += dpy[k] * uk;
            uyx += dpx[k] * vk;
            uyy += dpy[k] * vk;
        }
        // rigid velocity of the marker at the two stored levels
        const double r1x = c1 * rb.x - s1 * rb.y, r1y = s1 * rb.x + c1 * rb.y;
        const double dvx = (U0 - W0 * ry) - (U1 - W1 * r1y);
        const double dvy = (V0 + W0 * rx) - (V1 + W1 * r1x);
        const double p = CS2 * (r - 1.0) + r * PROBE * (dvx * nx + dvy * ny);
        const double mu = r * nu;
        const double txx = 2.0 * mu * uxx, tyy = 2.0 * mu * uyy, txy = mu * (uxy + uyx);
        const double tx = txx * nx + txy * ny - p * nx;
        const double ty = txy * nx + tyy * ny - p * ny;
        Fx += tx * Sl;
        Fy += ty * Sl;
        Mz += (rx * ty - ry * tx) * Sl;
    }
    Fx = warp_sum(Fx);
    Fy = warp_sum(Fy);
    Mz = warp_sum(Mz);
    if (lane == 0) {
        red[0][wid] = Fx;
        red[1][wid] = Fy;
        red[2][wid] = Mz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double F0 = 0, F1 = 0, M = 0;
        for (int w = 0; w < PT / 32; ++w) {
            F0 += red[0][w];
            F1 += red[1][w];
            M += red[2][w];
        }
        // ---- rigid-body update (Eqs. 15-16): one-level start, then BDF2
        const double buoy = (P->rho_s - 1.0) * P->area;
        const double ax = (F0 + buoy * a.gravity[0]) / P->mass;
        const double ay = (F1 + buoy * a.gravity[1]) / P->mass;
        const double al = M / P->inertia;
        double U, V, W, X, Y, T;
        if (P->nupd == 0) {
            U = U0 + ax;
            V = V0 + ay;
            W = W0 + al;
            X = X0 + U;
            Y = Y0 + V;
            T = th0 + W;
        } else {
            const double k = 2.0 / 3.0;
            U = k * (2.0 * U0 - 0.5 * U1 + ax);
            V = k * (2.0 * V0 - 0.5 * V1 + ay);
            W = k * (2.0 * W0 - 0.5 * W1 + al);
            X = k * (2.0 * X0 - 0.5 * P->X[1][0] + U);
            Y = k * (2.0 * Y0 - 0.5 * P->X[1][1] + V);
            T = k * (2.0 * th0 - 0.5 * th1 + W);
        }
        P->X[1][0] = X0; P->X[1][1] = Y0; P->th[1] = th0;
        P->U[1][0] = U0; P->U[1][1] = V0; P->W[1] = W0;
        P->X[0][0] = X; P->X[0][1] = Y; P->th[0] = T;
        P->U[0][0] = U; P->U[0][1] = V; P->W[0] = W;
        P->F[0] = F0; P->F[1] = F1; P->M = M;
        P->nupd += 1;
        if (!isfinite(X) || !isfinite(Y) || !isfinite(T)) err |= ERR_NONFINITE;
        st_new[0] = X; st_new[1] = Y; st_new[2] = T;
        st_new[3] = U; st_new[4] = V; st_new[5] = W;
    }
    __syncthreads();

    // ---- markers at the new level: interpolation, direct forcing, records
    const double X = st_new[0], Y = st_new[1];
    double cn, sn;
    sincos(st_new[2], &sn, &cn);
    const double U = st_new[3], V = st_new[4], W = st_new[5];
    int bx0 = INT_MAX, by0 = INT_MAX, bx1 = INT_MIN, by1 = INT_MIN;
    for (int l = threadIdx.x; l < nm; l += PT) {
        const double2 rb = a.rb[m0 + l];
        const double Sl = a.S[m0 + l];
        const double rx = cn * rb.x - sn * rb.y, ry = sn * rb.x + cn * rb.y;
        int i0, j0;
        double phi[9];
        mls<false>(a.weight, X + rx, Y + ry, i0, j0, phi, nullptr, nullptr);
        double ux = 0, uy = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double rk, uk, vk;
            if (!node_fields<S, C>(f, G, i0 + k % 3, j0 + k / 3, rk, uk, vk)) {
                err |= ERR_DOMAIN;
                uk = 0.0; vk = 0.0;
            }
            ux += phi[k] * uk;
            uy += phi[k] * vk;
        }
        const double Flx = (U - W * ry) - ux, Fly = (V + W * rx) - uy;  // Eq. 11, dt = 1
        Rec<C> rc;
        rc.i0 = i0;
        rc.j0 = j0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            rc.cx[k] = (C)(Sl * phi[k] * Flx);
            rc.cy[k] = (C)(Sl * phi[k] * Fly);
        }
        recs[m0 + l] = rc;
        bx0 = min(bx0, i0);
        by0 = min(by0, j0);
        bx1 = max(bx1, i0 + 2);
        by1 = max(by1, j0 + 2);
    }
    bx0 = warp_min(bx0);
    by0 = warp_min(by0);
    bx1 = warp_max(bx1);
    by1 = warp_max(by1);
    if (lane == 0) {
        ired[0][wid] = bx0;
        ired[1][wid] = by0;
        ired[2][wid] = bx1;
        ired[3][wid] = by1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int4 b = make_int4(INT_MAX, INT_MAX, INT_MIN, INT_MIN);
        for (int w = 0; w < PT / 32; ++w) {
            b.x = min(b.x, ired[0][w]);
            b.y = min(b.y, ired[1][w]);
            b.z = max(b.z, ired[2][w]);
            b.w = max(b.w, ired[3][w]);
        }
        a.boxes[blockIdx.x] = b;
    }
    if (err) atomicOr(a.err, err);
}

template <class C>
__global__ void __launch_bounds__(TILE * TILE) k_spread(SpreadArgs a) {
    const Geo& G = a.G;
    const DParticle* P = a.parts + blockIdx.y;
    const Rec<C>* recs = static_cast<const Rec<C>*>(a.recs);
    C* flb = static_cast<C*>(a.flb);
    __shared__ Rec<C> list[TILE * TILE];
    __shared__ int wcount[TILE * TILE / 32];
    const int4 box = a.boxes[blockIdx.y];
    if (box.x > box.z) return;
    const int tx = (box.z - box.x + TILE) / TILE, ty = (box.w - box.y + TILE) / TILE;
    if (blockIdx.x == 0 && threadIdx.x == 0 && tx * ty > (int)gridDim.x) atomicOr(a.err, ERR_DOMAIN);
    if ((int)blockIdx.x >= tx * ty) return;  // whole CTA
    const int x0 = box.x + (blockIdx.x % tx) * TILE, y0 = box.y + (blockIdx.x / tx) * TILE;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int cxl = x0 + t % TILE, cyl = y0 + t / TILE;  // this thread's (unwrapped) cell
    const int m0 = P->m0, nm = P->nm;
    C ax = C(0), ay = C(0);
    bool touched = false;
    for (int base = 0; base < nm; base += TILE * TILE) {
        const int l = base + t;
        bool rel = false;
        Rec<C> r;
        if (l < nm) {
            r = recs[m0 + l];
            rel = r.i0 <= x0 + TILE - 1 && r.i0 + 2 >= x0 && r.j0 <= y0 + TILE - 1 && r.j0 + 2 >= y0;
        }
        // order-preserving compaction of the relevant records
        const unsigned bal = __ballot_sync(0xffffffffu, rel);
        if (lane == 0) wcount[wid] = __popc(bal);
        __syncthreads();
        int off = 0, total = 0;
        for (int w = 0; w < TILE * TILE / 32; ++w) {
            off += (w < wid) ? wcount[w] : 0;
            total += wcount[w];
        }
        if (rel) list[off + __popc(bal & ((1u << lane) - 1u))] = r;
        __syncthreads();
        for (int m = 0; m < total; ++m) {
            const int da = cxl - list[m].i0, db = cyl - list[m].j0;
            if (da >= 0 && da < 3 && db >= 0 && db < 3) {
                ax += list[m].cx[db * 3 + da];
                ay += list[m].cy[db * 3 + da];
                touched = true;
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
    atomicAdd(flb + c, ax);
    atomicAdd(flb + G.plane + c, ay);
    a.flags[gy * G.nseg + (gx >> 5)] = 1;
}

}  // namespace

size_t rec_bytes(int prec) { return prec == LBM_FP64 ? sizeof(Rec<double>) : sizeof(Rec<float>); }

cudaError_t launch_particles(int prec, const ParticleArgs& a, int np, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    if (prec == LBM_FP64) k_particles<double, double><<<np, PT, 0, s>>>(a);
    else if (prec == LBM_FP32) k_particles<float, float><<<np, PT, 0, s>>>(a);
    else k_particles<__half, float><<<np, PT, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_spread(int prec, const SpreadArgs& a, int np, int tiles, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    const dim3 g(tiles, np);
    if (prec == LBM_FP64) k_spread<double><<<g, TILE * TILE, 0, s>>>(a);
    else k_spread<float><<<g, TILE * TILE, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbib
