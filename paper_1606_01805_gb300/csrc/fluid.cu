// fluid.cu -- lattice kernels: initial field, the fused pull-stream /
// Zou-He / moments / forced-BGK collide step, and field extraction.
#include "lbib_device.cuh"

namespace lbib {

namespace {

constexpr int BY = 8;  // rows per block of the init and field kernels

// BGK relaxation of Eq. 4 towards the shifted equilibrium f~eq_i = f_eq_i - w_i
// (Eq. 2), plus the Guo term (Eq. 5), in place on v:
//   v_i <- (1 - omega) v_i + omega f~eq_i + G_i.
// Written over opposite velocity pairs (i, i'): with e_i' = -e_i both terms
// split into a part even in e (shared) and a part odd in e (sign-flipped),
// and their sum collects into
//   omega f~eq_i + G_i = w (K0 + eu (a eu + b eF)) +- 3 w (c eu + cf eF)
// with eu = e.u, eF = e.F, c = omega rho, a = 4.5 c, cf = 1 - omega / 2,
// b = 9 cf and K0 = omega drho - 1.5 c u.u - 3 cf u.F (the rest population's
// value, w = 4/9, has eu = eF = 0).
template <class C>
__device__ __forceinline__ void collide(C v[9], C drho, C ux, C uy, C Fx, C Fy, C omega) {
    const C rho = C(1) + drho;
    const C usq = ux * ux + uy * uy;
    const C cf = C(1) - C(0.5) * omega;
    const C uF = ux * Fx + uy * Fy;
    const C keep = C(1) - omega;
    const C c = omega * rho, a = C(4.5) * c, b = C(9) * cf;
    const C K0 = omega * drho - C(1.5) * c * usq - C(3) * cf * uF;
    v[0] = keep * v[0] + C(4.0 / 9.0) * K0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        // pairs (1,3), (2,4), (5,7), (6,8): i has e = (ex, ey), i' has -e
        const int i = p == 0 ? 1 : p == 1 ? 2 : p == 2 ? 5 : 6;
        const int j = p == 0 ? 3 : p == 1 ? 4 : p == 2 ? 7 : 8;
        const C w = C(wt(i));
        const C eu = C(cx(i)) * ux + C(cy(i)) * uy;
        const C eF = C(cx(i)) * Fx + C(cy(i)) * Fy;
        const C even = w * (K0 + eu * (a * eu + b * eF));
        const C odd = C(3) * w * (c * eu + cf * eF);
        v[i] = keep * v[i] + (even + odd);
        v[j] = keep * v[j] + (even - odd);
    }
}

// N consecutive storage elements starting at an N-aligned index
template <class S, class C, int N> struct Vec;
template <class S, class C> struct Vec<S, C, 1> {
    static __device__ __forceinline__ void load(const S* p, C v[1]) { v[0] = ld<S, C>(p); }
    static __device__ __forceinline__ void store(S* p, const C v[1]) { st<S, C>(p, v[0]); }
};
template <> struct Vec<float, float, 4> {
    static __device__ __forceinline__ void load(const float* p, float v[4]) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    static __device__ __forceinline__ void store(float* p, const float v[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec<double, double, 4> {
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
template <> struct Vec<__half, float, 4> {
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

// Fused step of one tile: N consecutive cells (x0 .. x0+N-1, x0 = N * lane
// index) of one row per thread, a warp covering 32 N cells of a row, the
// block BY rows.  Populations move as vectors of N elements: a pull along
// +-x is a one-lane shuffle of the neighbouring vector, with one extra
// element load at the warp's two ends.  Cells of the first and last row
// (y walls, corners, periodic y edges) take the per-cell general path
// (emitted once, after the fast cells), and so do those of x walls when a
// thread holds four cells; with one cell per thread the x-wall cells in
// between stay on the vector path with their Zou-He completion.  The
// periodic x edge patches the three populations that cross it.
// PDL: launched with programmatic stream serialization after the spreading
// kernel: the population loads come first, the force flags and the forces
// after pdl_wait().  Otherwise the flags are loaded with the populations.
template <class S, class C, int N, bool PDL>
__device__ __forceinline__ void fluid_tile(const Geo& G, const S* __restrict__ fin,
                                           S* __restrict__ fout, C* __restrict__ flb,
                                           uint8_t* __restrict__ flags, int tx, int y) {
    const int lane = threadIdx.x;
    const int x0 = (tx * 32 + lane) * N;
    if (y >= G.ny) return;  // whole warp (one row)
    const long long row = (long long)y * G.pitch;
    // the vector values of cell x0 + k are its pulled populations whenever
    // all 9 sources are inside (none clamped); on an x wall all but the
    // three that the Zou-He completion replaces
    const bool rows_in = y >= 1 && y <= G.ny - 2;
    const bool any = x0 < G.nx;
    // force flags of the 32-cell segment of this thread
    const int seg = y * G.nseg + (x0 >> 5);
    bool forced = false;
    if (!PDL) forced = any && flags[seg] != 0;

    C v[9][N];
    // vector loads for every lane (addresses clamped in-bounds), shuffles by all
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int ys = min(max(y - cy(i), 0), G.ny - 1);
        const S* rp = fin + (long long)i * G.plane + (long long)ys * G.pitch;
        const int xa = min(x0, G.pitch - N);
        C q[N];
        Vec<S, C, N>::load(rp + xa, q);
        if (cx(i) == 0) {
#pragma unroll
            for (int k = 0; k < N; ++k) v[i][k] = q[k];
        } else if (cx(i) > 0) {  // source x - 1
            C left = __shfl_up_sync(0xffffffffu, q[N - 1], 1);
            if (lane == 0) left = ld<S, C>(rp + max(xa - 1, 0));
            v[i][0] = left;
#pragma unroll
            for (int k = 1; k < N; ++k) v[i][k] = q[k - 1];
        } else {  // source x + 1
            C right = __shfl_down_sync(0xffffffffu, q[0], 1);
            if (lane == 31) right = ld<S, C>(rp + min(xa + N, G.pitch - 1));
#pragma unroll
            for (int k = 0; k < N - 1; ++k) v[i][k] = q[k + 1];
            v[i][N - 1] = right;
        }
    }
    // periodic x: the cells x = 0 and x = nx - 1 get the three populations
    // that cross the periodic edge by scalar loads; their other six are
    // already in the vectors, so they stay on the fast path
    const bool wrap = G.px && rows_in && any;
    const int ke = G.nx - 1 - x0;  // position of x = nx - 1 in this thread's cells
    if (wrap && (x0 == 0 || (ke >= 0 && ke < N))) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const S* rp = fin + (long long)i * G.plane + (long long)(y - cy(i)) * G.pitch;
            if (cx(i) > 0 && x0 == 0) v[i][0] = ld<S, C>(rp + (G.nx - 1));
            if (cx(i) < 0 && ke >= 0 && ke < N) {
                const C w0 = ld<S, C>(rp);
#pragma unroll
                for (int k = 0; k < N; ++k)
                    if (k == ke) v[i][k] = w0;
            }
        }
    }
    if (PDL) {
        // the populations are on their way; the forces of this step come
        // from the spreading kernel before this one
        pdl_wait();
        pdl_trigger();
        forced = any && flags[seg] != 0;
    }
    if (any) {
        C fxi[N], fyi[N];
#pragma unroll
        for (int k = 0; k < N; ++k) fxi[k] = fyi[k] = C(0);
        if (forced) {
#pragma unroll
            for (int k = 0; k < N; ++k)
                if (x0 + k < G.nx) {
                    fxi[k] = flb[row + x0 + k];
                    fyi[k] = flb[G.plane + row + x0 + k];
                    flb[row + x0 + k] = C(0);
                    flb[G.plane + row + x0 + k] = C(0);
                }
        }
        // interior cells from the vector values.  With one cell per thread
        // so are the cells of an x wall between the two y edges: their six
        // known populations come from inside the row range, and the Zou-He
        // completion replaces the three that point into the fluid (with
        // four cells per thread the completion inlined per cell costs the
        // vector path registers, so those cells take the general path)
        constexpr bool XW = N == 1;
        unsigned edge = 0;  // bit k: cell x0 + k lies on an edge (and inside the lattice)
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int xk = x0 + k;
            if (rows_in && xk < G.nx && (wrap || XW || (xk >= 1 && xk <= G.nx - 2))) {
                C c[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) c[i] = v[i][k];
                if (XW && !G.px && (xk == 0 || xk == G.nx - 1)) {
                    const C gx = geo_g<C>(G, 0), gy = geo_g<C>(G, 1);
                    if (xk == 0) zou_he_edge<1, 0, C>(c, geo_uw<C>(G, 0, 0), geo_uw<C>(G, 0, 1), gx, gy);
                    else zou_he_edge<-1, 0, C>(c, geo_uw<C>(G, 1, 0), geo_uw<C>(G, 1, 1), gx, gy);
                }
                cell_update<C>(c, G, fxi[k], fyi[k]);
#pragma unroll
                for (int i = 0; i < 9; ++i) v[i][k] = c[i];
            } else if (xk < G.nx) {
                edge |= 1u << k;
            }
        }
        if (edge == 0 && x0 + N - 1 < G.nx) {
#pragma unroll
            for (int i = 0; i < 9; ++i) Vec<S, C, N>::store(fout + (long long)i * G.plane + row + x0, v[i]);
        } else {
#pragma unroll
            for (int k = 0; k < N; ++k)
                if (x0 + k < G.nx && !(edge >> k & 1u)) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) st<S, C>(fout + (long long)i * G.plane + row + x0 + k, v[i][k]);
                }
            // cells on a wall or periodic edge: general pull, wall completion,
            // collision, one at a time (emitted once, nothing else live)
#pragma unroll 1
            for (int k = 0; k < N; ++k) {
                if (!(edge >> k & 1u)) continue;
                const int xk = x0 + k;
                C c[9];
                pull_general<S, C>(fin, G, xk, y, c);
                complete_walls<S, C>(fin, G, xk, y, c);
                C gx = C(0), gy = C(0);
                if (forced) {  // forces of this cell were read (and zeroed) above
#pragma unroll
                    for (int j = 0; j < N; ++j)
                        if (j == k) {
                            gx = fxi[j];
                            gy = fyi[j];
                        }
                }
                cell_update<C>(c, G, gx, gy);
#pragma unroll
                for (int i = 0; i < 9; ++i) st<S, C>(fout + (long long)i * G.plane + row + xk, c[i]);
            }
        }
    }
    __syncwarp();
    if (forced && (lane & (32 / N - 1)) == 0) flags[seg] = 0;  // one lane per segment
}

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
        fluid_tile<S, C, N, false>(I.G, fin + I.f_off, fout + I.f_off, flb + I.flb_off,
                            a.flags + I.flags_off, task.y, task.z * BYt + threadIdx.y);
    }
}

// the same step for a context holding one lattice: its descriptor arrives
// by value (constant bank) and the grid is the tile grid itself, so no load
// stands in front of the population loads
template <class S, class C, int N, int BYt, bool PDL>
__global__ void __launch_bounds__(32 * BYt, FluidOccupancy<S, N, BYt>::value)
    k_fluid_one(FluidArgs a, Inst I) {
    fluid_tile<S, C, N, PDL>(I.G, static_cast<const S*>(a.fin) + I.f_off, static_cast<S*>(a.fout) + I.f_off,
                        static_cast<C*>(a.flb) + I.flb_off, a.flags + I.flags_off, blockIdx.x,
                        blockIdx.y * BYt + threadIdx.y);
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
    C rho, ux, uy;
    node_fields<S, C>(static_cast<const S*>(a.f) + a.I.f_off, a.I.G, &a.I.G, x, a.y0 + r, rho, ux, uy);
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

cudaError_t launch_fields(int prec, const FieldArgs& a, cudaStream_t s) {
    const dim3 b(32, BY), g = grid_for(a.I.G.nx, a.rows);
    if (prec == LBM_FP64) k_fields<double, double><<<g, b, 0, s>>>(a);
    else if (prec == LBM_FP32) k_fields<float, float><<<g, b, 0, s>>>(a);
    else if (prec == LBM_FP16_SHIFTED) k_fields<__half, float><<<g, b, 0, s>>>(a);
    else k_fields<TF, TF><<<g, b, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace lbib
