// fluid_core.cuh -- the fused fluid step of one tile (pull-streaming with
// Zou-He walls, moments, IB force, forced BGK collision), shared by the
// fluid kernels that read the streamed populations straight from global
// memory and the persistent kernel that stages them in shared memory.
#pragma once

#include <cuda/std/limits>
#include <type_traits>

#include "lbib_device.cuh"

namespace lbib {

namespace {

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
template <> struct Vec<float, float, 2> {
    static __device__ __forceinline__ void load(const float* p, float v[2]) {
        const float2 q = __ldg(reinterpret_cast<const float2*>(p));
        v[0] = q.x; v[1] = q.y;
    }
    static __device__ __forceinline__ void store(float* p, const float v[2]) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    }
};
template <> struct Vec<__half, float, 2> {
    static __device__ __forceinline__ void load(const __half* p, float v[2]) {
        const float2 a = __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
        v[0] = a.x; v[1] = a.y;
    }
    static __device__ __forceinline__ void store(__half* p, const float v[2]) {
        *reinterpret_cast<__half2*>(p) = __floats2half2_rn(v[0], v[1]);
    }
};
template <> struct Vec<double, double, 2> {
    static __device__ __forceinline__ void load(const double* p, double v[2]) {
        const double2 a = __ldg(reinterpret_cast<const double2*>(p));
        v[0] = a.x; v[1] = a.y;
    }
    static __device__ __forceinline__ void store(double* p, const double v[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
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

// Vectors of N storage elements in shared memory (plain loads; the staged
// kernel's tiles are 16-byte aligned there)
template <class S, class C, int N> struct VecS;
template <> struct VecS<float, float, 4> {
    static __device__ __forceinline__ void load(const float* p, float v[4]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
};
template <> struct VecS<float, float, 2> {
    static __device__ __forceinline__ void load(const float* p, float v[2]) {
        const float2 q = *reinterpret_cast<const float2*>(p);
        v[0] = q.x; v[1] = q.y;
    }
};
template <> struct VecS<__half, float, 4> {
    static __device__ __forceinline__ void load(const __half* p, float v[4]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&q.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&q.y));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};
template <> struct VecS<__half, float, 2> {
    static __device__ __forceinline__ void load(const __half* p, float v[2]) {
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(p));
        v[0] = a.x; v[1] = a.y;
    }
};
template <class S, class C> __device__ __forceinline__ C lds(const S* p);
template <> __device__ __forceinline__ float lds<float, float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float lds<__half, float>(const __half* p) { return __half2float(*p); }

// Where a tile reads its streamed populations.  row(i, y) is a pointer p
// with p[x] = the stored value of plane i at column x of the source row of
// destination row y (y - cy(i), clamped into the lattice), valid for the
// columns x0 - 1 .. x0 + 32 N the tile reads; vec() loads N aligned
// elements there, one() a single one.
// GlobalSrc: the population buffer itself (read-only path).
template <class S, class C, int N>
struct GlobalSrc {
    static constexpr bool GLOBAL = true;
    const S* f;
    long long plane;
    int pitch, ny;
    __device__ __forceinline__ const S* row(int i, int y) const {
        const int ys = min(max(y - cy(i), 0), ny - 1);
        return f + (long long)i * plane + (long long)ys * pitch;
    }
    __device__ __forceinline__ void vec(const S* p, C q[N]) const { Vec<S, C, N>::load(p, q); }
    __device__ __forceinline__ C one(const S* p) const { return ld<S, C>(p); }
};
template <class S, class C, int N>
__device__ __forceinline__ GlobalSrc<S, C, N> global_src(const S* f, const Geo& G) {
    return GlobalSrc<S, C, N>{f, G.plane, G.pitch, G.ny};
}
// StageSrc: a tile's rows copied into shared memory, [9][rows][sw] elements
// per plane and destination row, element 0 of a row holding column xs
// (pitch, ny: the lattice's row pitch and rows).
template <class S, class C, int N>
struct StageSrc {
    static constexpr bool GLOBAL = false;
    const S* st;
    int sw, rows, y0, xs, pitch, ny;
    __device__ __forceinline__ const S* row(int i, int y) const {
        return st + (i * rows + (y - y0)) * sw - xs;
    }
    __device__ __forceinline__ void vec(const S* p, C q[N]) const { VecS<S, C, N>::load(p, q); }
    __device__ __forceinline__ C one(const S* p) const { return lds<S, C>(p); }
};

// The watchdog's test of one cell: its density rho = 1 + drho is positive
// and finite.  drho is the sum of the cell's nine streamed populations, so
// a NaN or infinite population (or an infinite pair of opposite signs)
// fails it as well (NaN compares false).
template <class C>
__device__ __forceinline__ bool density_ok(const C& drho) {
    const auto d = value_of(drho);
    using T = decltype(d);
    return d > T(-1) && d <= cuda::std::numeric_limits<T>::max();
}

// one cell: moments, IB force, forced BGK collision (Eqs. 2, 4-7); returns
// the watchdog's verdict on the cell (density_ok)
template <class C>
__device__ __forceinline__ bool cell_update(C v[9], const Geo& G, C fx_ib, C fy_ib) {
    C drho, jx, jy;
    moments<C>(v, drho, jx, jy);
    const C Fx = geo_g<C>(G, 0) + fx_ib, Fy = geo_g<C>(G, 1) + fy_ib;
    const C inv = C(1) / (C(1) + drho);
    const C ux = (jx + C(0.5) * Fx) * inv, uy = (jy + C(0.5) * Fy) * inv;
    collide<C>(v, drho, ux, uy, Fx, Fy, geo_omega<C>(G));
    return density_ok(drho);
}

// When a tile may read the forces of this step.  NoWait: at once (the
// flags load goes out with the population loads).  PdlWait: launched with
// programmatic stream serialization after the spreading kernel: the
// populations are loaded first, then the kernel waits for the spreading
// kernel before it reads the flags.  A hook with LATE = true is called
// after the population loads (per warp).
struct NoWait {
    static constexpr bool LATE = false;
    __device__ __forceinline__ void operator()() const {}
};
struct PdlWait {
    static constexpr bool LATE = true;
    __device__ __forceinline__ void operator()() const {
        pdl_wait();
        pdl_trigger();
    }
};

// The forces of this thread's cells when its segment is flagged (zero
// otherwise); the field is cleared for the next step after the tile.
template <class C, int N>
__device__ __forceinline__ void load_forces(bool forced, const ForceT<C>* flb, long long row, long long plane,
                                            int x0, int nx, C fx[N], C fy[N]) {
    if (!forced) return;
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (x0 + k < nx) {
            fx[k] = ForceField<C>::get(flb[row + x0 + k]);
            fy[k] = ForceField<C>::get(flb[plane + row + x0 + k]);
        }
}

// Pulled values of plane i for the thread's N cells from its loaded vector
// q: a pull along +-x is a one-lane shuffle of the neighbouring vector; bnd
// is the element past the warp's row end (lanes 0 / 31); on the periodic x
// edge the cell x = 0 (wrap_l) or x = nx - 1 (at ke, wrap_r) takes wl.
template <class C, int N>
__device__ __forceinline__ void pulled_plane(int i, const C q[N], C bnd, C wl, int lane, bool wrap_l, bool wrap_r,
                                             int ke, C v[N]) {
    if (cx(i) == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = q[k];
    } else if (cx(i) > 0) {  // source x - 1
        C left = __shfl_up_sync(0xffffffffu, q[N - 1], 1);
        if (lane == 0) left = bnd;
        v[0] = wrap_l ? wl : left;
#pragma unroll
        for (int k = 1; k < N; ++k) v[k] = q[k - 1];
    } else {  // source x + 1
        C right = __shfl_down_sync(0xffffffffu, q[0], 1);
        if (lane == 31) right = bnd;
#pragma unroll
        for (int k = 0; k < N - 1; ++k) v[k] = q[k + 1];
        v[N - 1] = right;
        if (wrap_r) {
#pragma unroll
            for (int k = 0; k < N; ++k)
                if (k == ke) v[k] = wl;
        }
    }
}

// FP16 storage read straight from global memory, two or four cells per
// thread, stays packed (two halves per 32-bit word) from the loads through
// the pull to the stores; a cell's values are widened to FP32 only around
// its collision.  That takes half the registers of the widened
// vectors (which spilled at the register budget of 1024 threads per SM).
// The bits are those of the widened path: the pull only moves halves, the
// collisions see the same FP32 values, and the results round to FP16 the
// same way (round to nearest even).
template <int N> struct Packed {
    static_assert(N == 2 || N == 4, "packed FP16 vectors hold two or four cells");
    static constexpr int W = N / 2;
    unsigned w[W];  // w[j]: cell 2j in the low half, cell 2j + 1 in the high half
    __device__ __forceinline__ void load(const __half* p) {
        if constexpr (N == 4) {
            const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
            w[0] = q.x;
            w[1] = q.y;
        } else {
            w[0] = __ldg(reinterpret_cast<const unsigned*>(p));
        }
    }
    __device__ __forceinline__ void store(__half* p) const {
        if constexpr (N == 4) *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
        else *reinterpret_cast<unsigned*>(p) = w[0];
    }
    __device__ __forceinline__ unsigned half(int k) const { return k & 1 ? w[k >> 1] >> 16 : w[k >> 1] & 0xffffu; }
    __device__ __forceinline__ void set(int k, unsigned h) {
        w[k >> 1] = k & 1 ? (w[k >> 1] & 0xffffu) | (h << 16) : (w[k >> 1] & 0xffff0000u) | h;
    }
};
__device__ __forceinline__ unsigned ld_bits(const __half* p) {
    return __ldg(reinterpret_cast<const unsigned short*>(p));
}
__device__ __forceinline__ void st_bits(__half* p, unsigned h) {
    *reinterpret_cast<unsigned short*>(p) = static_cast<unsigned short>(h);
}
__device__ __forceinline__ float widen1(unsigned bits) {
    return __half2float(__ushort_as_half(static_cast<unsigned short>(bits)));
}
__device__ __forceinline__ unsigned narrow1(float v) { return __half_as_ushort(__float2half_rn(v)); }

// pulled_plane on packed halves: a pull along +-x moves every half one
// place (a byte permutation of neighbouring words), the half that enters
// at the warp's row end coming from the neighbouring lane's word (bnd at
// lanes 0 / 31); on the periodic x edge x = 0 (wrap_l) or x = nx - 1 (at ke,
// wrap_r) takes wl.
template <int N>
__device__ __forceinline__ void pulled_packed(int i, Packed<N>& q, unsigned bnd, unsigned wl, int lane, bool wrap_l,
                                              bool wrap_r, int ke) {
    constexpr int W = N / 2;
    if (cx(i) > 0) {  // source x - 1: the left neighbour's last half enters at cell 0
        unsigned left = __shfl_up_sync(0xffffffffu, q.w[W - 1], 1);
        if (lane == 0) left = bnd << 16;
#pragma unroll
        for (int j = W - 1; j >= 1; --j) q.w[j] = __byte_perm(q.w[j - 1], q.w[j], 0x5432);
        q.w[0] = __byte_perm(left, q.w[0], 0x5432);
        if (wrap_l) q.set(0, wl);
    } else if (cx(i) < 0) {  // source x + 1: the right neighbour's first half enters at cell N - 1
        unsigned right = __shfl_down_sync(0xffffffffu, q.w[0], 1);
        if (lane == 31) right = bnd;
#pragma unroll
        for (int j = 0; j < W - 1; ++j) q.w[j] = __byte_perm(q.w[j], q.w[j + 1], 0x5432);
        q.w[W - 1] = __byte_perm(q.w[W - 1], right, 0x5432);
        if (wrap_r) {
#pragma unroll
            for (int k = 0; k < N; ++k)
                if (k == ke) q.set(k, wl);
        }
    }
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
// wait: when the forces may be read (NoWait, PdlWait, or the fused step's
// wait for its instance's spreading tiles): with a LATE hook the population
// loads come first, the force flags and the forces after the hook;
// otherwise the flags are loaded with the populations.
// Watchdog (check != 0): a warp with a cell of non-positive or non-finite
// density sets ERR_NONFINITE in *err (one atomic per such warp).  keep != 0
// leaves the force field and its flags for another launch of the same step.
// src: where the streamed populations come from (GlobalSrc or StageSrc);
// the periodic patch and the per-cell general path read fin itself.
template <class S, class C, int N, class Src, class Wait>
__device__ __forceinline__ void fluid_tile(const Src& src, const Geo& G, const S* __restrict__ fin,
                                           S* __restrict__ fout, ForceT<C>* __restrict__ flb,
                                           uint8_t* __restrict__ flags, int tx, int y, int check,
                                           unsigned* err, int keep, const Wait& wait) {
    constexpr bool PDL = Wait::LATE;
    const int lane = threadIdx.x & 31;
    const int x0 = (tx * 32 + lane) * N;
    // (FP32 and FP16 vector tiles take the row count and pitch from the
    // source, so that their loads need no descriptor load; the others from
    // G, which measured faster for them on GB300)
    constexpr bool HOIST = (sizeof(S) == 4 || sizeof(S) == 2) && N >= 2;
    if (y >= (HOIST ? src.ny : G.ny)) return;  // whole warp (one row)
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
    bool bad = false;  // watchdog

    const bool wrap = G.px && rows_in && any;
    const int ke = G.nx - 1 - x0;  // position of x = nx - 1 in this thread's cells
    const bool wrap_l = wrap && x0 == 0, wrap_r = wrap && ke >= 0 && ke < N;
    constexpr bool PACKED = std::is_same<S, __half>::value && N >= 2 && Src::GLOBAL;
    if constexpr (PACKED) {
        // the HOIST load order on packed halves, then the cells one by one
        Packed<N> pv[9];
        C fxh[N], fyh[N];
        {
            unsigned bnd[9], wl[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const S* rp = src.row(i, y);
                const int xa = min(x0, src.pitch - N);
                pv[i].load(rp + xa);
                bnd[i] = wl[i] = 0u;
                if (cx(i) > 0 && lane == 0) bnd[i] = ld_bits(rp + max(xa - 1, 0));
                if (cx(i) < 0 && lane == 31) bnd[i] = ld_bits(rp + min(xa + N, src.pitch - 1));
                const S* wp = fin + (long long)i * G.plane + (long long)(y - cy(i)) * G.pitch;
                if (cx(i) > 0 && wrap_l) wl[i] = ld_bits(wp + (G.nx - 1));
                if (cx(i) < 0 && wrap_r) wl[i] = ld_bits(wp);
            }
            if (PDL) {
                wait();
                forced = any && flags[seg] != 0;
            }
#pragma unroll
            for (int k = 0; k < N; ++k) fxh[k] = fyh[k] = C(0);
            load_forces<C, N>(forced, flb, row, G.plane, x0, G.nx, fxh, fyh);
#pragma unroll
            for (int i = 0; i < 9; ++i) pulled_packed<N>(i, pv[i], bnd[i], wl[i], lane, wrap_l, wrap_r, ke);
        }
        if (any) {
            unsigned edge = 0;  // bit k: cell x0 + k lies on an edge (and inside the lattice)
            bool ok = true;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const int xk = x0 + k;
                if (rows_in && xk < G.nx && (wrap || (xk >= 1 && xk <= G.nx - 2))) {
                    C c[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) c[i] = widen1(pv[i].half(k));
                    ok &= cell_update<C>(c, G, fxh[k], fyh[k]);
#pragma unroll
                    for (int i = 0; i < 9; ++i) pv[i].set(k, narrow1(c[i]));
                } else if (xk < G.nx) {
                    edge |= 1u << k;
                }
            }
            if (edge == 0 && x0 + N - 1 < G.nx) {
#pragma unroll
                for (int i = 0; i < 9; ++i) pv[i].store(fout + (long long)i * G.plane + row + x0);
            } else {
#pragma unroll
                for (int k = 0; k < N; ++k)
                    if (x0 + k < G.nx && !(edge >> k & 1u)) {
#pragma unroll
                        for (int i = 0; i < 9; ++i)
                            st_bits(fout + (long long)i * G.plane + row + x0 + k, pv[i].half(k));
                    }
                // cells on a wall or periodic edge: the general path
#pragma unroll 1
                for (int k = 0; k < N; ++k) {
                    if (!(edge >> k & 1u)) continue;
                    const int xk = x0 + k;
                    C c[9];
                    pull_general<S, C>(fin, G, xk, y, c);
                    complete_walls<S, C>(fin, G, xk, y, c);
                    C gx = C(0), gy = C(0);
                    if (forced) {
#pragma unroll
                        for (int jj = 0; jj < N; ++jj)
                            if (jj == k) {
                                gx = fxh[jj];
                                gy = fyh[jj];
                            }
                    }
                    ok &= cell_update<C>(c, G, gx, gy);
#pragma unroll
                    for (int i = 0; i < 9; ++i) st<S, C>(fout + (long long)i * G.plane + row + xk, c[i]);
                }
            }
            bad = !ok;
        }
    } else {
        C v[9][N], fxh[N], fyh[N];  // (fxh, fyh: the forces read early, HOIST)
        // Two load orders, chosen per storage type and width by measurement on
        // GB300: FP32 and FP16 vectors of two or four cells issue every
        // population load and the force loads of a flagged segment before
        // consuming any (the flag -> force chain then overlaps the population
        // loads; the 512-lattice batch in FP16 storage 0.946 -> 0.902 ms per
        // step); FP64 and one-cell tiles load and shuffle plane by plane and
        // read the forces after the populations (fewer live registers).
        if constexpr (HOIST) {
            C q[9][N], bnd[9], wl[9];
    #pragma unroll
            for (int i = 0; i < 9; ++i) {
                const S* rp = src.row(i, y);
                const int xa = min(x0, src.pitch - N);
                src.vec(rp + xa, q[i]);
                bnd[i] = wl[i] = C(0);
                if (cx(i) > 0 && lane == 0) bnd[i] = src.one(rp + max(xa - 1, 0));
                if (cx(i) < 0 && lane == 31) bnd[i] = src.one(rp + min(xa + N, src.pitch - 1));
                const S* wp = fin + (long long)i * G.plane + (long long)(y - cy(i)) * G.pitch;
                if (cx(i) > 0 && wrap_l) wl[i] = ld<S, C>(wp + (G.nx - 1));
                if (cx(i) < 0 && wrap_r) wl[i] = ld<S, C>(wp);
            }
            if (PDL) {
                // the populations are on their way; the forces of this step
                // come from the spreading items before this one
                wait();
                forced = any && flags[seg] != 0;
            }
    #pragma unroll
            for (int k = 0; k < N; ++k) fxh[k] = fyh[k] = C(0);
            load_forces<C, N>(forced, flb, row, G.plane, x0, G.nx, fxh, fyh);
    #pragma unroll
            for (int i = 0; i < 9; ++i) pulled_plane<C, N>(i, q[i], bnd[i], wl[i], lane, wrap_l, wrap_r, ke, v[i]);
        } else {
    #pragma unroll
            for (int i = 0; i < 9; ++i) {
                const S* rp = src.row(i, y);
                const int xa = min(x0, G.pitch - N);
                C q[N], bnd = C(0), wl = C(0);
                src.vec(rp + xa, q);
                if (cx(i) > 0 && lane == 0) bnd = src.one(rp + max(xa - 1, 0));
                if (cx(i) < 0 && lane == 31) bnd = src.one(rp + min(xa + N, G.pitch - 1));
                pulled_plane<C, N>(i, q, bnd, wl, lane, false, false, ke, v[i]);
            }
            // periodic x: the three populations that cross the edge
            if (wrap_l || wrap_r) {
    #pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const S* wp = fin + (long long)i * G.plane + (long long)(y - cy(i)) * G.pitch;
                    if (cx(i) > 0 && wrap_l) v[i][0] = ld<S, C>(wp + (G.nx - 1));
                    if (cx(i) < 0 && wrap_r) {
                        const C w0 = ld<S, C>(wp);
    #pragma unroll
                        for (int k = 0; k < N; ++k)
                            if (k == ke) v[i][k] = w0;
                    }
                }
            }
            if (PDL) {
                wait();
                forced = any && flags[seg] != 0;
            }
        }
        if (any) {
            C fxi[N], fyi[N];
    #pragma unroll
            for (int k = 0; k < N; ++k) fxi[k] = fyi[k] = C(0);
            if constexpr (HOIST) {
    #pragma unroll
                for (int k = 0; k < N; ++k) {
                    fxi[k] = fxh[k];
                    fyi[k] = fyh[k];
                }
            } else {
                load_forces<C, N>(forced, flb, row, G.plane, x0, G.nx, fxi, fyi);
            }
            // interior cells from the vector values.  With one cell per thread
            // so are the cells of an x wall between the two y edges: their six
            // known populations come from inside the row range, and the Zou-He
            // completion replaces the three that point into the fluid (with
            // four cells per thread the completion inlined per cell costs the
            // vector path registers, so those cells take the general path)
            constexpr bool XW = N == 1;
            unsigned edge = 0;  // bit k: cell x0 + k lies on an edge (and inside the lattice)
            bool ok = true;     // the watchdog's verdict on this thread's cells
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
                    ok &= cell_update<C>(c, G, fxi[k], fyi[k]);
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
                    if (forced) {  // forces of this cell were read above
    #pragma unroll
                        for (int j = 0; j < N; ++j)
                            if (j == k) {
                                gx = fxi[j];
                                gy = fyi[j];
                            }
                    }
                    ok &= cell_update<C>(c, G, gx, gy);
    #pragma unroll
                    for (int i = 0; i < 9; ++i) st<S, C>(fout + (long long)i * G.plane + row + xk, c[i]);
                }
            }
            bad = !ok;
        }
    }
    // the force field and the flag are cleared for the next step only now,
    // after their values were used (stores right behind the loads of the
    // same words measured 35 % slower on the screening batch); keep: the
    // autotuner's repeated launches of one step leave them in place
    if (forced && !keep) {
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (x0 + k < G.nx) {
                flb[row + x0 + k] = ForceT<C>(0);
                flb[G.plane + row + x0 + k] = ForceT<C>(0);
            }
    }
    __syncwarp();
    if (check && __any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, ERR_NONFINITE);
    if (forced && !keep && (lane & (32 / N - 1)) == 0) flags[seg] = 0;  // one lane per segment
}

}  // namespace

}  // namespace lbib
