// dual.h -- forward-mode (tangent-linear) differentiation by dual numbers.
//
// Dual<T, K> carries a value and its derivatives along K directions.  Every
// arithmetic operation and every elementary function used by the LB-IB step
// propagates them by the chain rule, so running the step on duals gives the
// directional derivatives of every state variable with respect to K input
// parameters (seeded in the initial state), alongside the state itself.
// Comparisons and the choice of MLS support (floor) act on values: the
// support is piecewise constant, so it contributes no derivative.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define LBIB_HD __host__ __device__ __forceinline__
#else
#define LBIB_HD inline
#endif

namespace lbib {

// the scalar overloads stay visible next to the dual ones below
using ::sqrt;
using ::exp;
using ::cos;
using ::sin;
using ::hypot;

template <class T, int K>
struct Dual {
    T v;
    T d[K];

    Dual() = default;
    LBIB_HD Dual(T x) : v(x) {
        for (int k = 0; k < K; ++k) d[k] = T(0);
    }
    template <class U, int KK>
    LBIB_HD explicit Dual(const Dual<U, KK>& o) : v(T(o.v)) {
        static_assert(KK == K, "derivative counts must match");
        for (int k = 0; k < K; ++k) d[k] = T(o.d[k]);
    }
    LBIB_HD explicit operator T() const { return v; }

    LBIB_HD Dual& operator+=(const Dual& o) {
        v += o.v;
        for (int k = 0; k < K; ++k) d[k] += o.d[k];
        return *this;
    }
    LBIB_HD Dual& operator-=(const Dual& o) {
        v -= o.v;
        for (int k = 0; k < K; ++k) d[k] -= o.d[k];
        return *this;
    }
    LBIB_HD Dual& operator*=(const Dual& o) { return *this = *this * o; }
};

template <class T, int K>
LBIB_HD Dual<T, K> operator+(Dual<T, K> a, const Dual<T, K>& b) { return a += b; }
template <class T, int K>
LBIB_HD Dual<T, K> operator-(Dual<T, K> a, const Dual<T, K>& b) { return a -= b; }
template <class T, int K>
LBIB_HD Dual<T, K> operator-(const Dual<T, K>& a) {
    Dual<T, K> r;
    r.v = -a.v;
    for (int k = 0; k < K; ++k) r.d[k] = -a.d[k];
    return r;
}
template <class T, int K>
LBIB_HD Dual<T, K> operator*(const Dual<T, K>& a, const Dual<T, K>& b) {
    Dual<T, K> r;
    r.v = a.v * b.v;
    for (int k = 0; k < K; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <class T, int K>
LBIB_HD Dual<T, K> operator/(const Dual<T, K>& a, const Dual<T, K>& b) {
    Dual<T, K> r;
    const T inv = T(1) / b.v;
    r.v = a.v * inv;
    for (int k = 0; k < K; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * inv;
    return r;
}
// mixed with a plain scalar of the value type
#define LBIB_DUAL_MIXED(op)                                                              \
    template <class T, int K>                                                             \
    LBIB_HD Dual<T, K> operator op(const Dual<T, K>& a, T b) { return a op Dual<T, K>(b); } \
    template <class T, int K>                                                             \
    LBIB_HD Dual<T, K> operator op(T a, const Dual<T, K>& b) { return Dual<T, K>(a) op b; }
LBIB_DUAL_MIXED(+)
LBIB_DUAL_MIXED(-)
LBIB_DUAL_MIXED(*)
LBIB_DUAL_MIXED(/)
#undef LBIB_DUAL_MIXED

template <class T, int K> LBIB_HD bool operator<(const Dual<T, K>& a, const Dual<T, K>& b) { return a.v < b.v; }
template <class T, int K> LBIB_HD bool operator>(const Dual<T, K>& a, const Dual<T, K>& b) { return a.v > b.v; }
template <class T, int K> LBIB_HD bool operator<=(const Dual<T, K>& a, const Dual<T, K>& b) { return a.v <= b.v; }
template <class T, int K> LBIB_HD bool operator>=(const Dual<T, K>& a, const Dual<T, K>& b) { return a.v >= b.v; }

// elementary functions: f(a) with f'(a) times the derivatives
template <class T, int K>
LBIB_HD Dual<T, K> chain(const Dual<T, K>& a, T f, T fp) {
    Dual<T, K> r;
    r.v = f;
    for (int k = 0; k < K; ++k) r.d[k] = fp * a.d[k];
    return r;
}
template <class T, int K>
LBIB_HD Dual<T, K> sqrt(const Dual<T, K>& a) {
    using std::sqrt;
    const T s = sqrt(a.v);
    return chain(a, s, s > T(0) ? T(0.5) / s : T(0));
}
template <class T, int K>
LBIB_HD Dual<T, K> exp(const Dual<T, K>& a) {
    using std::exp;
    const T e = exp(a.v);
    return chain(a, e, e);
}
template <class T, int K>
LBIB_HD Dual<T, K> cos(const Dual<T, K>& a) {
    using std::cos;
    using std::sin;
    return chain(a, cos(a.v), -sin(a.v));
}
template <class T, int K>
LBIB_HD Dual<T, K> sin(const Dual<T, K>& a) {
    using std::cos;
    using std::sin;
    return chain(a, sin(a.v), cos(a.v));
}
template <class T, int K>
LBIB_HD Dual<T, K> hypot(const Dual<T, K>& a, const Dual<T, K>& b) { return sqrt(a * a + b * b); }
#ifdef __CUDACC__
using ::cospi;
using ::__shfl_xor_sync;
using ::__shfl_down_sync;
using ::__shfl_up_sync;
using ::__shfl_sync;
using ::atomicAdd;
using ::isfinite;
using ::sincos;

template <class T, int K>
__device__ __forceinline__ Dual<T, K> cospi(const Dual<T, K>& a) {
    const T pi = T(3.141592653589793);
    return chain(a, ::cospi(a.v), -pi * ::sinpi(a.v));
}
// warp shuffles move every component
template <class T, int K>
__device__ __forceinline__ Dual<T, K> __shfl_xor_sync(unsigned m, const Dual<T, K>& a, int o) {
    Dual<T, K> r;
    r.v = ::__shfl_xor_sync(m, a.v, o);
    for (int k = 0; k < K; ++k) r.d[k] = ::__shfl_xor_sync(m, a.d[k], o);
    return r;
}
template <class T, int K>
__device__ __forceinline__ Dual<T, K> __shfl_down_sync(unsigned m, const Dual<T, K>& a, int o) {
    Dual<T, K> r;
    r.v = ::__shfl_down_sync(m, a.v, o);
    for (int k = 0; k < K; ++k) r.d[k] = ::__shfl_down_sync(m, a.d[k], o);
    return r;
}
template <class T, int K>
__device__ __forceinline__ Dual<T, K> __shfl_up_sync(unsigned m, const Dual<T, K>& a, int o) {
    Dual<T, K> r;
    r.v = ::__shfl_up_sync(m, a.v, o);
    for (int k = 0; k < K; ++k) r.d[k] = ::__shfl_up_sync(m, a.d[k], o);
    return r;
}
template <class T, int K>
__device__ __forceinline__ Dual<T, K> __shfl_sync(unsigned m, const Dual<T, K>& a, int l) {
    Dual<T, K> r;
    r.v = ::__shfl_sync(m, a.v, l);
    for (int k = 0; k < K; ++k) r.d[k] = ::__shfl_sync(m, a.d[k], l);
    return r;
}
// component-wise atomic add (each component is an independent sum)
template <class T, int K>
__device__ __forceinline__ void atomicAdd(Dual<T, K>* p, const Dual<T, K>& a) {
    ::atomicAdd(&p->v, a.v);
    for (int k = 0; k < K; ++k) ::atomicAdd(&p->d[k], a.d[k]);
}
template <class T, int K>
__device__ __forceinline__ bool isfinite(const Dual<T, K>& a) {
    bool ok = ::isfinite(a.v);
    for (int k = 0; k < K; ++k) ok = ok && ::isfinite(a.d[k]);
    return ok;
}
template <class T, int K>
__device__ __forceinline__ void sincos(const Dual<T, K>& a, Dual<T, K>* s, Dual<T, K>* c) {
    T sv, cv;
    ::sincos(a.v, &sv, &cv);
    *s = chain(a, sv, cv);
    *c = chain(a, cv, -sv);
}
#endif

// floor of the value (the MLS support choice): piecewise constant, no derivative
template <class T, int K>
LBIB_HD T floor_value(const Dual<T, K>& a) {
    using std::floor;
    return floor(a.v);
}

LBIB_HD double floor_value(double a) { return std::floor(a); }
LBIB_HD float floor_value(float a) { return std::floor(a); }

template <class X> struct DualTraits {
    using value = X;
    static constexpr int K = 0;
};
template <class T, int K_> struct DualTraits<Dual<T, K_>> {
    using value = T;
    static constexpr int K = K_;
};

// value of a scalar or a dual, and its k-th derivative (0 for a scalar)
template <class X> LBIB_HD typename DualTraits<X>::value value_of(const X& x) { return x; }
template <class T, int K> LBIB_HD T value_of(const Dual<T, K>& x) { return x.v; }
template <class X> LBIB_HD typename DualTraits<X>::value derivative(const X&, int) { return 0; }
template <class T, int K> LBIB_HD T derivative(const Dual<T, K>& x, int k) { return x.d[k]; }

}  // namespace lbib
