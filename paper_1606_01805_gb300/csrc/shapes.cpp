// shapes.cpp -- Lagrangian markers and rigid-body properties of the particle
// shapes of Sections 3-4 (circle, ellipse, rectangle, square, equilateral
// triangle), in the body frame with the centroid at the origin.
//
// Markers sit at the midpoints of equal arc-length pieces of the perimeter
// and carry the piece length S_l; the normal is the analytic outward normal
// (circle, ellipse) or the face normal (polygons, each face cut into its own
// equal pieces so that no marker straddles a corner).
#include <algorithm>
#include <cmath>
#include <vector>

#include "lbib_internal.h"

namespace lbib {

namespace {

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on the
// Legendre recurrence.
struct GaussLegendre {
    std::vector<double> x, w;
    explicit GaussLegendre(int n) : x(n), w(n) {
        for (int i = 0; i < n; ++i) {
            double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0;
            for (int it = 0; it < 100; ++it) {
                double p0 = 1, p1 = z;
                for (int k = 2; k <= n; ++k) {
                    const double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                const double dz = p1 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            x[i] = z;
            w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
    }
};

// Arc length along (a cos t, b sin t), t in [0, 2 pi]: a table of the
// cumulative length at NT equal steps of t (one 20-point Gauss-Legendre
// panel per step), and within a step one more panel from the step's start
struct ArcRule {
    static constexpr int NT = 256;
    static constexpr double DT = 2.0 * M_PI / NT;
};

template <class T>
T arc_panel(const T& a, const T& b, double t0, const T& t1) {
    using std::cos;
    using std::hypot;
    using std::sin;
    static const GaussLegendre gl(20);
    const T h = t1 - t0, mid = t0 + 0.5 * h;
    T acc = T(0.0);
    for (size_t i = 0; i < gl.x.size(); ++i) {
        const T s = mid + (0.5 * gl.x[i]) * h;
        acc += gl.w[i] * hypot(a * sin(s), b * cos(s));
    }
    return 0.5 * h * acc;
}

template <class T>
struct EllipseArc {
    T a, b;
    std::vector<T> cum;
    EllipseArc(const T& a_, const T& b_) : a(a_), b(b_), cum(ArcRule::NT + 1) {
        cum[0] = T(0.0);
        for (int j = 0; j < ArcRule::NT; ++j)
            cum[j + 1] = cum[j] + arc_panel<T>(a, b, j * ArcRule::DT, T((j + 1) * ArcRule::DT));
    }
    T perimeter() const { return cum[ArcRule::NT]; }
    int step_of(double t) const { return std::min(std::max((int)std::floor(t / ArcRule::DT), 0), ArcRule::NT - 1); }
    T operator()(const T& t) const {  // length over [0, t]
        const int j = step_of(value_of(t));
        return cum[j] + arc_panel<T>(a, b, j * ArcRule::DT, t);
    }
    // the parameter where the length reaches s (values only): linear in the
    // table's step, the start of the Newton iteration
    double guess(double s) const {
        int j = 0;
        while (j < ArcRule::NT - 1 && value_of(cum[j + 1]) <= s) ++j;
        const double c0 = value_of(cum[j]), c1 = value_of(cum[j + 1]);
        return (j + (s - c0) / (c1 - c0)) * ArcRule::DT;
    }
};

}  // namespace

// T = double, or TD: the dimensions then carry derivatives, and so do the
// markers, normals, arc lengths, area and inertia (the marker count and the
// split of the polygon faces follow the values only)
template <class T>
int make_shape_t(const lbm_particle_desc& d, const T dim[2], double spacing, T* rb, T* nb, T* S,
                 int cap, ShapeOutT<T>* out) {
    using std::cos;
    using std::hypot;
    using std::sin;
    using std::sqrt;
    const double h0 = spacing > 0 ? spacing : 0.3;
    const T D0 = dim[0], D1 = dim[1];
    int n = 0;
    switch (d.shape) {
        case LBM_SHAPE_CIRCLE:
        case LBM_SHAPE_ELLIPSE: {
            const T a = 0.5 * D0, b = d.shape == LBM_SHAPE_CIRCLE ? 0.5 * D0 : 0.5 * D1;
            std::vector<EllipseArc<T>> arc;
            if (d.shape == LBM_SHAPE_ELLIPSE) arc.emplace_back(a, b);
            const T P = d.shape == LBM_SHAPE_CIRCLE ? M_PI * D0 : arc[0].perimeter();
            n = d.n_markers > 0 ? d.n_markers : (int)std::lround(value_of(P) / h0);
            if (n < 8) n = 8;
            if (n > cap) return -1;
            for (int l = 0; l < n; ++l) {
                T t = T(2.0 * M_PI * (l + 0.5) / n);
                if (d.shape == LBM_SHAPE_ELLIPSE) {  // invert the arc length by Newton
                    const T target = ((l + 0.5) / n) * P;
                    t = T(arc[0].guess(value_of(target)));
                    for (int it = 0; it < 60; ++it) {
                        const T g = arc[0](t) - target;
                        const T dt = g / hypot(a * sin(t), b * cos(t));
                        t -= dt;
                        // one more pass after the value has converged lets the
                        // derivatives converge too (Newton on the dual part)
                        if (std::fabs(value_of(dt)) < 1e-15) {
                            const T g2 = arc[0](t) - target;
                            t -= g2 / hypot(a * sin(t), b * cos(t));
                            break;
                        }
                    }
                }
                const T ct = cos(t), stt = sin(t);
                const T mx = b * ct, my = a * stt, mn = hypot(mx, my);
                rb[2 * l] = a * ct;
                rb[2 * l + 1] = b * stt;
                nb[2 * l] = mx / mn;
                nb[2 * l + 1] = my / mn;
                S[l] = P / (double)n;
            }
            if (d.shape == LBM_SHAPE_CIRCLE) {
                out->area = M_PI * a * a;
                out->inertia_per_mass = 0.5 * a * a;
                out->rcirc = value_of(a);
            } else {
                out->area = M_PI * a * b;
                out->inertia_per_mass = 0.25 * (a * a + b * b);
                out->rcirc = std::max(value_of(a), value_of(b));
            }
            break;
        }
        default: {
            std::vector<T> vx, vy;
            if (d.shape == LBM_SHAPE_TRIANGLE) {
                const T R = D0 / std::sqrt(3.0);
                for (int j = 0; j < 3; ++j) {
                    const double ang = M_PI / 2 + 2.0 * M_PI * j / 3.0;
                    vx.push_back(R * std::cos(ang));
                    vy.push_back(R * std::sin(ang));
                }
                out->area = (std::sqrt(3.0) / 4.0) * D0 * D0;
                out->inertia_per_mass = D0 * D0 / 12.0;
                out->rcirc = value_of(R);
            } else {
                const T w = D0, hh = d.shape == LBM_SHAPE_SQUARE ? D0 : D1;
                const T px[4] = {-0.5 * w, 0.5 * w, 0.5 * w, -0.5 * w};
                const T py[4] = {-0.5 * hh, -0.5 * hh, 0.5 * hh, 0.5 * hh};
                vx.assign(px, px + 4);
                vy.assign(py, py + 4);
                out->area = w * hh;
                out->inertia_per_mass = (w * w + hh * hh) / 12.0;
                out->rcirc = 0.5 * std::hypot(value_of(w), value_of(hh));
            }
            const int nv = (int)vx.size();
            double P = 0;
            for (int j = 0; j < nv; ++j)
                P += std::hypot(value_of(vx[(j + 1) % nv] - vx[j]), value_of(vy[(j + 1) % nv] - vy[j]));
            const double h = d.n_markers > 0 ? P / d.n_markers : h0;
            for (int j = 0; j < nv; ++j) {
                const T ex = vx[(j + 1) % nv] - vx[j], ey = vy[(j + 1) % nv] - vy[j];
                const T L = hypot(ex, ey);
                int cnt = (int)std::lround(value_of(L) / h);
                if (cnt < 1) cnt = 1;
                if (n + cnt > cap) return -1;
                for (int m = 0; m < cnt; ++m, ++n) {
                    const double s = (m + 0.5) / cnt;
                    rb[2 * n] = vx[j] + s * ex;
                    rb[2 * n + 1] = vy[j] + s * ey;
                    nb[2 * n] = ey / L;  // vertices counter-clockwise: outward = (ey, -ex)/L
                    nb[2 * n + 1] = -ex / L;
                    S[n] = L / (double)cnt;
                }
            }
            break;
        }
    }
    out->n = n;
    return n;
}

template int make_shape_t<double>(const lbm_particle_desc&, const double*, double, double*, double*,
                                  double*, int, ShapeOutT<double>*);
template int make_shape_t<TD>(const lbm_particle_desc&, const TD*, double, TD*, TD*, TD*, int,
                              ShapeOutT<TD>*);

int make_shape(const lbm_particle_desc& d, double spacing, double* rb, double* nb, double* S,
               int cap, ShapeOut* out) {
    return make_shape_t<double>(d, d.dim, spacing, rb, nb, S, cap, out);
}

}  // namespace lbib
