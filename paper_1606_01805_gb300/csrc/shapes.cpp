// shapes.cpp -- Lagrangian markers and rigid-body properties of the particle
// shapes of Sections 3-4 (circle, ellipse, rectangle, square, equilateral
// triangle), in the body frame with the centroid at the origin.
//
// Markers sit at the midpoints of equal arc-length pieces of the perimeter
// and carry the piece length S_l; the normal is the analytic outward normal
// (circle, ellipse) or the face normal (polygons, each face cut into its own
// equal pieces so that no marker straddles a corner).
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

// arc length of (a cos t, b sin t) over [0, t]: composite 20-point Gauss-Legendre
double ellipse_arc(double a, double b, double t) {
    static const GaussLegendre gl(20);
    const int panels = 64;
    const double h = t / panels;
    double acc = 0;
    for (int p = 0; p < panels; ++p) {
        const double mid = (p + 0.5) * h;
        for (size_t i = 0; i < gl.x.size(); ++i) {
            const double s = mid + 0.5 * h * gl.x[i];
            acc += gl.w[i] * std::hypot(a * std::sin(s), b * std::cos(s));
        }
    }
    return 0.5 * h * acc;
}

}  // namespace

int make_shape(const lbm_particle_desc& d, double spacing, double* rb, double* nb, double* S,
               int cap, ShapeOut* out) {
    const double h0 = spacing > 0 ? spacing : 0.3;
    const double D0 = d.dim[0], D1 = d.dim[1];
    int n = 0;
    switch (d.shape) {
        case LBM_SHAPE_CIRCLE:
        case LBM_SHAPE_ELLIPSE: {
            const double a = 0.5 * D0, b = d.shape == LBM_SHAPE_CIRCLE ? 0.5 * D0 : 0.5 * D1;
            const double P = d.shape == LBM_SHAPE_CIRCLE ? M_PI * D0 : ellipse_arc(a, b, 2.0 * M_PI);
            n = d.n_markers > 0 ? d.n_markers : (int)std::lround(P / h0);
            if (n < 8) n = 8;
            if (n > cap) return -1;
            for (int l = 0; l < n; ++l) {
                double t = 2.0 * M_PI * (l + 0.5) / n;
                if (d.shape == LBM_SHAPE_ELLIPSE) {  // invert the arc length by Newton
                    const double target = (l + 0.5) * P / n;
                    for (int it = 0; it < 60; ++it) {
                        const double g = ellipse_arc(a, b, t) - target;
                        const double dt = g / std::hypot(a * std::sin(t), b * std::cos(t));
                        t -= dt;
                        if (std::fabs(dt) < 1e-15) break;
                    }
                }
                const double ct = std::cos(t), stt = std::sin(t);
                const double mx = b * ct, my = a * stt, mn = std::hypot(mx, my);
                rb[2 * l] = a * ct;
                rb[2 * l + 1] = b * stt;
                nb[2 * l] = mx / mn;
                nb[2 * l + 1] = my / mn;
                S[l] = P / n;
            }
            if (d.shape == LBM_SHAPE_CIRCLE) {
                out->area = M_PI * a * a;
                out->inertia_per_mass = 0.5 * a * a;
                out->rcirc = a;
            } else {
                out->area = M_PI * a * b;
                out->inertia_per_mass = 0.25 * (a * a + b * b);
                out->rcirc = a > b ? a : b;
            }
            break;
        }
        default: {
            std::vector<double> vx, vy;
            if (d.shape == LBM_SHAPE_TRIANGLE) {
                const double R = D0 / std::sqrt(3.0);
                for (int j = 0; j < 3; ++j) {
                    const double ang = M_PI / 2 + 2.0 * M_PI * j / 3.0;
                    vx.push_back(R * std::cos(ang));
                    vy.push_back(R * std::sin(ang));
                }
                out->area = std::sqrt(3.0) / 4.0 * D0 * D0;
                out->inertia_per_mass = D0 * D0 / 12.0;
                out->rcirc = R;
            } else {
                const double w = D0, hh = d.shape == LBM_SHAPE_SQUARE ? D0 : D1;
                const double px[4] = {-w / 2, w / 2, w / 2, -w / 2};
                const double py[4] = {-hh / 2, -hh / 2, hh / 2, hh / 2};
                vx.assign(px, px + 4);
                vy.assign(py, py + 4);
                out->area = w * hh;
                out->inertia_per_mass = (w * w + hh * hh) / 12.0;
                out->rcirc = 0.5 * std::hypot(w, hh);
            }
            const int nv = (int)vx.size();
            double P = 0;
            for (int j = 0; j < nv; ++j) P += std::hypot(vx[(j + 1) % nv] - vx[j], vy[(j + 1) % nv] - vy[j]);
            const double h = d.n_markers > 0 ? P / d.n_markers : h0;
            for (int j = 0; j < nv; ++j) {
                const double ex = vx[(j + 1) % nv] - vx[j], ey = vy[(j + 1) % nv] - vy[j];
                const double L = std::hypot(ex, ey);
                int cnt = (int)std::lround(L / h);
                if (cnt < 1) cnt = 1;
                if (n + cnt > cap) return -1;
                for (int m = 0; m < cnt; ++m, ++n) {
                    const double s = (m + 0.5) / cnt;
                    rb[2 * n] = vx[j] + s * ex;
                    rb[2 * n + 1] = vy[j] + s * ey;
                    nb[2 * n] = ey / L;  // vertices counter-clockwise: outward = (ey, -ex)/L
                    nb[2 * n + 1] = -ex / L;
                    S[n] = L / cnt;
                }
            }
            break;
        }
    }
    out->n = n;
    return n;
}

}  // namespace lbib
