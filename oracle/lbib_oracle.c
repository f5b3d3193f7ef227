/*
 * lbib_oracle.c -- plain FP64 CPU oracle of the coupled LB-IB time step of
 * arXiv:1606.01805, Section 2 ("Method").
 *
 * TEST INFRASTRUCTURE ONLY: it checks the CUDA path and is never part of it.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline and
 * reference legs load it.  It shares no code, table or header with the CUDA
 * library.
 *
 * One call of ob_step() advances the state from level n-1 to level n in the
 * order of Sections 2.1-2.3 (weak, explicit coupling):
 *   1. pull-streaming of the post-collision populations (Eq. 4) and the
 *      Zou-He known-velocity completion at wall nodes (Section 2.1, end);
 *   2. density and velocity moments (Eqs. 6-7) without the immersed-boundary
 *      force of level n (the constant body force enters with its half step);
 *   3. hydrodynamic force and torque on each particle from probes placed
 *      1.2 dx along the outward normals (Eqs. 13-14, Section 2.3), then the
 *      second-order rigid-body update (Eqs. 15-16);
 *   4. Lagrangian markers at level n, MLS interpolation of the lattice
 *      velocity to them (Eqs. 8-10), direct-forcing marker force (Eq. 11),
 *      spreading to the lattice (Eq. 12);
 *   5. BGK collision with the Guo forcing term (Eqs. 2, 4, 5).
 * Readings of silent or garbled passages are stated next to the code.
 */
#include "lbib_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OB_MAXP 4096

typedef struct {
    int shape;
    double dim[2];
    double rho_s, area, mass, inertia;
    int nm;
    double* rb; /* body-frame marker positions, 2 per marker */
    double* nb; /* body-frame outward unit normals, 2 per marker */
    double* S;  /* arc length carried by each marker */
    /* history: index 0 = latest level, 1 = the level before it */
    double X[2][2], th[2], U[2][2], W[2];
    double F[2], M; /* hydrodynamic force and torque of the latest step */
    long nupd;      /* rigid-body updates done */
} ob_particle;

struct ob_sim {
    ob_config c;
    double nu;
    int e[9][2];
    double w[9];
    double* f;     /* pre-collision populations of the current level */
    double* fpost; /* post-collision populations (the stored state) */
    double *rho, *ux, *uy;
    double* flb; /* immersed-boundary body force, 2 * nx * ny */
    int np;
    ob_particle p[OB_MAXP];
    long step;
    char msg[256];
};

static const double CS2 = 1.0 / 3.0; /* c_s^2, c_s = 1/sqrt(3) (Section 2.1) */
static const double RW = 2.6;        /* MLS support side r_w (Section 2.2) */
static const double ALPHA = 0.3;     /* exponential weight parameter, Eq. 10 */
static const double PROBE = 1.2;     /* probe length along the normal (Section 2.3) */

static size_t IDX(const ob_sim* s, int i, int x, int y) {
    return ((size_t)i * s->c.ny + (size_t)y) * s->c.nx + (size_t)x;
}

/* ------------------------------------------------------------------ */
/* D2Q9 lattice (Eq. 3 and the weights below it)                      */
/* ------------------------------------------------------------------ */
void ob_lattice(int e[9][2], double w[9]) {
    const double pi = acos(-1.0);
    e[0][0] = 0;
    e[0][1] = 0;
    w[0] = 4.0 / 9.0;
    for (int i = 1; i <= 4; ++i) {
        double a = (i - 1) * pi / 2.0;
        e[i][0] = (int)lround(cos(a));
        e[i][1] = (int)lround(sin(a));
        w[i] = 1.0 / 9.0;
    }
    for (int i = 5; i <= 8; ++i) {
        double a = (2 * i - 9) * pi / 4.0;
        e[i][0] = (int)lround(sqrt(2.0) * cos(a));
        e[i][1] = (int)lround(sqrt(2.0) * sin(a));
        w[i] = 1.0 / 36.0;
    }
}

/* the table of Eq. 3, evaluated once */
static int LAT_E[9][2];
static double LAT_W[9];
static int LAT_READY = 0;
static void lattice_cached(const int (**e)[2], const double** w) {
    if (!LAT_READY) {
        ob_lattice(LAT_E, LAT_W);
        LAT_READY = 1;
    }
    *e = (const int(*)[2])LAT_E;
    *w = LAT_W;
}

static int ob_dir(const int e[9][2], int ex, int ey) {
    for (int i = 0; i < 9; ++i)
        if (e[i][0] == ex && e[i][1] == ey) return i;
    return -1;
}

/* Maxwell-Boltzmann equilibrium projected on second-order Hermite space, Eq. 2 */
void ob_feq(double rho, double ux, double uy, double feq[9]) {
    const int(*e)[2];
    const double* w;
    lattice_cached(&e, &w);
    double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double eu = e[i][0] * ux + e[i][1] * uy;
        feq[i] = w[i] * rho * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Guo forcing term, Eq. 5: (1 - 1/2tau) w_i [(e_i - u)/cs^2 + (e_i.u) e_i/cs^4] . F */
void ob_guo_term(double ux, double uy, double tau, double Fx, double Fy, double Fi[9]) {
    const int(*e)[2];
    const double* w;
    lattice_cached(&e, &w);
    for (int i = 0; i < 9; ++i) {
        double eu = e[i][0] * ux + e[i][1] * uy;
        double bx = (e[i][0] - ux) / CS2 + eu * e[i][0] / (CS2 * CS2);
        double by = (e[i][1] - uy) / CS2 + eu * e[i][1] / (CS2 * CS2);
        Fi[i] = (1.0 - 1.0 / (2.0 * tau)) * w[i] * (bx * Fx + by * Fy);
    }
}

/* Forced BGK collision, Eq. 4 with the moments of Eqs. 6-7.  Reading of
 * Eq. 7: the printed per-population term is the half-step of the body force,
 * rho u = sum f e + F/2 (Guo et al. 2002, the work Eq. 5 follows). */
void ob_collide(const double f[9], double tau, double Fx, double Fy, double f_out[9]) {
    const int(*e)[2];
    const double* w;
    lattice_cached(&e, &w);
    double rho = 0, jx = 0, jy = 0;
    for (int i = 0; i < 9; ++i) {
        rho += f[i];
        jx += f[i] * e[i][0];
        jy += f[i] * e[i][1];
    }
    double ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho;
    double feq[9], Fi[9];
    ob_feq(rho, ux, uy, feq);
    ob_guo_term(ux, uy, tau, Fx, Fy, Fi);
    for (int i = 0; i < 9; ++i) f_out[i] = f[i] - (f[i] - feq[i]) / tau + Fi[i];
}

/* ------------------------------------------------------------------ */
/* Streaming and the Zou-He known-velocity walls (Section 2.1)         */
/* ------------------------------------------------------------------ */
static int xwall(const ob_sim* s) { return s->c.bc[0] == OB_VELOCITY; }
static int ywall(const ob_sim* s) { return s->c.bc[2] == OB_VELOCITY; }

/* pull the populations arriving at (x, y) from the post-collision field;
   unknown ones (source outside a wall) are left at zero */
static void pull(const ob_sim* s, const double* fp, int x, int y, double f[9]) {
    int nx = s->c.nx, ny = s->c.ny;
    for (int i = 0; i < 9; ++i) {
        int sx = x - s->e[i][0], sy = y - s->e[i][1];
        if (sx < 0 || sx >= nx) {
            if (xwall(s)) { f[i] = 0.0; continue; }
            sx = (sx + nx) % nx;
        }
        if (sy < 0 || sy >= ny) {
            if (ywall(s)) { f[i] = 0.0; continue; }
            sy = (sy + ny) % ny;
        }
        f[i] = fp[IDX(s, i, sx, sy)];
    }
}

/*
 * Zou & He (1997) completion on the wall node itself.  The paper cites it
 * without printing it.  Readings:
 *  - the prescribed velocity is the wall's, and it is the *forced* velocity
 *    of Eq. 7 that must equal it, so the target momentum is
 *    J = rho u_w - g_f/2 with g_f the constant fluid body force (the
 *    immersed-boundary force of the level is not known yet at streaming);
 *  - the tangential unknowns follow the non-equilibrium bounce-back of the
 *    normal population plus the tangential momentum correction.
 */
static void zouhe_bottom(double f[9], double ux, double uy, double gx, double gy) {
    double K0 = f[0] + f[1] + f[3], Km = f[4] + f[7] + f[8];
    double rho = (K0 + 2.0 * Km - 0.5 * gy) / (1.0 - uy);
    double Jx = rho * ux - 0.5 * gx, Jy = rho * uy - 0.5 * gy;
    f[2] = f[4] + (2.0 / 3.0) * Jy;
    f[5] = f[7] - 0.5 * (f[1] - f[3]) + 0.5 * Jx + Jy / 6.0;
    f[6] = f[8] + 0.5 * (f[1] - f[3]) - 0.5 * Jx + Jy / 6.0;
}
static void zouhe_top(double f[9], double ux, double uy, double gx, double gy) {
    double K0 = f[0] + f[1] + f[3], Kp = f[2] + f[5] + f[6];
    double rho = (K0 + 2.0 * Kp + 0.5 * gy) / (1.0 + uy);
    double Jx = rho * ux - 0.5 * gx, Jy = rho * uy - 0.5 * gy;
    f[4] = f[2] - (2.0 / 3.0) * Jy;
    f[7] = f[5] + 0.5 * (f[1] - f[3]) - 0.5 * Jx - Jy / 6.0;
    f[8] = f[6] - 0.5 * (f[1] - f[3]) + 0.5 * Jx - Jy / 6.0;
}
static void zouhe_left(double f[9], double ux, double uy, double gx, double gy) {
    double K0 = f[0] + f[2] + f[4], Km = f[3] + f[6] + f[7];
    double rho = (K0 + 2.0 * Km - 0.5 * gx) / (1.0 - ux);
    double Jx = rho * ux - 0.5 * gx, Jy = rho * uy - 0.5 * gy;
    f[1] = f[3] + (2.0 / 3.0) * Jx;
    f[5] = f[7] - 0.5 * (f[2] - f[4]) + 0.5 * Jy + Jx / 6.0;
    f[8] = f[6] + 0.5 * (f[2] - f[4]) - 0.5 * Jy + Jx / 6.0;
}
static void zouhe_right(double f[9], double ux, double uy, double gx, double gy) {
    double K0 = f[0] + f[2] + f[4], Kp = f[1] + f[5] + f[8];
    double rho = (K0 + 2.0 * Kp + 0.5 * gx) / (1.0 + ux);
    double Jx = rho * ux - 0.5 * gx, Jy = rho * uy - 0.5 * gy;
    f[3] = f[1] - (2.0 / 3.0) * Jx;
    f[7] = f[5] + 0.5 * (f[2] - f[4]) - 0.5 * Jy - Jx / 6.0;
    f[6] = f[8] - 0.5 * (f[2] - f[4]) + 0.5 * Jy - Jx / 6.0;
}

/*
 * Corner of two walls (needed by the closed sedimentation box; the paper is
 * silent).  Reading: the density is that of the diagonal interior
 * neighbour at the same level; the axis and inward-diagonal unknowns follow
 * non-equilibrium bounce-back; the two remaining ("buried") diagonal
 * populations take the rest of the mass, split so that both momentum
 * components are met.  The corner moves with the wall along y.
 */
static void zouhe_corner(const ob_sim* s, double f[9], int sx, int sy, double rho, double ux,
                         double uy, double gx, double gy) {
    const int(*e)[2] = (const int(*)[2])s->e;
    double Jx = rho * ux - 0.5 * gx, Jy = rho * uy - 0.5 * gy;
    int ax = ob_dir(e, sx, 0), axo = ob_dir(e, -sx, 0);
    int ay = ob_dir(e, 0, sy), ayo = ob_dir(e, 0, -sy);
    int dg = ob_dir(e, sx, sy), dgo = ob_dir(e, -sx, -sy);
    int ba = ob_dir(e, -sx, sy), bb = ob_dir(e, sx, -sy);
    f[ax] = f[axo] + (2.0 / 3.0) * sx * Jx;
    f[ay] = f[ayo] + (2.0 / 3.0) * sy * Jy;
    f[dg] = f[dgo] + (sx * Jx + sy * Jy) / 6.0;
    double rest = rho;
    for (int i = 0; i < 9; ++i)
        if (i != ba && i != bb) rest -= f[i];
    double diff = (sx * Jx - sy * Jy) / 6.0; /* f[bb] - f[ba] */
    f[ba] = 0.5 * (rest - diff);
    f[bb] = 0.5 * (rest + diff);
}

/* streaming (Eq. 4, left-hand side, in pull form) plus wall completion */
static void stream(const ob_sim* s, const double* fp, double* fout) {
    int nx = s->c.nx, ny = s->c.ny;
    double gx = s->c.body_force[0], gy = s->c.body_force[1];
    double f[9];
#pragma omp parallel for private(f)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            pull(s, fp, x, y, f);
            int bot = ywall(s) && y == 0, top = ywall(s) && y == ny - 1;
            int lef = xwall(s) && x == 0, rig = xwall(s) && x == nx - 1;
            if ((bot || top) && (lef || rig)) {
                /* corner: density of the diagonal interior neighbour */
                int sx = lef ? 1 : -1, sy = bot ? 1 : -1;
                double g[9];
                pull(s, fp, x + sx, y + sy, g);
                double rho = 0;
                for (int i = 0; i < 9; ++i) rho += g[i];
                const double* uw = s->c.wall_u[bot ? 2 : 3];
                zouhe_corner(s, f, sx, sy, rho, uw[0], uw[1], gx, gy);
            } else if (bot) {
                zouhe_bottom(f, s->c.wall_u[2][0], s->c.wall_u[2][1], gx, gy);
            } else if (top) {
                zouhe_top(f, s->c.wall_u[3][0], s->c.wall_u[3][1], gx, gy);
            } else if (lef) {
                zouhe_left(f, s->c.wall_u[0][0], s->c.wall_u[0][1], gx, gy);
            } else if (rig) {
                zouhe_right(f, s->c.wall_u[1][0], s->c.wall_u[1][1], gx, gy);
            }
            for (int i = 0; i < 9; ++i) fout[IDX(s, i, x, y)] = f[i];
        }
}

/* Eqs. 6-7 without the immersed-boundary force: rho, u* = (sum f e + g_f/2)/rho */
static void moments(const ob_sim* s, const double* f, double* rho, double* ux, double* uy) {
    int nx = s->c.nx, ny = s->c.ny;
#pragma omp parallel for
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double r = 0, jx = 0, jy = 0;
            for (int i = 0; i < 9; ++i) {
                double v = f[IDX(s, i, x, y)];
                r += v;
                jx += v * s->e[i][0];
                jy += v * s->e[i][1];
            }
            size_t k = (size_t)y * nx + x;
            rho[k] = r;
            ux[k] = (jx + 0.5 * s->c.body_force[0]) / r;
            uy[k] = (jy + 0.5 * s->c.body_force[1]) / r;
        }
}

/* ------------------------------------------------------------------ */
/* Moving least squares (Section 2.2, Eqs. 8-10 and 17-20)            */
/* ------------------------------------------------------------------ */
double ob_weight(int weight, double r) {
    const double pi = acos(-1.0);
    if (r > 1.0) return 0.0;
    switch (weight) {
        case OB_W_CUBIC: /* Eq. 17 as printed */
            return 2.0 / 3.0 - 4.0 * r * r + 4.0 * r * r * r;
        case OB_W_QUARTIC: /* Eq. 18 */
            return 1.0 - 6.0 * r * r + 8.0 * r * r * r - 3.0 * r * r * r * r;
        case OB_W_COSINE: /* Eq. 19 as printed */
            return 0.25 * (1.0 + cos(pi * r / 2.0));
        case OB_W_POLY: {
            /* Eq. 20: as printed the second branch takes the square root of a
               negative number on (0.5, 0.79).  Reading: the breakpoints are
               those of the 4-point kernel it is, in the variable q = 2 r. */
            double q = 2.0 * r;
            if (q <= 1.0) return (3.0 - 2.0 * q + sqrt(1.0 + 4.0 * q - 4.0 * q * q)) / 8.0;
            return (5.0 - 2.0 * q - sqrt(-7.0 + 12.0 * q - 4.0 * q * q)) / 8.0;
        }
        default: /* Eq. 10 */
            return exp(-(r / ALPHA) * (r / ALPHA));
    }
}

/*
 * MLS transfer operator at x = (px, py).  The nine Eulerian points are the
 * 3x3 block of nodes around the nearest node (Figure 1: the nine points
 * closest to the marker).  The linear basis p = (1, x, y) is written in
 * coordinates relative to the evaluation point, so p(x) = (1, 0, 0); the
 * minimiser of Eq. 9 gives coefficients a = A^-1 B u with A = sum W p p^T and
 * B = [W_k p_k].  Row 0 of A^-1 B is phi_k (Eq. 8); rows 1 and 2 are the
 * weights of the linear coefficients, i.e. the x and y derivatives of the
 * fit.  The 3x3 system is solved by Gaussian elimination with partial
 * pivoting.
 */
int ob_mls(int weight, double px, double py, int ix[9], int iy[9], double phi[27]) {
    int i0 = (int)floor(px + 0.5), j0 = (int)floor(py + 0.5);
    double A[3][3] = {{0}}, B[3][9];
    for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) {
            int k = (b + 1) * 3 + (a + 1);
            ix[k] = i0 + a;
            iy[k] = j0 + b;
            double dx = ix[k] - px, dy = iy[k] - py;
            double r = sqrt(dx * dx + dy * dy) / RW;
            double W = ob_weight(weight, r);
            double p[3] = {1.0, dx, dy};
            for (int m = 0; m < 3; ++m) {
                B[m][k] = W * p[m];
                for (int n = 0; n < 3; ++n) A[m][n] += W * p[m] * p[n];
            }
        }
    /* solve A X = B */
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return OB_EINVAL;
        if (piv != col) {
            for (int n = 0; n < 3; ++n) {
                double t = A[col][n];
                A[col][n] = A[piv][n];
                A[piv][n] = t;
            }
            for (int k = 0; k < 9; ++k) {
                double t = B[col][k];
                B[col][k] = B[piv][k];
                B[piv][k] = t;
            }
        }
        for (int r = 0; r < 3; ++r) {
            if (r == col) continue;
            double fct = A[r][col] / A[col][col];
            for (int n = 0; n < 3; ++n) A[r][n] -= fct * A[col][n];
            for (int k = 0; k < 9; ++k) B[r][k] -= fct * B[col][k];
        }
    }
    for (int m = 0; m < 3; ++m)
        for (int k = 0; k < 9; ++k) phi[m * 9 + k] = B[m][k] / A[m][m];
    return OB_OK;
}

/* map an unwrapped node to a field index; -1 if it leaves a wall side */
static long node_index(const ob_sim* s, int x, int y) {
    int nx = s->c.nx, ny = s->c.ny;
    if (x < 0 || x >= nx) {
        if (xwall(s)) return -1;
        x = ((x % nx) + nx) % nx;
    }
    if (y < 0 || y >= ny) {
        if (ywall(s)) return -1;
        y = ((y % ny) + ny) % ny;
    }
    return (long)y * nx + x;
}

/* ------------------------------------------------------------------ */
/* Shapes and Lagrangian markers (Sections 3 and 4.1)                  */
/* ------------------------------------------------------------------ */
static double ell_speed(double a, double b, double t) {
    return sqrt(a * a * sin(t) * sin(t) + b * b * cos(t) * cos(t));
}
/* arc length of (a cos t, b sin t) from 0 to t, composite Simpson */
static double ell_arc(double a, double b, double t) {
    const int m = 8192;
    double h = t / m, acc = ell_speed(a, b, 0.0) + ell_speed(a, b, t);
    for (int k = 1; k < m; ++k) acc += (k % 2 ? 4.0 : 2.0) * ell_speed(a, b, k * h);
    return acc * h / 3.0;
}

/*
 * Marker layout (the paper: surface "uniformly discretized", spacing about
 * 0.3 dx; the 3-D "triangles" of Section 2.3 become a 2-D ring).  Reading:
 * markers sit at the midpoints of equal-length pieces of the perimeter and
 * carry that length as S_l; the normal is the analytic one for circle and
 * ellipse and the face normal for polygons, each face being cut into its
 * own equal pieces so that no marker straddles a corner.
 */
static int make_markers(ob_particle* q, const ob_particle_desc* d, double spacing) {
    const double pi = acos(-1.0);
    double h = spacing > 0 ? spacing : 0.3;
    if (d->shape == OB_CIRCLE || d->shape == OB_ELLIPSE) {
        double a, b;
        if (d->shape == OB_CIRCLE) {
            a = b = 0.5 * d->dim[0];
        } else {
            a = 0.5 * d->dim[0];
            b = 0.5 * d->dim[1];
        }
        double P = (d->shape == OB_CIRCLE) ? 2.0 * pi * a : ell_arc(a, b, 2.0 * pi);
        int n = d->n_markers > 0 ? d->n_markers : (int)lround(P / h);
        if (n < 8) n = 8;
        q->nm = n;
        q->rb = malloc(sizeof(double) * 2 * n);
        q->nb = malloc(sizeof(double) * 2 * n);
        q->S = malloc(sizeof(double) * n);
        for (int l = 0; l < n; ++l) {
            double t;
            if (d->shape == OB_CIRCLE) {
                t = 2.0 * pi * (l + 0.5) / n;
            } else {
                double target = (l + 0.5) * P / n;
                t = 2.0 * pi * target / P;
                for (int it = 0; it < 50; ++it) {
                    double dt = (ell_arc(a, b, t) - target) / ell_speed(a, b, t);
                    t -= dt;
                    if (fabs(dt) < 1e-15) break;
                }
            }
            double nx = b * cos(t), ny = a * sin(t), nn = sqrt(nx * nx + ny * ny);
            q->rb[2 * l] = a * cos(t);
            q->rb[2 * l + 1] = b * sin(t);
            q->nb[2 * l] = nx / nn;
            q->nb[2 * l + 1] = ny / nn;
            q->S[l] = P / n;
        }
        return 0;
    }
    double vx[4], vy[4];
    int nv;
    if (d->shape == OB_TRIANGLE) {
        double R = d->dim[0] / sqrt(3.0);
        nv = 3;
        for (int j = 0; j < 3; ++j) {
            double ang = pi / 2.0 + j * 2.0 * pi / 3.0;
            vx[j] = R * cos(ang);
            vy[j] = R * sin(ang);
        }
    } else {
        double w = d->dim[0], hh = (d->shape == OB_SQUARE) ? d->dim[0] : d->dim[1];
        nv = 4;
        vx[0] = -w / 2; vy[0] = -hh / 2;
        vx[1] = w / 2;  vy[1] = -hh / 2;
        vx[2] = w / 2;  vy[2] = hh / 2;
        vx[3] = -w / 2; vy[3] = hh / 2;
    }
    double P = 0;
    for (int j = 0; j < nv; ++j) P += hypot(vx[(j + 1) % nv] - vx[j], vy[(j + 1) % nv] - vy[j]);
    if (d->n_markers > 0) h = P / d->n_markers;
    int cnt[4], n = 0;
    for (int j = 0; j < nv; ++j) {
        double L = hypot(vx[(j + 1) % nv] - vx[j], vy[(j + 1) % nv] - vy[j]);
        cnt[j] = (int)lround(L / h);
        if (cnt[j] < 1) cnt[j] = 1;
        n += cnt[j];
    }
    q->nm = n;
    q->rb = malloc(sizeof(double) * 2 * n);
    q->nb = malloc(sizeof(double) * 2 * n);
    q->S = malloc(sizeof(double) * n);
    int l = 0;
    for (int j = 0; j < nv; ++j) {
        double dx = vx[(j + 1) % nv] - vx[j], dy = vy[(j + 1) % nv] - vy[j];
        double L = hypot(dx, dy);
        for (int m = 0; m < cnt[j]; ++m, ++l) {
            double t = (m + 0.5) / cnt[j];
            q->rb[2 * l] = vx[j] + t * dx;
            q->rb[2 * l + 1] = vy[j] + t * dy;
            q->nb[2 * l] = dy / L; /* counter-clockwise vertices: outward = (dy, -dx) */
            q->nb[2 * l + 1] = -dx / L;
            q->S[l] = L / cnt[j];
        }
    }
    return 0;
}

/* area and polar moment of inertia per unit depth about the centroid */
static void shape_props(ob_particle* q) {
    const double pi = acos(-1.0);
    double A, k; /* I = m * k */
    switch (q->shape) {
        case OB_CIRCLE: A = pi * q->dim[0] * q->dim[0] / 4.0; k = q->dim[0] * q->dim[0] / 8.0; break;
        case OB_ELLIPSE: {
            double a = q->dim[0] / 2, b = q->dim[1] / 2;
            A = pi * a * b;
            k = (a * a + b * b) / 4.0;
            break;
        }
        case OB_RECT: A = q->dim[0] * q->dim[1]; k = (q->dim[0] * q->dim[0] + q->dim[1] * q->dim[1]) / 12.0; break;
        case OB_SQUARE: A = q->dim[0] * q->dim[0]; k = q->dim[0] * q->dim[0] / 6.0; break;
        default: A = sqrt(3.0) / 4.0 * q->dim[0] * q->dim[0]; k = q->dim[0] * q->dim[0] / 12.0; break;
    }
    q->area = A;
    q->mass = q->rho_s * A;
    q->inertia = q->mass * k;
}

/* world-frame marker l of particle q at history level h */
static void marker_world(const ob_particle* q, int h, int l, double x[2], double n[2]) {
    double c = cos(q->th[h]), sn = sin(q->th[h]);
    double rx = q->rb[2 * l], ry = q->rb[2 * l + 1];
    x[0] = q->X[h][0] + c * rx - sn * ry;
    x[1] = q->X[h][1] + sn * rx + c * ry;
    n[0] = c * q->nb[2 * l] - sn * q->nb[2 * l + 1];
    n[1] = sn * q->nb[2 * l] + c * q->nb[2 * l + 1];
}

/* rigid-body velocity at a marker, level h: U + omega e_z x (x_l - X) */
static void marker_velocity(const ob_particle* q, int h, int l, double v[2]) {
    double x[2], n[2];
    marker_world(q, h, l, x, n);
    v[0] = q->U[h][0] - q->W[h] * (x[1] - q->X[h][1]);
    v[1] = q->U[h][1] + q->W[h] * (x[0] - q->X[h][0]);
}

/* ------------------------------------------------------------------ */
/* Fluid-structure interaction (Section 2.3)                           */
/* ------------------------------------------------------------------ */
/*
 * Eqs. 13-14 on the body at its latest level.  Readings:
 *  - pressure p = c_s^2 (rho - 1): the paper's p = c_s^2 rho up to the
 *    reference constant, which integrates to zero over a closed ring;
 *  - probe values come from the MLS fit at x_l + 1.2 n_l; the velocity
 *    derivatives are the linear coefficients of that fit;
 *  - viscous stress tau = rho nu (grad u + grad u^T) with the probe density;
 *  - the marker pressure p_l = p_P + rho_P * 1.2 * (d_t u_l . n_l): the
 *    printed "p_P + d_t u . n" with the probe length and density that make
 *    it a pressure; d_t u_l is the backward difference of the marker's
 *    rigid-body velocity over the two stored levels;
 *  - r_l = x_l - X_c and the 2-D moment is r_x t_y - r_y t_x.
 */
int ob_stress_force(ob_sim* s, int pi, const double* rho, const double* ux, const double* uy,
                    double F[2], double* M) {
    ob_particle* q = &s->p[pi];
    double Fx = 0, Fy = 0, Mz = 0;
    for (int l = 0; l < q->nm; ++l) {
        double x[2], n[2];
        marker_world(q, 0, l, x, n);
        double xp = x[0] + PROBE * n[0], yp = x[1] + PROBE * n[1];
        int ix[9], iy[9];
        double phi[27];
        if (ob_mls(s->c.weight, xp, yp, ix, iy, phi) != OB_OK) return OB_EINVAL;
        double r = 0, dux[2] = {0, 0}, duy[2] = {0, 0};
        for (int k = 0; k < 9; ++k) {
            long j = node_index(s, ix[k], iy[k]);
            if (j < 0) {
                snprintf(s->msg, sizeof s->msg, "probe support of particle %d leaves the domain", pi);
                return OB_EDOMAIN;
            }
            r += phi[k] * rho[j];
            dux[0] += phi[9 + k] * ux[j];
            dux[1] += phi[18 + k] * ux[j];
            duy[0] += phi[9 + k] * uy[j];
            duy[1] += phi[18 + k] * uy[j];
        }
        double v1[2], v2[2];
        marker_velocity(q, 0, l, v1);
        marker_velocity(q, 1, l, v2);
        double acc_n = (v1[0] - v2[0]) * n[0] + (v1[1] - v2[1]) * n[1];
        double p = CS2 * (r - 1.0) + r * PROBE * acc_n;
        double mu = r * s->nu;
        double txx = 2.0 * mu * dux[0], tyy = 2.0 * mu * duy[1], txy = mu * (dux[1] + duy[0]);
        double tx = txx * n[0] + txy * n[1] - p * n[0];
        double ty = txy * n[0] + tyy * n[1] - p * n[1];
        double rx = x[0] - q->X[0][0], ry = x[1] - q->X[0][1];
        Fx += tx * q->S[l];
        Fy += ty * q->S[l];
        Mz += (rx * ty - ry * tx) * q->S[l];
    }
    F[0] = Fx;
    F[1] = Fy;
    *M = Mz;
    return OB_OK;
}

/*
 * Rigid-body update, Eqs. 15-16 (BDF2 form of the "explicit second-order
 * Euler" scheme).  Readings: the acceleration adds the buoyancy-corrected
 * gravity (rho_s - 1) A g to the hydrodynamic force; position and angle are
 * advanced with the same two-level form using the new velocities; the first
 * update (one stored level only) is the one-level form u1 = u0 + a,
 * x1 = x0 + u1.
 */
void ob_rigid_update(ob_sim* s, int pi, const double F[2], double M) {
    ob_particle* q = &s->p[pi];
    double ax = (F[0] + (q->rho_s - 1.0) * q->area * s->c.gravity[0]) / q->mass;
    double ay = (F[1] + (q->rho_s - 1.0) * q->area * s->c.gravity[1]) / q->mass;
    double al = M / q->inertia;
    double U[2], W, X[2], th;
    if (q->nupd == 0) {
        U[0] = q->U[0][0] + ax;
        U[1] = q->U[0][1] + ay;
        W = q->W[0] + al;
        X[0] = q->X[0][0] + U[0];
        X[1] = q->X[0][1] + U[1];
        th = q->th[0] + W;
    } else {
        U[0] = 2.0 / 3.0 * (2.0 * q->U[0][0] - 0.5 * q->U[1][0] + ax);
        U[1] = 2.0 / 3.0 * (2.0 * q->U[0][1] - 0.5 * q->U[1][1] + ay);
        W = 2.0 / 3.0 * (2.0 * q->W[0] - 0.5 * q->W[1] + al);
        X[0] = 2.0 / 3.0 * (2.0 * q->X[0][0] - 0.5 * q->X[1][0] + U[0]);
        X[1] = 2.0 / 3.0 * (2.0 * q->X[0][1] - 0.5 * q->X[1][1] + U[1]);
        th = 2.0 / 3.0 * (2.0 * q->th[0] - 0.5 * q->th[1] + W);
    }
    q->X[1][0] = q->X[0][0];
    q->X[1][1] = q->X[0][1];
    q->th[1] = q->th[0];
    q->U[1][0] = q->U[0][0];
    q->U[1][1] = q->U[0][1];
    q->W[1] = q->W[0];
    q->X[0][0] = X[0];
    q->X[0][1] = X[1];
    q->th[0] = th;
    q->U[0][0] = U[0];
    q->U[0][1] = U[1];
    q->W[0] = W;
    q->F[0] = F[0];
    q->F[1] = F[1];
    q->M = M;
    q->nupd += 1;
}

/*
 * Markers at the latest level: MLS velocity (Eq. 8), direct-forcing force
 * F_l = U_b,l - U_l (Eq. 11, dt = 1; no density factor, as printed) and
 * spreading f_lb(k) += c_l phi_k F_l (Eq. 12).  Reading of c_l: total-force
 * conservation between the Lagrangian ring (arc S_l, unit thickness) and the
 * unit-area lattice cells gives c_l = S_l, since the phi_k sum to one.
 */
int ob_spread_only(ob_sim* s, int pi, const double* ux, const double* uy, double* flb,
                   double sumSF[2], double* sum_torque) {
    ob_particle* q = &s->p[pi];
    size_t nc = (size_t)s->c.nx * s->c.ny;
    double tx = 0, ty = 0, tq = 0;
    for (int l = 0; l < q->nm; ++l) {
        double x[2], n[2], ub[2];
        marker_world(q, 0, l, x, n);
        marker_velocity(q, 0, l, ub);
        int ix[9], iy[9];
        double phi[27];
        if (ob_mls(s->c.weight, x[0], x[1], ix, iy, phi) != OB_OK) return OB_EINVAL;
        long j[9];
        double U[2] = {0, 0};
        for (int k = 0; k < 9; ++k) {
            j[k] = node_index(s, ix[k], iy[k]);
            if (j[k] < 0) {
                snprintf(s->msg, sizeof s->msg, "marker support of particle %d leaves the domain", pi);
                return OB_EDOMAIN;
            }
            U[0] += phi[k] * ux[j[k]];
            U[1] += phi[k] * uy[j[k]];
        }
        double Fl[2] = {ub[0] - U[0], ub[1] - U[1]};
        for (int k = 0; k < 9; ++k) {
            flb[j[k]] += q->S[l] * phi[k] * Fl[0];
            flb[nc + j[k]] += q->S[l] * phi[k] * Fl[1];
        }
        tx += q->S[l] * Fl[0];
        ty += q->S[l] * Fl[1];
        tq += q->S[l] * (x[0] * Fl[1] - x[1] * Fl[0]);
    }
    if (sumSF) {
        sumSF[0] = tx;
        sumSF[1] = ty;
    }
    if (sum_torque) *sum_torque = tq;
    return OB_OK;
}

/* ------------------------------------------------------------------ */
/* Simulation object                                                   */
/* ------------------------------------------------------------------ */
static void init_fields(ob_sim* s) {
    const double pi = acos(-1.0);
    int nx = s->c.nx, ny = s->c.ny;
    double H = ny - 1;
#pragma omp parallel for
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double rho = 1.0, ux = 0.0, uy = 0.0;
            if (s->c.init == OB_INIT_COUETTE) {
                /* planar Couette profile between the y walls (Section 4.1) */
                double ub = s->c.wall_u[2][0], ut = s->c.wall_u[3][0];
                ux = ub + (ut - ub) * y / H;
            } else if (s->c.init == OB_INIT_TAYLOR_GREEN) {
                double kx = 2.0 * pi / nx, ky = 2.0 * pi / ny, U0 = s->c.init_u;
                ux = -U0 * cos(kx * x) * sin(ky * y);
                uy = U0 * (kx / ky) * sin(kx * x) * cos(ky * y);
                rho = 1.0 - 0.25 * U0 * U0 / CS2 *
                                (cos(2.0 * kx * x) + (kx * kx) / (ky * ky) * cos(2.0 * ky * y));
            }
            double feq[9];
            ob_feq(rho, ux, uy, feq);
            for (int i = 0; i < 9; ++i) s->fpost[IDX(s, i, x, y)] = feq[i];
        }
}

ob_sim* ob_create(const ob_config* cfg, int* err) {
    *err = OB_EINVAL;
    if (cfg->nx < 3 || cfg->ny < 3 || !(cfg->tau > 0.5)) return NULL;
    if ((cfg->bc[0] == OB_PERIODIC) != (cfg->bc[1] == OB_PERIODIC)) return NULL;
    if ((cfg->bc[2] == OB_PERIODIC) != (cfg->bc[3] == OB_PERIODIC)) return NULL;
    ob_sim* s = calloc(1, sizeof(ob_sim));
    s->c = *cfg;
    if (!(s->c.spacing > 0)) s->c.spacing = 0.3;
    /* Reading of the viscosity relation of Section 2.1: the printed
       (2 tau - 1) dt / c_s^2 is dimensionally off; the BGK value is
       nu = c_s^2 (tau - 1/2) = (2 tau - 1)/6. */
    s->nu = CS2 * (cfg->tau - 0.5);
    ob_lattice(s->e, s->w);
    {   /* fill the shared table before any parallel loop reads it */
        const int(*e)[2];
        const double* w;
        lattice_cached(&e, &w);
    }
    size_t nc = (size_t)cfg->nx * cfg->ny;
    s->f = calloc(9 * nc, sizeof(double));
    s->fpost = calloc(9 * nc, sizeof(double));
    s->rho = calloc(nc, sizeof(double));
    s->ux = calloc(nc, sizeof(double));
    s->uy = calloc(nc, sizeof(double));
    s->flb = calloc(2 * nc, sizeof(double));
    init_fields(s);
    *err = OB_OK;
    return s;
}

void ob_destroy(ob_sim* s) {
    if (!s) return;
    for (int i = 0; i < s->np; ++i) {
        free(s->p[i].rb);
        free(s->p[i].nb);
        free(s->p[i].S);
    }
    free(s->f);
    free(s->fpost);
    free(s->rho);
    free(s->ux);
    free(s->uy);
    free(s->flb);
    free(s);
}

int ob_add_particle(ob_sim* s, const ob_particle_desc* d) {
    if (s->np >= OB_MAXP || s->step > 0) return OB_EINVAL;
    if (d->shape < OB_CIRCLE || d->shape > OB_TRIANGLE || !(d->dim[0] > 0) || !(d->rho_s > 0)) return OB_EINVAL;
    if ((d->shape == OB_ELLIPSE || d->shape == OB_RECT) && !(d->dim[1] > 0)) return OB_EINVAL;
    ob_particle* q = &s->p[s->np];
    memset(q, 0, sizeof *q);
    q->shape = d->shape;
    q->dim[0] = d->dim[0];
    q->dim[1] = d->dim[1];
    q->rho_s = d->rho_s;
    shape_props(q);
    make_markers(q, d, s->c.spacing);
    for (int h = 0; h < 2; ++h) {
        q->X[h][0] = d->xc;
        q->X[h][1] = d->yc;
        q->th[h] = d->theta;
        q->U[h][0] = d->u0[0];
        q->U[h][1] = d->u0[1];
        q->W[h] = d->omega0;
    }
    /* every marker and probe support must lie inside the walls */
    for (int l = 0; l < q->nm; ++l) {
        double x[2], n[2];
        marker_world(q, 0, l, x, n);
        for (int pass = 0; pass < 2; ++pass) {
            double px = x[0] + pass * PROBE * n[0], py = x[1] + pass * PROBE * n[1];
            int i0 = (int)floor(px + 0.5), j0 = (int)floor(py + 0.5);
            if (node_index(s, i0 - 1, j0 - 1) < 0 || node_index(s, i0 + 1, j0 + 1) < 0) {
                free(q->rb);
                free(q->nb);
                free(q->S);
                snprintf(s->msg, sizeof s->msg, "particle support leaves the domain at creation");
                return OB_EINVAL;
            }
        }
    }
    s->np += 1;
    return OB_OK;
}

int ob_step(ob_sim* s, int nsteps) {
    int nx = s->c.nx, ny = s->c.ny;
    size_t nc = (size_t)nx * ny;
    for (int it = 0; it < nsteps; ++it) {
        /* 1. stream + walls */
        stream(s, s->fpost, s->f);
        /* 2. moments of level n */
        moments(s, s->f, s->rho, s->ux, s->uy);
        /* 3. particles: force from the fluid at n on the body at n-1, update */
        for (int p = 0; p < s->np; ++p) {
            double F[2], M;
            int rc = ob_stress_force(s, p, s->rho, s->ux, s->uy, F, &M);
            if (rc != OB_OK) return rc;
            ob_rigid_update(s, p, F, M);
        }
        /* 4. markers at level n: interpolation, direct forcing, spreading */
        memset(s->flb, 0, sizeof(double) * 2 * nc);
        for (int p = 0; p < s->np; ++p) {
            int rc = ob_spread_only(s, p, s->ux, s->uy, s->flb, NULL, NULL);
            if (rc != OB_OK) return rc;
        }
        /* 5. forced collision with the total force g_f + f_lb */
        double f[9], fo[9];
#pragma omp parallel for private(f, fo)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t k = (size_t)y * nx + x;
                for (int i = 0; i < 9; ++i) f[i] = s->f[IDX(s, i, x, y)];
                double Fx = s->c.body_force[0] + s->flb[k];
                double Fy = s->c.body_force[1] + s->flb[nc + k];
                ob_collide(f, s->c.tau, Fx, Fy, fo);
                for (int i = 0; i < 9; ++i) s->fpost[IDX(s, i, x, y)] = fo[i];
            }
        s->step += 1;
    }
    return OB_OK;
}

const char* ob_last_error(const ob_sim* s) { return s->msg; }

/* Threads of the lattice loops (built with OpenMP; otherwise one).  Each
   row is computed by one thread with the same arithmetic, so the results
   do not depend on the count. */
int ob_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
int ob_nx(const ob_sim* s) { return s->c.nx; }
int ob_ny(const ob_sim* s) { return s->c.ny; }
long ob_steps_done(const ob_sim* s) { return s->step; }

void ob_get_populations(const ob_sim* s, double* f) {
    memcpy(f, s->fpost, sizeof(double) * 9 * (size_t)s->c.nx * s->c.ny);
}
void ob_set_populations(ob_sim* s, const double* f) {
    memcpy(s->fpost, f, sizeof(double) * 9 * (size_t)s->c.nx * s->c.ny);
}

int ob_get_fields(ob_sim* s, double* rho, double* ux, double* uy) {
    stream(s, s->fpost, s->f);
    moments(s, s->f, rho, ux, uy);
    return OB_OK;
}

int ob_get_particles(const ob_sim* s, ob_particle_state* out, int cap) {
    int n = s->np < cap ? s->np : cap;
    for (int i = 0; i < n; ++i) {
        const ob_particle* q = &s->p[i];
        out[i].xc = q->X[0][0];
        out[i].yc = q->X[0][1];
        out[i].theta = q->th[0];
        out[i].u[0] = q->U[0][0];
        out[i].u[1] = q->U[0][1];
        out[i].omega = q->W[0];
        out[i].F[0] = q->F[0];
        out[i].F[1] = q->F[1];
        out[i].M = q->M;
    }
    return s->np;
}

int ob_get_markers(const ob_sim* s, int p, double* rb, double* nb, double* S, int cap) {
    const ob_particle* q = &s->p[p];
    int n = q->nm < cap ? q->nm : cap;
    for (int l = 0; l < n; ++l) {
        rb[2 * l] = q->rb[2 * l];
        rb[2 * l + 1] = q->rb[2 * l + 1];
        nb[2 * l] = q->nb[2 * l];
        nb[2 * l + 1] = q->nb[2 * l + 1];
        S[l] = q->S[l];
    }
    return q->nm;
}

void ob_particle_props(const ob_sim* s, int p, double* m, double* I, double* A) {
    *m = s->p[p].mass;
    *I = s->p[p].inertia;
    *A = s->p[p].area;
}

void ob_get_force_field(const ob_sim* s, double* flb) {
    memcpy(flb, s->flb, sizeof(double) * 2 * (size_t)s->c.nx * s->c.ny);
}

void ob_set_history(ob_sim* s, int pi, const double X1[2], double th1, const double U1[2], double W1,
                    const double X2[2], double th2, const double U2[2], double W2) {
    ob_particle* q = &s->p[pi];
    q->X[0][0] = X1[0];
    q->X[0][1] = X1[1];
    q->th[0] = th1;
    q->U[0][0] = U1[0];
    q->U[0][1] = U1[1];
    q->W[0] = W1;
    q->X[1][0] = X2[0];
    q->X[1][1] = X2[1];
    q->th[1] = th2;
    q->U[1][0] = U2[0];
    q->U[1][1] = U2[1];
    q->W[1] = W2;
}
