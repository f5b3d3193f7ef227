/*
 * lbib_oracle.h -- plain FP64 CPU oracle of the coupled lattice-Boltzmann /
 * immersed-boundary (LB-IB) time step of Coclite, de Tullio, Pascazio and
 * Decuzzi (arXiv:1606.01805), Section 2 ("Method").
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path.  Only
 * tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg may load it.  It shares no source with the CUDA library (its own
 * tables, its own marker generators, its own boundary formulas) and never
 * includes a header of it.
 *
 * Every function computes in double precision with plain loops, in the
 * order the paper gives the steps.  Where the paper is silent or garbled,
 * the reading taken is written next to the code that implements it.
 */
#ifndef LBIB_ORACLE_H
#define LBIB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* boundary kinds per side, sides ordered x-, x+, y-, y+ */
#define OB_PERIODIC 0
#define OB_VELOCITY 1

/* initial fields */
#define OB_INIT_REST 0
#define OB_INIT_COUETTE 1
#define OB_INIT_TAYLOR_GREEN 2

/* particle shapes (Section 4.1 and 4.3) */
#define OB_CIRCLE 0
#define OB_ELLIPSE 1
#define OB_RECT 2
#define OB_SQUARE 3
#define OB_TRIANGLE 4

/* MLS weight functions: Eq. 10 (exponential) and Eqs. 17-20 */
#define OB_W_EXP 0
#define OB_W_CUBIC 1
#define OB_W_QUARTIC 2
#define OB_W_COSINE 3
#define OB_W_POLY 4

/* error codes */
#define OB_OK 0
#define OB_EINVAL 1
#define OB_EDOMAIN 7

typedef struct ob_sim ob_sim;

typedef struct {
    int nx, ny;
    double tau;
    int bc[4];            /* x-, x+, y-, y+ */
    double wall_u[4][2];  /* wall velocity per side */
    double body_force[2]; /* constant fluid body-force density g_f */
    double gravity[2];    /* gravity acting on the particles only */
    int init;             /* OB_INIT_* */
    double init_u;        /* Taylor-Green amplitude U0 */
    int weight;           /* OB_W_* */
    double spacing;       /* target marker spacing; <= 0 means 0.3 */
} ob_config;

typedef struct {
    int shape;
    double dim[2];        /* circle: D; ellipse: major, minor (full axes);
                             rect: w, h; square: side; triangle: side */
    double xc, yc, theta;
    double rho_s;
    double u0[2], omega0;
    int n_markers;        /* 0: from the target spacing */
} ob_particle_desc;

typedef struct {
    double xc, yc, theta, u[2], omega, F[2], M;
} ob_particle_state;

ob_sim* ob_create(const ob_config* cfg, int* err);
void ob_destroy(ob_sim* s);
int ob_add_particle(ob_sim* s, const ob_particle_desc* d);
int ob_step(ob_sim* s, int nsteps);
const char* ob_last_error(const ob_sim* s);
/* threads of the lattice loops (OpenMP builds; n <= 0 keeps the count);
   returns the count in use.  Results do not depend on it. */
int ob_set_threads(int n);
int ob_nx(const ob_sim* s);
int ob_ny(const ob_sim* s);
long ob_steps_done(const ob_sim* s);

/* post-collision populations f*[i][y][x] (9*ny*nx doubles) */
void ob_get_populations(const ob_sim* s, double* f);
void ob_set_populations(ob_sim* s, const double* f);
/* density and velocity of the streamed populations (start of next step) */
int ob_get_fields(ob_sim* s, double* rho, double* ux, double* uy);
int ob_get_particles(const ob_sim* s, ob_particle_state* out, int cap);
/* body-frame markers of particle p: positions (2*n), normals (2*n), S (n) */
int ob_get_markers(const ob_sim* s, int p, double* rb, double* nb, double* S, int cap);
/* mass, inertia, area of particle p */
void ob_particle_props(const ob_sim* s, int p, double* m, double* I, double* A);
/* the body force field f_lb of the last step, 2*ny*nx (component-major) */
void ob_get_force_field(const ob_sim* s, double* flb);

/* ---- individual steps, exposed for the pins ---- */
void ob_lattice(int e[9][2], double w[9]);
void ob_feq(double rho, double ux, double uy, double feq[9]);
/* BGK collision with the Guo term (Eqs. 4-7): f in, f_out out */
void ob_collide(const double f[9], double tau, double Fx, double Fy, double f_out[9]);
void ob_guo_term(double ux, double uy, double tau, double Fx, double Fy, double Fi[9]);
/* MLS transfer weights at point (x, y): nodes (ix, iy) unwrapped and
   rows phi (value), dphi/dx, dphi/dy over the 9 nodes */
int ob_mls(int weight, double x, double y, int ix[9], int iy[9], double phi[27]);
double ob_weight(int weight, double r);
/* hydrodynamic force and torque (Eqs. 13-14) on particle p from given
   density and velocity fields (ny*nx each), with the body at its latest
   stored level.  Returns OB_EDOMAIN if a probe support leaves the domain. */
int ob_stress_force(ob_sim* s, int p, const double* rho, const double* ux,
                    const double* uy, double F[2], double* M);
/* set the stored history of particle p: levels n-1 and n-2 */
void ob_set_history(ob_sim* s, int p, const double X1[2], double th1, const double U1[2],
                    double W1, const double X2[2], double th2, const double U2[2], double W2);
/* spread the marker forces of particle p at its latest stored level into
   f_lb from given velocity fields; returns total Lagrangian force sum S_l F_l */
int ob_spread_only(ob_sim* s, int p, const double* ux, const double* uy,
                   double* flb, double sumSF[2], double* sum_torque);
/* rigid-body update of a free particle with a given force / torque */
void ob_rigid_update(ob_sim* s, int p, const double F[2], double M);

#ifdef __cplusplus
}
#endif
#endif
