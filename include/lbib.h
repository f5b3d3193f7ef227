/*
 * lbib.h -- C ABI of the GB300 (sm_103a) library for the coupled
 * lattice-Boltzmann / immersed-boundary (LB-IB) method of Coclite,
 * de Tullio, Pascazio and Decuzzi, "A combined Lattice Boltzmann and
 * Immersed Boundary approach for predicting the vascular transport of
 * differently shaped particles" (arXiv:1606.01805).
 *
 * One context holds one D2Q9 lattice and its rigid particles on one GPU.
 * A step (lbm_step) is, in this order (Section 2, weak coupling):
 *   1. pull-streaming (Eq. 4) with Zou-He known-velocity walls (Section 2.1);
 *   2. density and velocity moments (Eqs. 6-7);
 *   3. per particle: probe-based surface stress, force and torque (Eqs.
 *      13-14, Section 2.3) and the two-level rigid-body update (Eqs. 15-16);
 *   4. MLS interpolation of lattice velocity to the Lagrangian markers
 *      (Eqs. 8-10), direct-forcing marker force (Eq. 11), spreading of the
 *      marker forces to the lattice (Eq. 12);
 *   5. BGK collision with the Guo forcing term (Eqs. 2, 4, 5).
 * With the FP32 compute type (LBM_FP32, LBM_FP16_SHIFTED) the force field
 * of step 4 is held in fixed point (units of 2^-40 in 64-bit integers):
 * each marker adds its contributions straight into it with integer atomics,
 * so the result does not depend on the order of the additions.  LBM_FP64
 * and the tangent mode gather the contributions per cell in marker order
 * (a spreading kernel) and keep the field in their compute type.
 *
 * Conventions shared by every call:
 *  - Lattice units: dx = dt = 1.  Nodes (x, y), 0 <= x < nx, 0 <= y < ny.
 *    Wall nodes are the first/last row (column) of nodes, so a channel
 *    between y walls has height H = ny - 1.
 *  - Host arrays of fields are y-major: element (x, y) at index y * nx + x.
 *    Populations are [9][ny][nx] in the velocity order e_0 = (0,0),
 *    e_1..e_4 = (1,0), (0,1), (-1,0), (0,-1), e_5..e_8 = (1,1), (-1,1),
 *    (-1,-1), (1,-1) (Eq. 3).
 *  - Every call returns an lbm_status; nothing throws across the ABI.  On
 *    an error, lbm_last_error() gives a one-line reason.
 *  - A context is used by one host thread at a time.
 *  - Device work is enqueued on cfg.cuda_stream (NULL: the legacy default
 *    stream).  lbm_step does not synchronise; every lbm_get_* call does.
 */
#ifndef LBIB_H
#define LBIB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx; /* opaque, owned by the library */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,     /* bad argument or configuration */
    LBM_ENOMEM = 2,     /* workspace too small or allocation failed */
    LBM_ECUDA = 3,      /* a CUDA runtime call failed */
    LBM_ETIMEOUT = 4,   /* a bounded device wait expired */
    LBM_ENONFINITE = 5, /* a lattice cell of non-positive or non-finite density
                           (watchdog of the fluid kernel), or a non-finite
                           particle state */
    LBM_EINTERNAL = 6,
    LBM_EDOMAIN = 7     /* a marker or probe support crossed a wall */
} lbm_status;

/* side kinds, for sides ordered x-, x+, y-, y+ */
typedef enum { LBM_BC_PERIODIC = 0, LBM_BC_VELOCITY = 1 } lbm_bc;

/* storage / arithmetic of the populations.  The particle state, the MLS
   3x3 solves, the force and torque sums and the rigid-body update are
   always FP64 (FP64 with derivatives in the tangent mode); marker and
   probe geometry, MLS weights and moments, fits and tractions run in the
   population arithmetic (FP32, or FP64 for LBM_FP64). */
typedef enum {
    LBM_FP64 = 0,         /* FP64 populations, FP64 collision */
    LBM_FP32 = 1,         /* FP32 populations stored as f - w_i, FP32 collision */
    LBM_FP16_SHIFTED = 2, /* FP16 storage of f - w_i, FP32 collision */
    LBM_FP32_TANGENT = 3  /* LBM_FP32 plus forward-mode derivatives along
                             LBM_TANGENTS directions (see lbm_add_particle_tangent) */
} lbm_precision;

#define LBM_TANGENTS 3

typedef enum { LBM_INIT_REST = 0, LBM_INIT_COUETTE = 1, LBM_INIT_TAYLOR_GREEN = 2 } lbm_init_kind;

/* particle shapes of Sections 3 and 4 */
typedef enum {
    LBM_SHAPE_CIRCLE = 0,   /* dim[0] = diameter */
    LBM_SHAPE_ELLIPSE = 1,  /* dim[0] = major axis, dim[1] = minor axis (full) */
    LBM_SHAPE_RECT = 2,     /* dim[0] = width (body x), dim[1] = height */
    LBM_SHAPE_SQUARE = 3,   /* dim[0] = side */
    LBM_SHAPE_TRIANGLE = 4  /* equilateral, dim[0] = side */
} lbm_shape;

/* MLS weight functions: Eq. 10 (default) and Eqs. 17-20 */
typedef enum {
    LBM_W_EXP = 0, LBM_W_CUBIC = 1, LBM_W_QUARTIC = 2, LBM_W_COSINE = 3, LBM_W_POLY = 4
} lbm_weight;

typedef struct {
    int32_t nx, ny;         /* lattice nodes, each >= 3 */
    double tau;             /* BGK relaxation time, > 0.5; nu = (tau - 1/2)/3 */
    int32_t bc[4];          /* lbm_bc per side x-, x+, y-, y+; opposite sides equal */
    double wall_u[4][2];    /* velocity of each wall side (ignored if periodic) */
    double body_force[2];   /* constant fluid body-force density g_f */
    double gravity[2];      /* gravity on the particles (buoyancy-corrected) */
    int32_t precision;      /* lbm_precision */
    int32_t init;           /* lbm_init_kind; Couette uses wall_u of y- and y+ */
    double init_u;          /* Taylor-Green amplitude */
    int32_t weight;         /* lbm_weight */
    double marker_spacing;  /* target marker spacing; <= 0 means 0.3 */
    int32_t max_particles;  /* capacity; <= 0 means 16 */
    int32_t max_markers;    /* total marker capacity; <= 0 means 16384 */
    void* cuda_stream;      /* cudaStream_t, or NULL */
    void* d_workspace;      /* caller-owned device memory, or NULL to allocate */
    size_t workspace_bytes; /* size of d_workspace */
    int32_t check_every;    /* watchdog period: the fluid kernel checks every
                               cell on the steps whose count since init is a
                               multiple of check_every; 0 or 1: every step;
                               else 2, 4, 8, 16 or 32 (LBM_EINVAL otherwise) */
} lbm_config;

typedef struct {
    int32_t shape;          /* lbm_shape */
    double dim[2];          /* see lbm_shape */
    double xc, yc, theta;   /* centroid and orientation of the body x axis */
    double rho_s;           /* solid density (fluid reference density is 1) */
    double u0[2], omega0;   /* initial velocity and angular velocity */
    int32_t n_markers;      /* 0: perimeter / marker_spacing */
} lbm_particle_desc;

typedef struct {
    double xc, yc, theta;   /* centroid (unwrapped in periodic x) and angle */
    double u[2], omega;     /* velocity and angular velocity */
    double F[2], M;         /* hydrodynamic force and torque of the last step */
    double omega_sum;       /* sum of omega over the rigid-body updates done
                               (mean angular velocity = omega_sum / steps) */
} lbm_particle_state;

/*
 * Device bytes the context needs for cfg (sizes, precision and capacities).
 * A caller that owns device memory (e.g. a PyTorch tensor) passes a block of
 * at least this size in cfg.d_workspace; the library then allocates nothing
 * on the device.  Returns LBM_EINVAL for an invalid configuration.
 */
lbm_status lbm_workspace_bytes(const lbm_config* cfg, size_t* bytes);

/*
 * Create a context and its initial field f* = f^eq(rho, u0) (Eq. 2): rest,
 * the planar Couette profile between the y walls (Section 4.1) or a
 * Taylor-Green vortex.  Errors: LBM_EINVAL (tau <= 0.5, nx or ny < 3,
 * opposite sides of different kinds, bad capacities), LBM_ENOMEM (workspace
 * too small, or cudaMalloc failed when d_workspace is NULL), LBM_ECUDA.
 * On success *out owns host state only; device memory is the caller's
 * workspace or library-allocated and freed by lbm_destroy.
 */
lbm_status lbm_init(const lbm_config* cfg, lbm_ctx** out);

/*
 * Add a rigid particle before the first step (Sections 3-4).  Markers are
 * placed at the midpoints of equal arc-length pieces of the perimeter
 * (polygons: per face), with S_l the piece length and the outward normal.
 * Errors: LBM_EINVAL (after the first step, bad shape or size, capacity
 * exceeded, or a marker/probe support crossing a wall).  *out_id receives
 * the particle index.  Copies the markers host -> device and synchronises.
 */
lbm_status lbm_add_particle(lbm_ctx* ctx, const lbm_particle_desc* desc, int32_t* out_id);

/*
 * Advance nsteps >= 0 time steps (the five stages above per step),
 * asynchronously on the context's stream.  Errors detected on the device
 * are reported by the next lbm_sync / lbm_get_* call: LBM_EDOMAIN (a
 * marker or probe support crossed a wall), LBM_ENONFINITE (the watchdog:
 * on its steps, see lbm_config.check_every, the fluid kernel flags any
 * cell whose streamed density rho = sum_i f_i of Eq. 6 is not positive or
 * not finite -- a NaN or infinite population makes the sum non-finite;
 * every rigid-body update flags a non-finite particle state).  The flags
 * are sticky: once set, every later lbm_sync / lbm_get_* call reports them.
 */
lbm_status lbm_step(lbm_ctx* ctx, int32_t nsteps);

/*
 * As lbm_step, with CUDA events around each step and around its fused
 * stream-collide launch.  Synchronises; adds the summed device time of
 * the steps (ms) to *ms_step and of the stream-collide launches to
 * *ms_fluid (either may be NULL).  With ms_fluid NULL no event sits before
 * the stream-collide launch, which may then start its population loads
 * while the immersed-boundary kernel before it finishes, as in lbm_step;
 * with ms_fluid it starts after that kernel, so that its time is its own.
 */
lbm_status lbm_step_timed(lbm_ctx* ctx, int32_t nsteps, double* ms_step, double* ms_fluid);

/* Wait for the stream; report a device-side error flagged since init
   (LBM_EDOMAIN, LBM_ENONFINITE or LBM_ETIMEOUT, in that order of priority). */
lbm_status lbm_sync(lbm_ctx* ctx);

/*
 * Test hook of the host's error path (the paper has no counterpart): sets,
 * on the device and in stream order, the flag a kernel sets when it
 * detects `status` (LBM_EDOMAIN, LBM_ENONFINITE or LBM_ETIMEOUT; else
 * LBM_EINVAL), so that the next lbm_sync / lbm_get_* call reports it.
 * Nothing faults; the context stays usable but keeps reporting the flag.
 */
lbm_status lbm_inject_status(lbm_ctx* ctx, int32_t status);

/*
 * Test hook of the bounded device waits (the paper has no counterpart).
 * With a staged tile variant (6..9, see lbm_get_tile), the next step's
 * fluid launch arms the mbarrier of its first CTA's first tile for 16
 * bytes more than its copies bring, so that the CTA's wait for it runs out
 * after wait_cycles clock cycles; the CTA then sets the LBM_ETIMEOUT flag,
 * lets its copies in flight land and returns without computing its tiles.
 * In the fused step mode (lbm_set_step_mode), the next step's first fluid
 * item waits for one spreading tile more than its instance has; its wait
 * runs out after wait_cycles, sets the flag and aborts the step's other
 * waits.  Else LBM_EINVAL, as for wait_cycles outside 1e6 .. 2e9 (the
 * kernels' own limit is 2e9, about a second).  The step is launched
 * directly (not from a captured graph).  Nothing faults; lbm_sync reports
 * LBM_ETIMEOUT, and the step's results are not usable.
 */
lbm_status lbm_inject_stall(lbm_ctx* ctx, int64_t wait_cycles);

/*
 * Density and velocity (host, nx*ny doubles each, y-major) of the
 * populations after streaming of the stored state, i.e. the moments of
 * Eqs. 6-7 at the start of the next step (constant body force with its
 * half step, no immersed-boundary force).  Any pointer may be NULL.
 */
lbm_status lbm_get_fields(lbm_ctx* ctx, double* rho, double* ux, double* uy);

/*
 * Stored post-collision populations f*_i of Eq. 4 (the right-hand side of
 * the lattice BGK equation before streaming), unshifted (f_i, not f_i -
 * w_i): host array of [9][ny][nx] doubles, caller-owned, in the velocity
 * order of Eq. 3.  Synchronises.  Errors: LBM_EINVAL (null argument),
 * LBM_ECUDA.
 */
lbm_status lbm_get_populations(lbm_ctx* ctx, double* f);
/*
 * Replace the stored post-collision populations f*_i of Eq. 4 (host,
 * [9][ny][nx] doubles, caller-owned, read only; rounded to the storage
 * precision).  The next step streams them.  Synchronises.  Errors as for
 * lbm_get_populations.
 */
lbm_status lbm_set_populations(lbm_ctx* ctx, const double* f);

/*
 * Particle states (host, caller-owned array of cap entries): the centroid,
 * angle, velocity and angular velocity of the latest rigid-body update
 * (Eqs. 15-16) and the hydrodynamic force and torque it used (Eqs. 13-14,
 * the surface integrals of Section 2.3).  *n receives the particle count;
 * min(cap, count) entries are written, in the order the particles were
 * added.  Synchronises.  Errors: a device flag as for lbm_sync (LBM_EDOMAIN
 * still returns the states).
 */
lbm_status lbm_get_particles(lbm_ctx* ctx, lbm_particle_state* out, int32_t cap, int32_t* n);

/*
 * lbm_step_static -- the paper has no counterpart: this is a deployment
 * variant of lbm_step for callers that cannot allocate device memory while
 * they run, e.g. a host program whose device memory all comes from a
 * fixed pool set up at start-up, or one that must never let an allocation
 * stall or synchronise the device mid-run.  It advances nsteps steps
 * exactly as lbm_step does (same kernels, same order, same results) but
 * keeps the immersed-boundary scratch -- per marker block force/torque
 * sums, per-particle completion counters and support boxes, per-marker
 * spreading records -- in one static device array of
 * LBM_STATIC_SCRATCH_BYTES compiled into the library, instead of in the
 * context's workspace.  It allocates nothing: no cudaMalloc, no cudaFree,
 * no allocating library routine; the populations and particle state it
 * reads and writes are the context's, as for lbm_step.
 *  - Limits: at most LBM_STATIC_MAX_PARTICLES particles and
 *    LBM_STATIC_MAX_MARKERS markers in the context, in every precision
 *    (the array is sized for the largest per-marker record, that of
 *    LBM_FP32_TANGENT), else LBM_EINVAL with the reason in lbm_last_error.
 *  - The static array is held by every GPU that loads the library until
 *    the process exits.  The first call on a device looks up its device
 *    address (once per device, with that device current) and keeps it;
 *    make that first call before any stream capture, and do not reset the
 *    device (cudaDeviceReset) after it while the library stays loaded.
 *  - All calls share the one array, which keeps the last call's contents;
 *    each call clears the counters that must start at zero (every other
 *    entry is reset or written before it is read within a step).  Calls
 *    that overlap on the GPU (other streams, other contexts, other threads)
 *    race on the array: serialise them.
 *  - Launches directly on the context's stream, asynchronously; errors as
 *    for lbm_step.
 */
#define LBM_STATIC_SCRATCH_BYTES (6u << 20)
#define LBM_STATIC_MAX_PARTICLES 1024
#define LBM_STATIC_MAX_MARKERS 16384
lbm_status lbm_step_static(lbm_ctx* ctx, int32_t nsteps);

/* ---------------------------------------------------------------------
 * Batches: many independent lattices (instances) of uneven sizes advanced
 * together, for screening many particle shapes and placements (the "4S"
 * screening motivation of the Introduction).  One context holds them all:
 * every step is still the five stages above, for every instance, with one
 * launch per kernel for the whole batch (the fluid kernel walks a list of
 * 128 x 8-cell tiles of all instances).  Instances never interact.
 * The single-lattice calls above are the one-instance case and act on
 * instance 0 (lbm_step, lbm_step_timed, lbm_sync and lbm_get_particles act
 * on the whole batch; particle ids run over the whole batch in the order
 * the particles were added).
 * ------------------------------------------------------------------- */

/* Device bytes for a batch of n configurations (see lbm_init_batch). */
lbm_status lbm_batch_workspace_bytes(const lbm_config* cfgs, int32_t n, size_t* bytes);

/*
 * Create a context holding n >= 1 instances.  cfgs[i] gives instance i its
 * lattice (nx, ny, tau, bc, wall_u, body_force, gravity, init, init_u,
 * marker_spacing); cfgs[0] alone gives the stream, the workspace, the
 * capacities (max_particles, max_markers: totals over the batch), the
 * precision (all instances must give the same one) and the MLS weight.
 * Errors as for lbm_init.
 */
lbm_status lbm_init_batch(const lbm_config* cfgs, int32_t n, lbm_ctx** out);

/* Instances in the context (1 for lbm_init). */
int32_t lbm_instances(const lbm_ctx* ctx);

/* lbm_add_particle into instance `instance` (0 <= instance < lbm_instances). */
lbm_status lbm_add_particle_to(lbm_ctx* ctx, int32_t instance, const lbm_particle_desc* desc,
                               int32_t* out_id);

/* lbm_get_fields / lbm_get_populations / lbm_set_populations of one instance
   (arrays sized by that instance's nx, ny). */
lbm_status lbm_get_instance_fields(lbm_ctx* ctx, int32_t instance, double* rho, double* ux, double* uy);
lbm_status lbm_get_instance_populations(lbm_ctx* ctx, int32_t instance, double* f);
lbm_status lbm_set_instance_populations(lbm_ctx* ctx, int32_t instance, const double* f);

/*
 * Tile variant of the fused fluid kernel.  The first step of a context
 * (lbm_step or lbm_step_timed) runs its immersed-boundary kernels once, times
 * every variant the precision has on the context's own lattices with those
 * forces and keeps the fastest (all variants give bit-identical results);
 * lbm_get_tile reports the choice (index, cells per thread, rows per tile)
 * and lbm_set_tile forces variant `variant` and skips the timing
 * (LBM_EINVAL for an index out of 0 .. LBM_TILE_VARIANTS - 1 or one the
 * precision does not have).
 * lbm_tile_info describes any variant: cells per thread (the tile is 32
 * times as wide), rows per tile, and the stages of a staged variant (0 for
 * a direct one), and whether `precision` has it (returns LBM_OK) or not
 * (LBM_EINVAL).  The variants:
 *   0..5  direct kernels, one CTA per tile, streamed populations loaded
 *         from global memory: 4 x 8, 4 x 4, 1 x 8, 2 x 8, 2 x 4, 1 x 4;
 *   6..9  the persistent kernel that stages each tile's rows in shared
 *         memory with bulk asynchronous copies, 8 rows per tile: 4 cells
 *         per thread with 2 or 3 stages, 2 cells with 3 or 4 stages
 *         (LBM_FP32 and LBM_FP16_SHIFTED only).
 * LBM_FP64 has variants 0..5, the tangent mode variant 2 only.
 */
#define LBM_TILE_VARIANTS 10
lbm_status lbm_get_tile(const lbm_ctx* ctx, int32_t* variant, int32_t* cells_per_thread,
                        int32_t* rows_per_block);
lbm_status lbm_tile_info(int32_t variant, int32_t precision, int32_t* cells_per_thread, int32_t* rows,
                         int32_t* stages);
lbm_status lbm_set_tile(lbm_ctx* ctx, int32_t variant);

/*
 * Step mode of a batch.  LBM_STEP_SEPARATE (the mode of a single lattice):
 * each step is the immersed-boundary kernels (probes and rigid update,
 * markers, and the spreading kernel in LBM_FP64 and the tangent mode) and
 * then the fluid kernel, each one launch over all instances.
 * LBM_STEP_OVERLAP (the default of a batch of two or more instances): the
 * instances are split into two halves of about equal
 * cell count, and lbm_step's captured runs of steps advance each half with
 * its own chain of the same kernels on a stream of its own: the particle
 * work of one half can run beside the fluid kernel of the other, step
 * after step.  Steps launched one by one (lbm_step_timed,
 * the remainder of a run that is not a multiple of 32 steps) run both
 * halves as in LBM_STEP_SEPARATE.  The split needs the particles numbered
 * in instance order across it; otherwise the mode runs as
 * LBM_STEP_SEPARATE.  It needs a batch of two or more instances (else
 * LBM_EINVAL).
 * LBM_STEP_FUSED: each step is one persistent launch whose CTAs take the
 * step's work items in a fixed order -- probe blocks, marker blocks,
 * spreading tiles and fluid tiles of every instance, the stages of one
 * instance a few instances apart, so that the particle work of some
 * instances runs beside the fluid work of others.  Within an instance an
 * item waits (bounded; LBM_ETIMEOUT on expiry) for the items it needs.
 * The fused mode needs a batch of two or more instances (lbm_init_batch) in
 * LBM_FP64, LBM_FP32 or LBM_FP16_SHIFTED (else LBM_EINVAL); it uses its own
 * fluid tile (4 cells per thread, 8 rows: lbm_get_tile reports variant 0)
 * and lbm_step_timed then reports the fused launch as the fluid time.
 * All modes give the same results, bit for bit.  Set the mode before or
 * between steps.
 */
#define LBM_STEP_SEPARATE 0
#define LBM_STEP_FUSED 1
#define LBM_STEP_OVERLAP 2
lbm_status lbm_set_step_mode(lbm_ctx* ctx, int32_t mode);
lbm_status lbm_get_step_mode(const lbm_ctx* ctx, int32_t* mode);

/*
 * Tangent mode (precision LBM_FP32_TANGENT) -- forward-mode
 * differentiation of the whole step (the paper has no counterpart; it
 * serves sensitivity studies of the transport results of Sections 4.1-4.3,
 * e.g. of the equilibrium position or the rotation rate to the aspect ratio,
 * the initial position or the wall speed).  Every population, force-field
 * value and particle quantity carries, besides its value, its derivatives
 * along LBM_TANGENTS input directions p_1..p_K; each step propagates them
 * through Eqs. 2-16 by the chain rule, so after n steps they are the exact
 * derivatives of the discrete n-step map (the choice of the 3x3 MLS support
 * is piecewise constant and contributes none).  Values are those of
 * LBM_FP32 (populations FP32 stored as f - w_i, particle work FP64);
 * derivatives of the populations are FP32, of the particle state FP64.
 * A population element is 16 bytes (value, K derivatives).
 *
 * Seeds, all before the first step:
 *  - lbm_set_wall_tangents: dwall[(side * 2 + c) * LBM_TANGENTS + k] =
 *    d(wall_u[side][c]) / dp_k (sides x-, x+, y-, y+).  Re-creates the
 *    initial field of the instance (the Couette profile then carries the
 *    derivatives of the wall speeds).
 *  - lbm_add_particle_tangent: as lbm_add_particle_to, with
 *    seed[k * 6 + j] = d(q_j) / dp_k for q = (dim[0], dim[1], xc, yc,
 *    theta, rho_s).  The marker count is fixed by the values of the
 *    dimensions (it does not change under a perturbation); markers, normals,
 *    arc lengths, area and inertia carry the derivatives.
 * Outputs:
 *  - lbm_get_particle_tangents: out[(i * LBM_TANGENTS + k) *
 *    LBM_TANGENT_FIELDS + j] = d(s_j) / dp_k of particle i, for
 *    s = (xc, yc, theta, u[0], u[1], omega, F[0], F[1], M, omega_sum) of
 *    lbm_particle_state; out holds cap * LBM_TANGENTS * LBM_TANGENT_FIELDS
 *    doubles, *n receives the particle count.
 *  - lbm_get_field_tangents: d(rho, ux, uy)/dp_k of lbm_get_fields, each
 *    output [LBM_TANGENTS][ny][nx] doubles (any may be NULL, not all).
 * Errors: LBM_EINVAL when the context is not in the tangent mode, after the
 * first step (seeds), or for a bad instance or missing seeds.
 */
#define LBM_TANGENT_FIELDS 10
lbm_status lbm_set_wall_tangents(lbm_ctx* ctx, int32_t instance, const double* dwall);
lbm_status lbm_add_particle_tangent(lbm_ctx* ctx, int32_t instance, const lbm_particle_desc* desc,
                                    const double* seed, int32_t* out_id);
lbm_status lbm_get_particle_tangents(lbm_ctx* ctx, double* out, int32_t cap, int32_t* n);
lbm_status lbm_get_field_tangents(lbm_ctx* ctx, int32_t instance, double* drho, double* dux,
                                  double* duy);

/*
 * Reverse-mode differentiation (adjoint) of nsteps steps of the LB-IB map
 * (Eqs. 2-16, the same discrete map as lbm_step), for two outputs at once
 * (the paper has no counterpart; it serves the same sensitivity studies as
 * the tangent mode, with a cost that does not grow with the number of
 * inputs):
 *   J_0 = sum_p seed[2p] * yc_p(N),   J_1 = sum_p seed[2p + 1] * omega_sum_p(N)
 * over the particles p after N = nsteps steps (seed[2p + 1] = 1/N makes J_1
 * the mean angular velocity).  The call runs the N steps forward (the
 * context then holds the state after them, as after lbm_step), keeping the
 * populations and bodies every checkpoint_every steps; it then walks the
 * steps backwards, recomputing each segment between two checkpoints and
 * carrying the adjoint of the populations and of the bodies back one step
 * at a time (collision, streaming with the Zou-He walls, spreading, direct
 * forcing, MLS interpolation, probe stress, force and torque sums, the
 * two-level rigid update, all reversed).  Outputs (host, caller-owned):
 *   dparticle[(p * 2 + o) * 6 + j] = d J_o / d q_j of particle p, for
 *     q = (dim[0], dim[1], xc, yc, theta, rho_s) of its lbm_particle_desc
 *     (the marker count held fixed);
 *   dwall[(i * 2 + o) * 8 + (side * 2 + c)] = d J_o / d wall_u[side][c] of
 *     instance i (through the Zou-He walls and, for the Couette initial
 *     field, through the initial profile).
 * In a batch whose instances hold one particle each, J_o of instance i is
 * the output of its particle, so its rows are that particle's gradients.
 * Requirements (else LBM_EINVAL): LBM_FP32, no step done yet, at least one
 * particle, periodic x sides, fewer than 2^31 / 9 nodes per lattice, not
 * the fused step mode; a marker or probe
 * support must stay off the wall rows (else LBM_EDOMAIN).  The call
 * allocates its own device memory (checkpoints, one segment of steps, the
 * adjoint buffers; LBM_ENOMEM if it does not fit) and frees it before it
 * returns.  Synchronises.
 */
lbm_status lbm_adjoint(lbm_ctx* ctx, int32_t nsteps, int32_t checkpoint_every, const double* seed,
                       double* dparticle, double* dwall);

/* Steps done since lbm_init. */
int64_t lbm_steps_done(const lbm_ctx* ctx);

/* One-line reason for the last error on ctx (never NULL). */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Free the context (and the device memory it allocated itself). */
void lbm_destroy(lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
