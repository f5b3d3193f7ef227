// lbib_internal.h -- structures shared by the host API and the kernels of
// the LB-IB library (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lbib.h"
#include "dual.h"

namespace lbib {

// tangent mode: K directions; FP32 populations and FP64 particle work
constexpr int KT = LBM_TANGENTS;
using TF = Dual<float, KT>;
using TD = Dual<double, KT>;

// two-component vector of a real type (double2-compatible for double)
template <class R>
struct Vec2 {
    R x, y;
};

// Lattice geometry and the constants of the fluid step of one instance.
// Populations are stored shifted, f~_i = f_i - w_i, in 9 planes of ny rows
// of `pitch` elements (pitch a multiple of 32).
struct Geo {
    int nx, ny, pitch, nseg;  // nseg = pitch / 32 force-flag segments per row
    long long plane;          // elements per population plane
    int px, py;               // periodic in x / y
    double uw[4][2];          // wall velocities, sides x-, x+, y-, y+
    double g[2];              // constant fluid body force
    double grav[2];           // gravity on the particles of this lattice
    double tau, omega;        // relaxation time and its inverse
    // the same constants in FP32, precomputed on the host: the FP32 kernels
    // must not touch FP64 (a small fraction of the FP32 rate on this part)
    float uwf[4][2], gf[2], omegaf;
    // tangent mode: derivatives of the wall velocities along the K directions
    double uwd[4][2][KT];
    float uwdf[4][2][KT];
};

// One lattice of a context (a context holds one or a batch of them).  Its
// populations start at element f_off of each population buffer, its force
// field at element flb_off of the force buffer, its flags at byte flags_off.
// 16-byte aligned, so that a kernel can copy it in 16-byte pieces.
struct alignas(16) Inst {
    Geo G;
    long long f_off, flb_off, flags_off;
};

// Rigid particle on the device, real type R (FP64, or FP64 with tangents).
// Index 0 of the history arrays is the latest level, index 1 the level
// before it.
template <class R>
struct DParticleT {
    R X[2][2], th[2], U[2][2], W[2];
    R cs[2][2];               // (cos, sin) of th[0] and th[1]
    R F[2], M;
    R wsum;                   // sum of the angular velocity over the updates done
    R mass, inertia, area, rho_s, inv_mass, inv_inertia;
    int m0, nm;               // first marker, marker count
    int b0, nblk;             // first marker block, marker blocks (MB markers each)
    int inst, pad_;           // lattice the particle lives in
    long long nupd;           // rigid-body updates done
};
using DParticle = DParticleT<double>;

// Pose and velocities of a particle in the compute type C, written beside
// DParticleT by the FP64 rigid-body update (and when the particle is added)
// and double-buffered with it.  The marker kernels form marker and probe
// positions in C relative to the node (ix, iy) at or below the centre, so
// none of their geometry needs FP64.  v[]: centre minus (ix, iy); cos, sin
// of the angle; u, v, omega; the changes of u, v, omega, cos, sin from the
// previous level, and that level's omega (the marker acceleration of the
// probe pressure).
enum { PC_XF, PC_YF, PC_C, PC_S, PC_U, PC_V, PC_W, PC_DU, PC_DV, PC_DW, PC_W1, PC_DC, PC_DS, PC_N };
template <class C>
struct __align__(16) PoseC {
    int ix, iy, pad_[2];
    C v[PC_N];
};

// Body-frame position and outward normal of one marker, in C.
template <class C>
struct __align__(16) MGeo {
    C rx, ry, nx, ny;
};

constexpr int MB = 8;         // markers per block of the marker kernels (one warp, 4 lanes each)
constexpr int INLINE_BLOCKS = 128, INLINE_PARTICLES = 64;

// Spreading record of one marker: the unwrapped lower-left node (i0, j0) of
// its 3x3 support and the 9 contributions S_l phi_k F_l (Eq. 12).
template <class C>
struct __align__(16) Rec {
    int i0, j0;
    C cx[9], cy[9];
};

// Device error bits (OR-ed into the error word).
enum : unsigned { ERR_DOMAIN = 1u, ERR_NONFINITE = 2u, ERR_TIMEOUT = 4u };

// The particle state is double-buffered with the populations: a step that
// reads populations buffer c reads particles pin = state[c] and writes the
// updated bodies to pout = state[c ^ 1].
// Arrays of the real type R and of the compute type C are passed untyped
// (the kernel's R and C decide).
struct ParticleArgs {
    const void* f;            // post-collision populations buffer (storage type)
    const Inst* insts;
    const void* pin;          // DParticleT<R>: bodies at the start of the step
    void* pout;               // DParticleT<R>: bodies after the rigid-body update
    const void* pcin;         // PoseC<C> of pin
    void* pcout;              // PoseC<C> of pout
    const int4* blk;          // per marker block: (particle, first marker, markers, instance)
    void* partial;            // R per marker block: F_x, F_y, M partial sums
    unsigned* count;          // per particle: probe blocks done (the last one resets it)
    const void* mg;           // MGeo<C>: body-frame marker positions and normals
    const void* S;            // C: marker arc lengths
    void* recs;               // Rec<C>[max_markers]
    int4* boxes;              // per particle: support box (x0, y0, x1, y1)
    void* flb;                // force field and its flags: the marker kernel spreads into them
    uint8_t* flags;           // directly when the field is fixed point (ForceField)
    unsigned* err;
    int weight;
    int blk_base;             // marker block of the kernels' first CTA (a range of the table)
    int single;               // the context holds one lattice: `one` is its descriptor
    Inst one;
    // a context of at most INLINE_BLOCKS marker blocks also passes the block
    // table in the parameters (no dependent load in front of the block's work)
    int nblk_inline;          // 0 or the block count
    int4 blk_inline[INLINE_BLOCKS];
};

struct SpreadArgs {
    const Inst* insts;
    const void* recs;
    const int4* boxes;
    void* flb;                // force buffer (2 planes of compute type per instance)
    uint8_t* flags;           // flags buffer ([ny][nseg] bytes per instance)
    unsigned* err;
    int single;               // as in ParticleArgs
    Inst one;
    const int4* ptab;         // per particle: (first marker, markers, instance, tiles of its box)
    int p_base;               // particle of the kernel's first CTA row (a range of the particles)
    int np_inline;            // 0 or the particle count (at most INLINE_PARTICLES)
    int4 part_inline[INLINE_PARTICLES];  // the first np_inline entries of ptab
};

// One tile of a task list: instance, tile x, tile y (a tile being 32 * cpt
// cells of by rows), and the instance's population offset and row geometry,
// so that a kernel can address the tile's populations after one load.
struct alignas(16) Task {
    int inst, tx, ty, pitch;
    long long f_off;
    int ny, pad_;
};

// Fluid step over a list of tiles (Task).  One launch covers every tile of
// every instance; a CTA takes tasks blockIdx.x, blockIdx.x + gridDim.x, ...
struct FluidArgs {
    const void* fin;
    void* fout;
    void* flb;
    uint8_t* flags;
    const Inst* insts;
    const Task* tasks;
    int ntasks;
    int check;                // watchdog: flag a non-positive density or a non-finite value
    int stall;                // test hook: the staged kernel's first CTA waits for 16 bytes too many
    int keep;                 // autotuner: leave the force field and its flags in place
    unsigned* err;
    // staged variants: the tensor maps of the population buffer read, per
    // instance (device array of CUtensorMap), and of a single lattice (host)
    const void* tmaps;
    const void* tmap_one;
};

constexpr int TASKS_PER_CTA = 4;  // consecutive tiles a CTA of the task-list kernel takes

// fluid tile variants: (cells per thread, rows per block, stages); the
// autotuner picks one.  stages = 0: a direct kernel (one CTA per tile, the
// streamed populations loaded from global memory); stages > 0: the
// persistent kernel that stages that many tiles ahead in shared memory
// (FP32 and FP16 storage only; 8 rows per tile).
constexpr int N_FLUID_VARIANTS = LBM_TILE_VARIANTS;
struct FluidVariant {
    int cpt, by, stages;
};
constexpr FluidVariant FLUID_VARIANTS[N_FLUID_VARIANTS] = {
    {4, 8, 0}, {4, 4, 0}, {1, 8, 0}, {2, 8, 0}, {2, 4, 0},
    {1, 4, 0}, {4, 8, 2}, {4, 8, 3}, {2, 8, 3}, {2, 8, 4}};
// the variants a precision has: the tangent mode the one-cell direct tile
// only, FP64 the direct kernels, FP32 and FP16 storage all
constexpr bool variant_valid(int prec, int v) {
    return v >= 0 && v < N_FLUID_VARIANTS &&
           (prec == LBM_FP32_TANGENT ? v == 2 : (prec == LBM_FP64 ? FLUID_VARIANTS[v].stages == 0 : true));
}

// The fused step of a batch (one persistent launch per step): its work
// list and counters.  Item kinds, as int4 (kind, a, b, c):
//   FI_PROBES  (kind, first marker block, blocks <= 8, particle)
//   FI_MARKERS (kind, first marker block, blocks <= 8, particle)
//   FI_SPREAD  (kind, tile, particle, the particle's tile bound)
//   FI_FLUID   (kind, task of the 2 x 8 task list, instance, spreading
//               tiles of the instance)
enum { FI_PROBES = 0, FI_MARKERS = 1, FI_SPREAD = 2, FI_FLUID = 3 };
struct FusedArgs {
    FluidArgs fa;             // fluid tiles (the 2 x 8 task list)
    ParticleArgs pa;          // probes, rigid update, markers
    SpreadArgs sa;            // spreading tiles
    const int4* items;
    int nitems;
    int np, ninst;
    int parity;               // counter set of this step (the other one is cleared for the next)
    unsigned* counters[2];    // two sets of 2 np + ninst + 2 words
    long long wait_limit;     // clock cycles of a bounded wait
    int stall, stall_ticket;  // test hook: that fluid item waits for one spreading tile too many
};

// The reverse (adjoint) step of FP32 contexts, two outputs at once
// (adjoint.cu).  Adjoint buffers of populations have the layout of a
// population buffer (FP32), one per output, pop_elems apart; lam_F holds
// the force adjoint of flagged cells, [output][component] blocks of
// flb_elems, indexed like the force field.
// per marker, the probe Jacobians of one reverse level (adjoint.cu):
// d(F_x, F_y, M)/d(the 15 pose and geometry inputs) and d/d(the 5 MLS fits),
// the fits' weights (phi, dphi/dx, dphi/dy) at the 9 support nodes, the
// nodes' density deviation and velocity, and the nodes themselves
struct ProbePre {
    float jF[3][15], jG[3][5], w[3][9], nf[3][9];
    int node[2][9];
    int ok;
};

struct AdjArgs {
    const float* f;            // f*(n) (stored shifted populations of level n)
    long long* flb;            // the step's force field (recomputed; fixed point), cleared at the end
    uint8_t* flags;            // its flags, cleared at the end
    const Inst* insts;
    const DParticle* Pn;       // P(n)
    const DParticle* Pn1;      // P(n+1) (recomputed)
    const double* mgeo;        // per marker: body-frame position (2), normal (2), arc length (FP64)
    const int* marker_particle;
    const int4* ptab;          // per particle: (first marker, markers, instance, -)
    int np, nmark, weight;
    long long pop_elems, flb_elems;
    const float* lam_gp;       // lambda of the streamed populations of level n + 1, per output
    float* lam_g;              // the same of level n
    float* lam_F;
    double* lamP_new;          // per particle and output: lambda(P(n+1)) (see adjoint.cu)
    double* lamP_old;          // lambda(P(n)), accumulated
    double* lamFM;             // per particle and output: lambda of F_x, F_y, M
    double* lam_shape;         // per particle and output: lambda of 1/m, 1/I, area, rho_s
    double* lam_mgeo;          // per marker and output: lambda of rb (2), nb (2), S
    double* lam_wall;          // per instance and output: lambda of wall_u[4][2]
    float* zh;                 // per instance and y wall: the Zou-He transpose (9 x 9)
    ProbePre* ppre;            // per marker: the probe Jacobians of the level
    const int4* cblk;          // blocks of the cell kernels: (instance, bx, by, flags)
    int ncblk;
    unsigned* err;
};

struct FieldArgs {
    const void* f;            // population buffer
    Inst I;
    int y0, rows;
    double *rho, *ux, *uy;    // [rows][nx]
    double* tan;              // tangent mode, optional: [3][KT][rows][nx] (rho, ux, uy)
};

// kernel launchers (fluid*.cu / particles.cu); prec is an lbm_precision
cudaError_t launch_init(int prec, void* fbuf, const Inst& I, int kind, double init_u, cudaStream_t s);
// one != nullptr: the context holds that single lattice (tile grid,
// descriptor by value); otherwise the task list over all instances.
// grid: CTAs of a direct task-list kernel; sms: the device's SMs (the staged
// kernel's grid); pdl: launched with programmatic stream serialization (see
// pdl_wait), only when the kernel before it in the stream is the spreading
// kernel; wait_limit: clock cycles a staged CTA waits for a tile's copies
// before it gives up with ERR_TIMEOUT.  cudaErrorInvalidValue for a
// variant the precision does not have.
cudaError_t launch_fluid(int prec, int variant, const FluidArgs& a, const Inst* one, int grid, int sms,
                         cudaStream_t s, bool pdl, long long wait_limit);
cudaError_t launch_fluid_direct_a(int prec, int cpt, int by, const FluidArgs& a, const Inst* one, int grid,
                                  cudaStream_t s, bool pdl);
cudaError_t launch_fluid_direct_b(int prec, int cpt, int by, const FluidArgs& a, const Inst* one, int grid,
                                  cudaStream_t s, bool pdl);
cudaError_t launch_fluid_staged(int prec, int cpt, int stages, const FluidArgs& a, const Inst* one, int sms,
                                cudaStream_t s, bool pdl, long long wait_limit);
// the tensor map (CUtensorMap, 128 bytes at out) of lattice I in population
// buffer fbuf for the staged variants of `cpt` cells per thread: a 3-D
// tensor [9][ny][pitch] with boxes of one plane, 8 rows and the tile width
// plus 16 bytes on each side
constexpr size_t TMAP_BYTES = 128;
cudaError_t encode_stage_map(int prec, int cpt, const void* fbuf, const Inst& I, void* out);
cudaError_t launch_fields(int prec, const FieldArgs& a, cudaStream_t s);
// host-layout populations ([9][rows][nx] unshifted doubles at device
// address h) into / out of the stored shifted populations of rows
// [y0, y0 + rows) of lattice I in population buffer fbuf
cudaError_t launch_put_pops(int prec, const double* h, const Inst& I, int y0, int rows, void* fbuf,
                            cudaStream_t s);
cudaError_t launch_get_pops(int prec, const void* fbuf, const Inst& I, int y0, int rows, double* h,
                            cudaStream_t s);
// the fused step (step_fused.cu): one launch for the whole step of a batch;
// its spreading tiles have fused_spread_rows() rows and its fluid tiles
// are the task list of variant fused_fluid_variant()
cudaError_t launch_step_fused(int prec, const FusedArgs& f, int sms, cudaStream_t s);
int fused_spread_rows();
int fused_fluid_variant();
// the reverse step (adjoint.cu): setup (the Zou-He transposes), the kernels
// of one step in order, and the initial Couette profile's share of the
// wall-speed adjoint.  The cell kernels' block list has blocks of 32 x
// adjoint_block_rows() cells; flags bit 0: the instance starts from the
// Couette profile
int adjoint_block_rows();
cudaError_t launch_adjoint_setup(const AdjArgs& a, int ninst, cudaStream_t s);
cudaError_t launch_adjoint_step(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adjoint_init(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adjoint_probes_pre(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adjoint_probes_fin(const AdjArgs& a, cudaStream_t s);
// OR `bits` into the device error word, as a kernel that detects an error does
cudaError_t launch_raise(unsigned* err, unsigned bits, cudaStream_t s);
cudaError_t launch_probes(int prec, const ParticleArgs& a, int nblocks, cudaStream_t s);
cudaError_t launch_markers(int prec, const ParticleArgs& a, int nblocks, cudaStream_t s);
cudaError_t launch_spread(int prec, const SpreadArgs& a, int np, int tiles, cudaStream_t s);
size_t storage_bytes(int prec);
size_t compute_bytes(int prec);
size_t force_bytes(int prec);
// the precisions whose marker kernel adds the spreading (Eq. 12) straight
// into the fixed-point force field, with no spreading kernel in the
// separate step (the fused step still gathers by tiles, to the same bits)
bool markers_spread(int prec);
size_t rec_bytes(int prec);
size_t real_bytes(int prec);      // the particle real type R
size_t particle_bytes(int prec);  // sizeof(DParticleT<R>)
size_t pose_bytes(int prec);      // sizeof(PoseC<C>)

// shapes.cpp: body-frame markers and rigid-body properties of a shape, in
// double or, with derivatives of the dimensions, in TD
template <class T>
struct ShapeOutT {
    T area, inertia_per_mass;
    double rcirc;
    int n;
};
using ShapeOut = ShapeOutT<double>;
template <class T>
int make_shape_t(const lbm_particle_desc& d, const T dim[2], double spacing, T* rb, T* nb, T* S,
                 int cap, ShapeOutT<T>* out);
int make_shape(const lbm_particle_desc& d, double spacing, double* rb, double* nb, double* S,
               int cap, ShapeOut* out);

}  // namespace lbib
