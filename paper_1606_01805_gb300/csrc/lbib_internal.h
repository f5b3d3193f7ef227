// lbib_internal.h -- structures shared by the host API and the kernels of
// the LB-IB library (not part of the public ABI).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/lbib.h"

namespace lbib {

// Lattice geometry and the constants of the fluid step, passed by value to
// every lattice kernel.  Populations are stored shifted, f~_i = f_i - w_i,
// in 9 planes of ny rows of `pitch` elements (pitch a multiple of 32).
struct Geo {
    int nx, ny, pitch, nseg;  // nseg = pitch / 32 force-flag segments per row
    long long plane;          // elements per population plane
    int px, py;               // periodic in x / y
    double uw[4][2];          // wall velocities, sides x-, x+, y-, y+
    double g[2];              // constant fluid body force
    double tau, omega;        // relaxation time and its inverse
    // the same constants in FP32, precomputed on the host: the FP32 kernels
    // must not touch FP64 (a small fraction of the FP32 rate on this part)
    float uwf[4][2], gf[2], omegaf;
};

// Rigid particle on the device (all FP64).  Index 0 of the history arrays
// is the latest level, index 1 the level before it.
struct DParticle {
    double X[2][2], th[2], U[2][2], W[2];
    double cs[2][2];          // (cos, sin) of th[0] and th[1]
    double F[2], M;
    double mass, inertia, area, rho_s, inv_mass, inv_inertia;
    int m0, nm;               // first marker, marker count
    int b0, nblk;             // first marker block, marker blocks (MB markers each)
    long long nupd;           // rigid-body updates done
};

constexpr int MB = 8;         // markers per block of the marker kernels (one warp, 4 lanes each)

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
struct ParticleArgs {
    const void* f;            // post-collision populations (storage type)
    Geo G;
    const DParticle* pin;     // bodies at the start of the step
    DParticle* pout;          // bodies after the rigid-body update
    const int4* blk;          // per marker block: (particle, first marker, markers, 0)
    double* partial;          // per marker block: F_x, F_y, M partial sums
    const double2* rb;        // body-frame marker positions
    const double2* nb;        // body-frame normals
    const double* S;          // marker arc lengths
    void* recs;               // Rec<C>[max_markers]
    int4* boxes;              // per particle: support box (x0, y0, x1, y1)
    unsigned* err;
    double gravity[2];
    int weight;
};

struct SpreadArgs {
    Geo G;
    const DParticle* parts;   // either state buffer (marker ranges only)
    const void* recs;
    const int4* boxes;
    void* flb;                // 2 planes of compute type
    uint8_t* flags;           // [ny][nseg]
    unsigned* err;
};

struct FluidArgs {
    const void* fin;
    void* fout;
    void* flb;
    uint8_t* flags;
    Geo G;
};

struct FieldArgs {
    const void* f;
    Geo G;
    int y0, rows;
    double *rho, *ux, *uy;    // [rows][nx]
};

// kernel launchers (fluid.cu / particles.cu); prec is an lbm_precision
cudaError_t launch_init(int prec, void* f, const Geo& G, int kind, double init_u, cudaStream_t s);
cudaError_t launch_fluid(int prec, const FluidArgs& a, cudaStream_t s);
cudaError_t launch_fields(int prec, const FieldArgs& a, cudaStream_t s);
cudaError_t launch_probes(int prec, const ParticleArgs& a, int nblocks, cudaStream_t s);
cudaError_t launch_markers(int prec, const ParticleArgs& a, int nblocks, cudaStream_t s);
cudaError_t launch_spread(int prec, const SpreadArgs& a, int np, int tiles, cudaStream_t s);
size_t storage_bytes(int prec);
size_t compute_bytes(int prec);
size_t rec_bytes(int prec);

// shapes.cpp: body-frame markers and rigid-body properties of a shape
struct ShapeOut {
    double area, inertia_per_mass, rcirc;
    int n;
};
int make_shape(const lbm_particle_desc& d, double spacing, double* rb, double* nb, double* S,
               int cap, ShapeOut* out);

}  // namespace lbib
