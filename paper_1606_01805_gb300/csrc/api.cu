// api.cu -- host side of the C ABI declared in include/lbib.h: configuration
// checks, the device workspace layout of one lattice or a batch of them,
// particle set-up, the fluid-tile autotuner and the per-step launch sequence
// (probes -> markers -> spreading -> fused fluid step).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "lbib_internal.h"

using namespace lbib;

namespace {
constexpr int GRAPH_STEPS = 32;  // even, so a replay returns to the same buffer
// clock cycles a CTA of the staged fluid kernel waits for a tile's copies
// before it reports ERR_TIMEOUT (about a second at the GB300's 2.07 GHz)
constexpr long long WAIT_LIMIT = 2000000000LL;
}

struct lbm_ctx {
    lbm_config cfg;                 // first configuration: stream, workspace, capacities
    std::vector<lbm_config> icfg;   // per instance
    std::vector<Inst> hinst;        // per instance, host copy
    int ninst = 0;
    int prec;
    size_t sb, cb;                  // bytes per stored / computed element
    cudaStream_t stream;
    void* ws = nullptr;
    bool owns_ws = false;
    void* f[2];
    int cur = 0;
    void* flb;
    uint8_t* flags;
    Inst* insts;
    Task* tasks[N_FLUID_VARIANTS];
    int ntasks[N_FLUID_VARIANTS];
    // tensor maps of the staged variants: [buffer][cells per thread 2, 4][instance]
    // on the device, and their host copies; staged_ok: they could be made
    char* tmaps = nullptr;
    std::vector<unsigned char> htmaps;
    bool staged_ok = false;
    int variant = 0;                // fluid tile shape in use
    int sms = 1;
    size_t rsz, psz;                // bytes of the particle real type R / of DParticleT<R>
    char* parts;                    // two state buffers of cap_particles DParticleT<R> each
    char* poses;                    // two buffers of cap_particles PoseC<C> each (beside parts)
    size_t pcsz;                    // bytes of PoseC<C>
    int4* blk;
    void* partial;                  // R[3][blocks]
    unsigned* count;
    void* mg;                       // MGeo<C>[markers]
    void* S;                        // C[markers]
    void* recs;
    int4* boxes;
    int4* ptab;                     // device copy of hpart
    unsigned* err;
    double* scratch;                // staging area of field and population copies
    int scratch_rows, scratch_cols, scratch_planes;  // its capacity: planes x rows x cols doubles
    int np = 0, nmark = 0, nblk = 0;
    std::vector<int4> hblk;         // host copies of the marker-block table and
    std::vector<int4> hpart;        // of the per-particle (first marker, markers, instance)
    double rc_max = 0;
    int64_t steps = 0;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    int check_every = 1;            // watchdog period of the fluid kernel (steps)
    long long stall_limit = 0;      // lbm_inject_stall: wait limit of the next step's stalled launch
    // GRAPH_STEPS steps from buffer 0 / 1, starting at a step count of each
    // residue modulo check_every (the watchdog steps sit at fixed places)
    cudaGraphExec_t graph[2][GRAPH_STEPS] = {};
    bool graphs_ok = true;
    cudaGraphExec_t timed[2][2] = {};  // one step with its timing events (without / with the watchdog)
    cudaGraphExec_t timed0[2][2] = {}; // the same without the event before the fluid kernel
    bool timed_ok = true;
    bool tuned = false;             // the tile variant was picked (tune_step or lbm_set_tile)
    // fused step of a batch (lbm_set_step_mode): work list and counters
    int step_mode = LBM_STEP_SEPARATE;
    int4* items = nullptr;
    size_t items_cap = 0;
    std::vector<int4> hitems;
    bool items_dirty = true;
    unsigned* counters = nullptr;
    size_t counter_words = 0;       // per set
    // overlapped step of a batch (LBM_STEP_OVERLAP): runs of the instances,
    // each a range of the marker blocks, the particles and every variant's
    // task list; empty when the batch cannot be split that way
    struct Half {
        int b0, b1, p0, p1;
        int t0[N_FLUID_VARIANTS], t1[N_FLUID_VARIANTS];
    };
    std::vector<Half> halves;
    bool halves_dirty = true;
    std::vector<double> hrc;        // per particle: circumscribed radius
    // for the adjoint: body-frame marker geometry in FP64 (rb, nb, S per
    // marker), each marker's particle, each particle's description
    std::vector<double> hgeo;
    std::vector<int> hmpart;
    std::vector<lbm_particle_desc> hdesc;
    long long pop_elems = 0, flb_elems = 0;  // elements of one population buffer / force field
    std::string msg;
};

namespace {

constexpr size_t ALIGN = 256;
size_t up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

int cap_particles(const lbm_config& c) { return c.max_particles > 0 ? c.max_particles : 16; }
int cap_markers(const lbm_config& c) { return c.max_markers > 0 ? c.max_markers : 16384; }
// marker blocks: every particle starts a new block of MB markers
int cap_blocks(const lbm_config& c) { return cap_markers(c) / MB + cap_particles(c) + 1; }

const char* check_config(const lbm_config* c) {
    if (!c) return "null configuration";
    if (c->nx < 3 || c->ny < 3) return "nx and ny must be >= 3";
    if (!(c->tau > 0.5)) return "tau must exceed 1/2";
    for (int i = 0; i < 4; ++i)
        if (c->bc[i] != LBM_BC_PERIODIC && c->bc[i] != LBM_BC_VELOCITY) return "unknown side kind";
    if ((c->bc[0] == LBM_BC_PERIODIC) != (c->bc[1] == LBM_BC_PERIODIC)) return "x sides differ";
    if ((c->bc[2] == LBM_BC_PERIODIC) != (c->bc[3] == LBM_BC_PERIODIC)) return "y sides differ";
    if (c->precision < LBM_FP64 || c->precision > LBM_FP32_TANGENT) return "unknown precision";
    if (c->init < LBM_INIT_REST || c->init > LBM_INIT_TAYLOR_GREEN) return "unknown init";
    if (c->weight < LBM_W_EXP || c->weight > LBM_W_POLY) return "unknown weight";
    if (c->init == LBM_INIT_COUETTE && c->bc[2] != LBM_BC_VELOCITY) return "Couette needs y walls";
    if ((long long)c->nx * c->ny > (1LL << 40)) return "lattice too large";
    if (c->check_every < 0 || c->check_every > GRAPH_STEPS || (c->check_every > 0 && GRAPH_STEPS % c->check_every))
        return "check_every must be 0 or divide 32";
    return nullptr;
}

const char* check_batch(const lbm_config* cfgs, int n) {
    if (!cfgs || n < 1) return "a batch needs at least one configuration";
    for (int i = 0; i < n; ++i) {
        if (const char* why = check_config(cfgs + i)) return why;
        if (cfgs[i].precision != cfgs[0].precision) return "all instances must share one precision";
    }
    return nullptr;
}

Geo make_geo(const lbm_config& c) {
    Geo G;
    std::memset(&G, 0, sizeof G);
    G.nx = c.nx;
    G.ny = c.ny;
    G.pitch = (c.nx + 31) / 32 * 32;
    G.nseg = G.pitch / 32;
    G.plane = (long long)G.pitch * c.ny;
    G.px = c.bc[0] == LBM_BC_PERIODIC;
    G.py = c.bc[2] == LBM_BC_PERIODIC;
    for (int i = 0; i < 4; ++i) {
        G.uw[i][0] = c.wall_u[i][0];
        G.uw[i][1] = c.wall_u[i][1];
        G.uwf[i][0] = (float)c.wall_u[i][0];
        G.uwf[i][1] = (float)c.wall_u[i][1];
    }
    G.g[0] = c.body_force[0];
    G.g[1] = c.body_force[1];
    G.gf[0] = (float)G.g[0];
    G.gf[1] = (float)G.g[1];
    G.grav[0] = c.gravity[0];
    G.grav[1] = c.gravity[1];
    G.tau = c.tau;
    G.omega = 1.0 / c.tau;
    G.omegaf = (float)G.omega;
    return G;
}

// fluid tiles of variant v over all instances
std::vector<Task> make_tasks(const std::vector<Inst>& insts, int v) {
    const int w = 32 * FLUID_VARIANTS[v].cpt, by = FLUID_VARIANTS[v].by;
    std::vector<Task> t;
    for (int i = 0; i < (int)insts.size(); ++i) {
        const Geo& G = insts[i].G;
        for (int ty = 0; ty < (G.ny + by - 1) / by; ++ty)
            for (int tx = 0; tx < (G.nx + w - 1) / w; ++tx) {
                Task k{};
                k.inst = i;
                k.tx = tx;
                k.ty = ty;
                k.pitch = G.pitch;
                k.f_off = insts[i].f_off;
                k.ny = G.ny;
                t.push_back(k);
            }
    }
    return t;
}

struct Layout {
    std::vector<Inst> insts;
    size_t f0, f1, flb, flags, insts_off, tasks[N_FLUID_VARIANTS], tmaps, items, counters, parts, poses, blk,
        partial, count, mg, S, recs, boxes, ptab, err, scratch, total;
    size_t items_cap, counter_words;
    int ntasks[N_FLUID_VARIANTS];
    int scratch_rows, scratch_cols, scratch_planes;
    long long pop_elems, flb_elems;
};

Layout layout(const lbm_config* cfgs, int n) {
    Layout L;
    const lbm_config& c0 = cfgs[0];
    const int prec = c0.precision;
    long long fe = 0, fle = 0, fge = 0;  // elements / bytes so far
    int max_nx = 0;
    for (int i = 0; i < n; ++i) {
        Inst I;
        I.G = make_geo(cfgs[i]);
        I.f_off = fe;
        I.flb_off = fle;
        I.flags_off = fge;
        fe += 9 * I.G.plane;
        fle += 2 * I.G.plane;
        fge += (long long)I.G.ny * I.G.nseg;
        max_nx = std::max(max_nx, I.G.nx);
        L.insts.push_back(I);
    }
    const size_t P = cap_particles(c0), M = cap_markers(c0), NB = cap_blocks(c0);
    // rows of FP64 field output staged per lbm_get_fields chunk (<= 24 MB;
    // the tangent mode adds KT derivative planes per field)
    const int fplanes = prec == LBM_FP32_TANGENT ? 3 * (1 + KT) : 3;
    L.scratch_rows = (int)std::max<size_t>(1, (size_t)(3u << 20) / fplanes / max_nx);
    // at least one row of populations (9 planes) fits
    L.scratch_planes = std::max(fplanes, (9 + L.scratch_rows - 1) / L.scratch_rows);
    L.scratch_cols = max_nx;
    const size_t R = real_bytes(prec);
    size_t o = 0;
    L.f0 = o; o = up(o + fe * storage_bytes(prec));
    L.f1 = o; o = up(o + fe * storage_bytes(prec));
    L.flb = o; o = up(o + fle * force_bytes(prec));
    L.flags = o; o = up(o + fge);
    L.insts_off = o; o = up(o + n * sizeof(Inst));
    for (int v = 0; v < N_FLUID_VARIANTS; ++v) {
        L.ntasks[v] = (int)make_tasks(L.insts, v).size();
        L.tasks[v] = o;
        o = up(o + (size_t)L.ntasks[v] * sizeof(Task));
    }
    L.tmaps = o; o = up(o + 4 * (size_t)n * TMAP_BYTES);
    // the fused step's work list (batches): fluid tiles of its task list,
    // probe and marker items (at most one per 8 marker blocks and one more
    // per particle each), spreading tiles (a particle's support box lies in
    // its lattice: at most (nx / 32 + 3) (ny / 8 + 3) tiles of 32 x 8)
    L.items_cap = 0;
    L.counter_words = 2 * P + n + 2;
    if (n >= 2) {
        int max_ny = 0;
        for (const Inst& I : L.insts) max_ny = std::max(max_ny, I.G.ny);
        L.items_cap = (size_t)L.ntasks[fused_fluid_variant()] + 2 * (NB / MB + P + 1) +
                      P * (size_t)(max_nx / 32 + 3) * (max_ny / fused_spread_rows() + 3);
    }
    L.items = o; o = up(o + L.items_cap * sizeof(int4));
    L.counters = o; o = up(o + 2 * L.counter_words * sizeof(unsigned));
    L.parts = o; o = up(o + 2 * P * particle_bytes(prec));
    L.poses = o; o = up(o + 2 * P * pose_bytes(prec));
    L.blk = o; o = up(o + NB * sizeof(int4));
    L.partial = o; o = up(o + 3 * NB * R);
    L.count = o; o = up(o + P * sizeof(unsigned));
    L.mg = o; o = up(o + M * 4 * compute_bytes(prec));
    L.S = o; o = up(o + M * compute_bytes(prec));
    L.recs = o; o = up(o + M * rec_bytes(prec));
    L.boxes = o; o = up(o + P * sizeof(int4));
    L.ptab = o; o = up(o + P * sizeof(int4));
    L.err = o; o = up(o + 16);
    L.scratch = o; o = up(o + (size_t)L.scratch_planes * L.scratch_rows * max_nx * sizeof(double));
    L.total = o;
    L.pop_elems = fe;
    L.flb_elems = fle;
    return L;
}

lbm_status fail(lbm_ctx* ctx, lbm_status s, const std::string& m) {
    if (ctx) ctx->msg = m;
    return s;
}

lbm_status cuda_fail(lbm_ctx* ctx, cudaError_t e, const char* where) {
    return fail(ctx, LBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                             \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

lbm_status device_error(lbm_ctx* ctx) {
    unsigned e = 0;
    CK(cudaMemcpyAsync(&e, ctx->err, sizeof e, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (e & ERR_DOMAIN) return fail(ctx, LBM_EDOMAIN, "a marker or probe support crossed a wall");
    if (e & ERR_NONFINITE)
        return fail(ctx, LBM_ENONFINITE, "a non-finite value or a non-positive density in the lattice, "
                                         "or a non-finite particle state");
    if (e & ERR_TIMEOUT) return fail(ctx, LBM_ETIMEOUT, "a device wait expired");
    return LBM_OK;
}

// particle state buffer `buf` (0 or 1), and its pose in the compute type
char* state(const lbm_ctx* ctx, int buf) {
    return ctx->parts + (size_t)buf * cap_particles(ctx->cfg) * ctx->psz;
}
char* pose(const lbm_ctx* ctx, int buf) {
    return ctx->poses + (size_t)buf * cap_particles(ctx->cfg) * ctx->pcsz;
}

ParticleArgs particle_args(lbm_ctx* ctx, int cur) {
    ParticleArgs pa;
    pa.f = ctx->f[cur];
    pa.insts = ctx->insts;
    pa.pin = state(ctx, cur);
    pa.pout = state(ctx, cur ^ 1);
    pa.pcin = pose(ctx, cur);
    pa.pcout = pose(ctx, cur ^ 1);
    pa.blk = ctx->blk;
    pa.partial = ctx->partial;
    pa.count = ctx->count;
    pa.mg = ctx->mg;
    pa.S = ctx->S;
    pa.recs = ctx->recs;
    pa.boxes = ctx->boxes;
    pa.flb = ctx->flb;
    pa.flags = ctx->flags;
    pa.err = ctx->err;
    pa.weight = ctx->cfg.weight;
    pa.blk_base = 0;
    pa.single = ctx->ninst == 1;
    pa.one = ctx->hinst[0];
    pa.nblk_inline = ctx->nblk <= INLINE_BLOCKS ? ctx->nblk : 0;
    for (int k = 0; k < pa.nblk_inline; ++k) pa.blk_inline[k] = ctx->hblk[k];
    return pa;
}

SpreadArgs spread_args(lbm_ctx* ctx, const ParticleArgs& pa) {
    SpreadArgs sa;
    sa.insts = ctx->insts;
    sa.ptab = ctx->ptab;
    sa.p_base = 0;
    sa.recs = pa.recs;
    sa.boxes = pa.boxes;
    sa.flb = ctx->flb;
    sa.flags = ctx->flags;
    sa.err = ctx->err;
    sa.single = ctx->ninst == 1;
    sa.one = ctx->hinst[0];
    sa.np_inline = ctx->np <= INLINE_PARTICLES ? ctx->np : 0;
    for (int k = 0; k < sa.np_inline; ++k) sa.part_inline[k] = ctx->hpart[k];
    return sa;
}

// tiles of 32 x 16 cells covering the support box of a particle whose
// markers lie within rc of its centroid (the box spans at most 2 rc + 4
// cells per side), and for the largest particle of the context
int box_tiles(double rc, int rows = 16) {
    const double ext = 2.0 * rc + 4.0;
    return ((int)std::ceil(ext / 32.0) + 1) * ((int)std::ceil(ext / rows) + 1);
}
int spread_tiles(const lbm_ctx* ctx) { return box_tiles(ctx->rc_max); }

// the tile variants this context can run (the staged ones need their tensor maps)
bool ctx_variant_ok(const lbm_ctx* ctx, int v) {
    return variant_valid(ctx->prec, v) && (FLUID_VARIANTS[v].stages == 0 || ctx->staged_ok);
}

// The fluid kernel's watchdog runs on the steps whose count since init
// (1-based) is a multiple of check_every.
bool watched(const lbm_ctx* ctx, int64_t step) { return (step + 1) % ctx->check_every == 0; }

// pdl: launch the fluid kernel with programmatic stream serialization (only
// right after the kernel that spreads the forces -- the marker kernel, or
// the spreading kernel in FP64 and the tangent mode: its prologue loads the
// populations the previous step's fluid kernel wrote); check: the kernel runs its watchdog;
// stall: the test hook of lbm_inject_stall; keep: leave the forces and
// their flags in place (the autotuner's repeated launches of one step)
lbm_status launch_fluid_step(lbm_ctx* ctx, cudaStream_t st, int cur, int v, bool pdl = false,
                             bool check = false, bool stall = false, bool keep = false, int t0 = 0,
                             int tn = -1) {
    FluidArgs fa;
    fa.fin = ctx->f[cur];
    fa.fout = ctx->f[cur ^ 1];
    fa.flb = ctx->flb;
    fa.flags = ctx->flags;
    fa.insts = ctx->insts;
    fa.tasks = ctx->tasks[v] + t0;  // tasks t0 .. t0 + tn - 1 (all by default)
    fa.ntasks = tn < 0 ? ctx->ntasks[v] : tn;
    fa.err = ctx->err;
    fa.check = check ? 1 : 0;
    fa.stall = stall ? 1 : 0;
    fa.keep = keep ? 1 : 0;
    fa.tmaps = fa.tmap_one = nullptr;
    if (FLUID_VARIANTS[v].stages) {
        const size_t k = (size_t)(cur * 2 + (FLUID_VARIANTS[v].cpt == 4 ? 1 : 0)) * ctx->ninst;
        fa.tmaps = ctx->tmaps + k * TMAP_BYTES;
        fa.tmap_one = ctx->htmaps.data() + k * TMAP_BYTES;
    }
    // direct task-list kernel: one CTA per TASKS_PER_CTA tiles (the block
    // scheduler keeps every SM filled as CTAs finish)
    const int grid = std::max(1, (fa.ntasks + TASKS_PER_CTA - 1) / TASKS_PER_CTA);
    CK(launch_fluid(ctx->prec, v, fa, ctx->ninst == 1 ? &ctx->hinst[0] : nullptr, grid, ctx->sms, st, pdl,
                    stall ? ctx->stall_limit : WAIT_LIMIT));
    return LBM_OK;
}

// The fused step's work list, in rounds: round r holds the probe items of
// instance r, the marker items of instance r - D, the spreading tiles of
// r - 2D and the fluid tiles of r - 3D, so that within one instance every
// item follows the items it waits for by about D rounds.  D is chosen so
// that D rounds outlast one stage of a particle (tens of microseconds:
// a probe or marker item is a chain of dependent loads and FP64 work) while
// a round's fluid tiles take about a microsecond of the whole GPU.
constexpr int FUSED_LAG = 32;

lbm_status build_items(lbm_ctx* ctx) {
    const int n = ctx->ninst, rows = fused_spread_rows(), fv = fused_fluid_variant();
    std::vector<std::vector<int4>> pi(n), mi(n), si(n), fi(n);
    std::vector<int> nsp(n, 0);
    for (int p = 0; p < ctx->np; ++p) {
        const int4 pr = ctx->hpart[p];  // (first marker, markers, instance, tiles of 32 x 16)
        const int inst = pr.z, tiles = box_tiles(ctx->hrc[p], rows);
        nsp[inst] += tiles;
        for (int t = 0; t < tiles; ++t) si[inst].push_back(make_int4(FI_SPREAD, t, p, tiles));
    }
    for (int b = 0; b < ctx->nblk;) {  // runs of up to 8 blocks of one particle
        const int p = ctx->hblk[b].x;
        int e = b;
        while (e < ctx->nblk && e - b < 8 && ctx->hblk[e].x == p) ++e;
        const int inst = ctx->hblk[b].w;
        pi[inst].push_back(make_int4(FI_PROBES, b, e - b, p));
        mi[inst].push_back(make_int4(FI_MARKERS, b, e - b, p));
        b = e;
    }
    const std::vector<Task> tasks = make_tasks(ctx->hinst, fv);
    for (int t = 0; t < (int)tasks.size(); ++t)
        fi[tasks[t].inst].push_back(make_int4(FI_FLUID, t, tasks[t].inst, nsp[tasks[t].inst]));
    std::vector<int4>& out = ctx->hitems;
    out.clear();
    for (int r = 0; r < n + 3 * FUSED_LAG; ++r) {
        const int ip = r, im = r - FUSED_LAG, is = r - 2 * FUSED_LAG, iF = r - 3 * FUSED_LAG;
        if (ip < n) out.insert(out.end(), pi[ip].begin(), pi[ip].end());
        if (im >= 0 && im < n) out.insert(out.end(), mi[im].begin(), mi[im].end());
        if (is >= 0 && is < n) out.insert(out.end(), si[is].begin(), si[is].end());
        if (iF >= 0 && iF < n) out.insert(out.end(), fi[iF].begin(), fi[iF].end());
    }
    if (out.size() > ctx->items_cap) return fail(ctx, LBM_EINTERNAL, "fused step work list exceeds its space");
    CK(cudaMemcpyAsync(ctx->items, out.data(), out.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->items_dirty = false;
    return LBM_OK;
}

// the whole step `step` from buffer `cur` as one fused launch
lbm_status launch_fused_step(lbm_ctx* ctx, cudaStream_t st, int cur, int64_t step, bool stall) {
    FusedArgs f;
    std::memset(&f, 0, sizeof f);
    const int fv = fused_fluid_variant();
    f.fa.fin = ctx->f[cur];
    f.fa.fout = ctx->f[cur ^ 1];
    f.fa.flb = ctx->flb;
    f.fa.flags = ctx->flags;
    f.fa.insts = ctx->insts;
    f.fa.tasks = ctx->tasks[fv];
    f.fa.ntasks = ctx->ntasks[fv];
    f.fa.check = watched(ctx, step) ? 1 : 0;
    f.fa.err = ctx->err;
    f.pa = particle_args(ctx, cur);
    f.pa.nblk_inline = 0;  // the block table from memory (the items carry block indices)
    f.sa = spread_args(ctx, f.pa);
    f.items = ctx->items;
    f.nitems = (int)ctx->hitems.size();
    f.np = ctx->np;
    f.ninst = ctx->ninst;
    f.parity = cur;
    f.counters[0] = ctx->counters;
    f.counters[1] = ctx->counters + ctx->counter_words;
    f.wait_limit = stall ? ctx->stall_limit : WAIT_LIMIT;
    f.stall = stall ? 1 : 0;
    f.stall_ticket = 0;
    for (int t = 0; t < f.nitems; ++t)
        if (ctx->hitems[t].x == FI_FLUID) {
            f.stall_ticket = t;
            break;
        }
    CK(launch_step_fused(ctx->prec, f, ctx->sms, st));
    return LBM_OK;
}

bool fused(const lbm_ctx* ctx) { return ctx->step_mode == LBM_STEP_FUSED; }

// The overlapped step's parts: OVERLAP_PARTS runs of instances of about
// equal cell count, each also a run of the particles and of the marker
// blocks (particles numbered in instance order); none when that fails.
constexpr int OVERLAP_PARTS = 2;

void plan_halves(lbm_ctx* ctx) {
    ctx->halves.clear();
    ctx->halves_dirty = false;
    const int n = ctx->ninst, P = std::min(OVERLAP_PARTS, n);
    if (P < 2) return;
    long long tot = 0;
    for (const Inst& I : ctx->hinst) tot += (long long)I.G.nx * I.G.ny;
    // first instance of each part
    std::vector<int> cut(P + 1, n);
    cut[0] = 0;
    long long acc = 0;
    int part = 1;
    for (int i = 0; i < n && part < P; ++i) {
        acc += (long long)ctx->hinst[i].G.nx * ctx->hinst[i].G.ny;
        if (acc * P >= tot * part && i + 1 < n) cut[part++] = i + 1;
    }
    if (part < P) return;
    // the same runs over particles, blocks and tasks (instance never decreasing)
    auto runs = [&](int count, auto inst_of, std::vector<int>& at) {
        at.assign(P + 1, count);
        at[0] = 0;
        int q = 1;
        for (int i = 0; i < count; ++i) {
            if (i > 0 && inst_of(i) < inst_of(i - 1)) return false;
            while (q < P && inst_of(i) >= cut[q]) at[q++] = i;
        }
        return true;
    };
    std::vector<int> pa, ba;
    if (!runs(ctx->np, [&](int p) { return ctx->hpart[p].z; }, pa)) return;
    if (!runs(ctx->nblk, [&](int b) { return ctx->hblk[b].w; }, ba)) return;
    std::vector<lbm_ctx::Half> parts(P);
    for (int q = 0; q < P; ++q) parts[q] = lbm_ctx::Half{ba[q], ba[q + 1], pa[q], pa[q + 1], {}, {}};
    for (int v = 0; v < N_FLUID_VARIANTS; ++v) {
        const std::vector<Task> t = make_tasks(ctx->hinst, v);
        std::vector<int> ta;
        if (!runs((int)t.size(), [&](int i) { return t[i].inst; }, ta)) return;
        for (int q = 0; q < P; ++q) {
            parts[q].t0[v] = ta[q];
            parts[q].t1[v] = ta[q + 1];
        }
    }
    ctx->halves = parts;
}

bool overlapped(const lbm_ctx* ctx) { return ctx->step_mode == LBM_STEP_OVERLAP && ctx->halves.size() >= 2; }

// time step number `step` of one part of the instances from buffer `cur`
// on stream `st`: its IB kernels, then its fluid tasks
lbm_status enqueue_half(lbm_ctx* ctx, cudaStream_t st, int cur, int64_t step, const lbm_ctx::Half& h) {
    const bool ib = h.p1 > h.p0;
    if (ib) {
        ParticleArgs pa = particle_args(ctx, cur);
        pa.blk_base = h.b0;
        CK(launch_probes(ctx->prec, pa, h.b1 - h.b0, st));
        CK(launch_markers(ctx->prec, pa, h.b1 - h.b0, st));
        if (!markers_spread(ctx->prec)) {
            SpreadArgs sa = spread_args(ctx, pa);
            sa.p_base = h.p0;
            CK(launch_spread(ctx->prec, sa, h.p1 - h.p0, spread_tiles(ctx), st));
        }
    }
    const int v = ctx->variant;
    if (h.t1[v] <= h.t0[v]) return LBM_OK;
    return launch_fluid_step(ctx, st, cur, v, ib, watched(ctx, step), false, false, h.t0[v], h.t1[v] - h.t0[v]);
}

// Part of time step number `step` (steps done before it) from buffer `cur`
// on stream `st`: the immersed-boundary kernels (ib = true: probes / rigid
// update / markers, spreading) or the fused fluid kernel over every
// instance (ib = false).  Bookkeeping is the caller's.
lbm_status enqueue_step_part(lbm_ctx* ctx, cudaStream_t st, int cur, int64_t step, bool ib,
                             bool pdl = false, bool stall = false) {
    if (fused(ctx)) return ib ? LBM_OK : launch_fused_step(ctx, st, cur, step, stall);
    if (!ib)
        return launch_fluid_step(ctx, st, cur, ctx->variant, pdl && ctx->np > 0, watched(ctx, step), stall);
    if (ctx->np == 0) return LBM_OK;
    const ParticleArgs pa = particle_args(ctx, cur);
    CK(launch_probes(ctx->prec, pa, ctx->nblk, st));
    CK(launch_markers(ctx->prec, pa, ctx->nblk, st));
    if (!markers_spread(ctx->prec))
        CK(launch_spread(ctx->prec, spread_args(ctx, pa), ctx->np, spread_tiles(ctx), st));
    return LBM_OK;
}

// time step number `step` from buffer `cur` on stream `st` (mid: optional
// event between the IB kernels and the fluid kernel, which then starts only
// after it, so that mid -> end times the fluid kernel alone).  Bookkeeping
// is the caller's.
lbm_status enqueue_step(lbm_ctx* ctx, cudaStream_t st, int cur, int64_t step, cudaEvent_t mid,
                        bool stall = false) {
    lbm_status s = enqueue_step_part(ctx, st, cur, step, true);
    if (s != LBM_OK) return s;
    if (mid) CK(cudaEventRecord(mid, st));
    return enqueue_step_part(ctx, st, cur, step, false, mid == nullptr, stall);
}

// Capture GRAPH_STEPS steps starting from buffer `cur` at step count
// `step` on a private stream (the caller's stream may be the legacy
// default stream, which cannot be captured).  The graph serves every start
// with the same buffer and the same step count modulo check_every.
// Returns false if capture is not possible here.
bool capture_graph(lbm_ctx* ctx, int cur, int64_t step) {
    cudaGraphExec_t& ge = ctx->graph[cur][step % ctx->check_every];
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return false;
    // the overlapped step: every part after the first on a stream of its
    // own, forked from the capture and joined back at its end
    const bool two = overlapped(ctx);
    const int P = two ? (int)ctx->halves.size() : 1;
    std::vector<cudaStream_t> side(P > 1 ? P - 1 : 0, nullptr);
    std::vector<cudaEvent_t> evs(P, nullptr);  // fork, then one join per side stream
    bool made = true;
    for (auto& x : side) made = made && cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) == cudaSuccess;
    if (two)
        for (auto& e : evs) made = made && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    auto release = [&] {
        for (auto x : side)
            if (x) cudaStreamDestroy(x);
        for (auto e : evs)
            if (e) cudaEventDestroy(e);
    };
    if (!made) {
        release();
        cudaStreamDestroy(cs);
        cudaGetLastError();
        return false;
    }
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        int c = cur;
        if (two) {
            ok = cudaEventRecord(evs[0], cs) == cudaSuccess;
            for (auto x : side) ok = ok && cudaStreamWaitEvent(x, evs[0], 0) == cudaSuccess;
            for (int k = 0; k < GRAPH_STEPS && ok; ++k, c ^= 1)
                for (int q = 0; q < P && ok; ++q)
                    ok = enqueue_half(ctx, q ? side[q - 1] : cs, c, step + k, ctx->halves[q]) == LBM_OK;
            // the joins, whatever happened, so that the capture can end
            bool joined = true;
            for (int q = 1; q < P; ++q)
                joined = cudaEventRecord(evs[q], side[q - 1]) == cudaSuccess &&
                         cudaStreamWaitEvent(cs, evs[q], 0) == cudaSuccess && joined;
            ok = ok && joined;
        } else {
            for (int k = 0; k < GRAPH_STEPS && ok; ++k, c ^= 1)
                ok = enqueue_step(ctx, cs, c, step + k, nullptr) == LBM_OK;
        }
        cudaGraph_t g = nullptr;
        const bool ended = cudaStreamEndCapture(cs, &g) == cudaSuccess;
        ok = ok && ended && g && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cs);
    release();
    cudaGetLastError();  // a failed capture leaves no sticky error
    if (!ok) ge = nullptr;
    return ok;
}

// enqueue_step for capture: the event between the IB kernels and the fluid
// kernel (with_mid) is an external record, i.e. a real event-record node
lbm_status enqueue_timed_step(lbm_ctx* ctx, cudaStream_t st, int cur, int64_t step, bool with_mid) {
    lbm_status s = enqueue_step_part(ctx, st, cur, step, true);
    if (s != LBM_OK) return s;
    if (with_mid) CK(cudaEventRecordWithFlags(ctx->ev[1], st, cudaEventRecordExternal));
    return enqueue_step_part(ctx, st, cur, step, false, !with_mid);
}

// One step from buffer `cur` with the timing events recorded inside the
// graph (same launches as enqueue_step, replayed like lbm_step replays);
// with_mid adds the event between the IB kernels and the fluid kernel.  The
// graph serves every step with the same buffer and watchdog setting.
bool capture_timed(lbm_ctx* ctx, int cur, int64_t step, bool with_mid) {
    const int w = watched(ctx, step) ? 1 : 0;
    cudaGraphExec_t& ge = with_mid ? ctx->timed[cur][w] : ctx->timed0[cur][w];
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return false;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        // external records: real event-record nodes, not capture-internal
        // dependencies
        ok = cudaEventRecordWithFlags(ctx->ev[0], cs, cudaEventRecordExternal) == cudaSuccess &&
             enqueue_timed_step(ctx, cs, cur, step, with_mid) == LBM_OK &&
             cudaEventRecordWithFlags(ctx->ev[2], cs, cudaEventRecordExternal) == cudaSuccess;
        cudaGraph_t g = nullptr;
        const bool ended = cudaStreamEndCapture(cs, &g) == cudaSuccess;
        ok = ok && ended && g && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cs);
    cudaGetLastError();
    if (!ok) ge = nullptr;
    return ok;
}

void drop_graphs(lbm_ctx* ctx) {
    for (int c = 0; c < 2; ++c) {
        for (auto& g : ctx->graph[c])
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
        for (int w = 0; w < 2; ++w)
            for (auto* g : {&ctx->timed[c][w], &ctx->timed0[c][w]})
                if (*g) {
                    cudaGraphExecDestroy(*g);
                    *g = nullptr;
                }
    }
}

// Autotuner of the fluid tile variant, run as the context's first step:
// the immersed-boundary kernels of that step run once (so the force field
// and its flags are those of a real step), then the fluid kernel of every
// variant the context has (FLUID_VARIANTS: cells per thread x rows per tile
// x staging depth) is timed on the context's own lattices, reading buffer
// cur, writing the other one and leaving the forces in place; the fastest is
// kept and launched once more as the step's own fluid kernel.  All variants
// compute the same cells with the same arithmetic, so the choice changes
// speed only.  lbm_set_tile before the first step skips it.
lbm_status tune_step(lbm_ctx* ctx, bool* stepped) {
    ctx->tuned = true;
    *stepped = false;
    if (ctx->prec == LBM_FP32_TANGENT || fused(ctx)) return LBM_OK;  // one tile variant only
    struct Events {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Events() {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    CK(cudaEventCreate(&ev.a));
    CK(cudaEventCreate(&ev.b));
    lbm_status s = enqueue_step_part(ctx, ctx->stream, ctx->cur, ctx->steps, true);
    if (s != LBM_OK) return s;
    float best[N_FLUID_VARIANTS];
    for (int v = 0; v < N_FLUID_VARIANTS; ++v) {  // warm every shape first
        best[v] = 1e30f;
        if (!ctx_variant_ok(ctx, v)) continue;
        s = launch_fluid_step(ctx, ctx->stream, ctx->cur, v, false, false, false, true);
        if (s != LBM_OK) return s;
    }
    for (int round = 0; round < 2; ++round)
        for (int v = 0; v < N_FLUID_VARIANTS; ++v) {
            if (!ctx_variant_ok(ctx, v)) continue;
            CK(cudaEventRecord(ev.a, ctx->stream));
            for (int k = 0; k < 2; ++k) {
                s = launch_fluid_step(ctx, ctx->stream, ctx->cur, v, false, false, false, true);
                if (s != LBM_OK) return s;
            }
            CK(cudaEventRecord(ev.b, ctx->stream));
            CK(cudaEventSynchronize(ev.b));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, ev.a, ev.b));
            best[v] = std::min(best[v], ms);
        }
    const int pick = (int)(std::min_element(best, best + N_FLUID_VARIANTS) - best);
    if (pick != ctx->variant) drop_graphs(ctx);
    ctx->variant = pick;
    s = launch_fluid_step(ctx, ctx->stream, ctx->cur, pick, false, watched(ctx, ctx->steps));
    if (s != LBM_OK) return s;
    ctx->cur ^= 1;
    ctx->steps += 1;
    *stepped = true;
    return LBM_OK;
}

lbm_status init_contexts(const lbm_config* cfgs, int n, lbm_ctx** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (check_batch(cfgs, n)) return LBM_EINVAL;
    cudaGetLastError();  // a stale error of earlier work must not fail this context
    Layout L = layout(cfgs, n);
    lbm_ctx* ctx = new lbm_ctx();
    ctx->cfg = cfgs[0];
    ctx->icfg.assign(cfgs, cfgs + n);
    ctx->ninst = n;
    ctx->hinst = L.insts;
    ctx->prec = cfgs[0].precision;
    ctx->sb = storage_bytes(ctx->prec);
    ctx->cb = compute_bytes(ctx->prec);
    ctx->stream = static_cast<cudaStream_t>(cfgs[0].cuda_stream);
    ctx->check_every = cfgs[0].check_every > 0 ? cfgs[0].check_every : 1;
    if (ctx->prec == LBM_FP32_TANGENT) ctx->variant = 2;  // its one tile variant
    if (cfgs[0].d_workspace) {
        if (cfgs[0].workspace_bytes < L.total) {
            delete ctx;
            return LBM_ENOMEM;
        }
        ctx->ws = cfgs[0].d_workspace;
    } else {
        if (cudaMalloc(&ctx->ws, L.total) != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return LBM_ENOMEM;
        }
        ctx->owns_ws = true;
    }
    char* b = static_cast<char*>(ctx->ws);
    ctx->f[0] = b + L.f0;
    ctx->f[1] = b + L.f1;
    ctx->flb = b + L.flb;
    ctx->flags = reinterpret_cast<uint8_t*>(b + L.flags);
    ctx->insts = reinterpret_cast<Inst*>(b + L.insts_off);
    for (int v = 0; v < N_FLUID_VARIANTS; ++v) {
        ctx->tasks[v] = reinterpret_cast<Task*>(b + L.tasks[v]);
        ctx->ntasks[v] = L.ntasks[v];
    }
    ctx->tmaps = b + L.tmaps;
    ctx->pop_elems = L.pop_elems;
    ctx->flb_elems = L.flb_elems;
    ctx->items = reinterpret_cast<int4*>(b + L.items);
    ctx->items_cap = L.items_cap;
    ctx->counters = reinterpret_cast<unsigned*>(b + L.counters);
    ctx->counter_words = L.counter_words;
    ctx->rsz = real_bytes(ctx->prec);
    ctx->psz = particle_bytes(ctx->prec);
    ctx->parts = b + L.parts;
    ctx->pcsz = pose_bytes(ctx->prec);
    ctx->poses = b + L.poses;
    ctx->blk = reinterpret_cast<int4*>(b + L.blk);
    ctx->partial = b + L.partial;
    ctx->count = reinterpret_cast<unsigned*>(b + L.count);
    ctx->mg = b + L.mg;
    ctx->S = b + L.S;
    ctx->recs = b + L.recs;
    ctx->boxes = reinterpret_cast<int4*>(b + L.boxes);
    ctx->ptab = reinterpret_cast<int4*>(b + L.ptab);
    ctx->err = reinterpret_cast<unsigned*>(b + L.err);
    ctx->scratch = reinterpret_cast<double*>(b + L.scratch);
    ctx->scratch_rows = L.scratch_rows;
    ctx->scratch_cols = L.scratch_cols;
    ctx->scratch_planes = L.scratch_planes;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
    // a batch steps its instances in overlapped parts by default
    if (n >= 2) ctx->step_mode = LBM_STEP_OVERLAP;
    if (ctx->sms < 1) ctx->sms = 1;
    std::vector<std::vector<Task>> tasks(N_FLUID_VARIANTS);
    for (int v = 0; v < N_FLUID_VARIANTS; ++v) tasks[v] = make_tasks(L.insts, v);
    // zero everything (padding columns, force fields, flags, error word),
    // then the instance table, the tile lists and the initial fields
    cudaError_t e = cudaMemsetAsync(ctx->ws, 0, L.total, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ctx->insts, L.insts.data(), n * sizeof(Inst), cudaMemcpyHostToDevice, ctx->stream);
    for (int v = 0; v < N_FLUID_VARIANTS && e == cudaSuccess; ++v)
        e = cudaMemcpyAsync(ctx->tasks[v], tasks[v].data(), tasks[v].size() * sizeof(Task),
                            cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && (ctx->prec == LBM_FP32 || ctx->prec == LBM_FP16_SHIFTED)) {
        // the staged variants' tensor maps; without them those variants are off
        ctx->htmaps.assign(4 * (size_t)n * TMAP_BYTES, 0);
        ctx->staged_ok = true;
        for (int bf = 0; bf < 2 && ctx->staged_ok; ++bf)
            for (int c = 0; c < 2 && ctx->staged_ok; ++c)
                for (int i = 0; i < n && ctx->staged_ok; ++i)
                    ctx->staged_ok = encode_stage_map(ctx->prec, c ? 4 : 2, ctx->f[bf], L.insts[i],
                                                      ctx->htmaps.data() + ((bf * 2 + c) * (size_t)n + i) *
                                                                               TMAP_BYTES) == cudaSuccess;
        if (ctx->staged_ok)
            e = cudaMemcpyAsync(ctx->tmaps, ctx->htmaps.data(), ctx->htmaps.size(), cudaMemcpyHostToDevice,
                                ctx->stream);
    }
    for (int i = 0; i < n && e == cudaSuccess; ++i)
        e = launch_init(ctx->prec, ctx->f[0], L.insts[i], cfgs[i].init, cfgs[i].init_u, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ctx->owns_ws) cudaFree(ctx->ws);
        delete ctx;
        return LBM_ECUDA;
    }
    *out = ctx;
    return LBM_OK;
}

// seeds of the tangent mode: d(dim0, dim1, xc, yc, theta, rho_s)/dp_k
constexpr int NSEED = 6;
template <class R> R seeded(double v, const double* seed, int j);
template <> double seeded<double>(double v, const double*, int) { return v; }
template <> TD seeded<TD>(double v, const double* seed, int j) {
    TD r(v);
    for (int k = 0; k < KT; ++k) r.d[k] = seed ? seed[k * NSEED + j] : 0.0;
    return r;
}

template <class R, class C>
lbm_status add_particle_t(lbm_ctx* ctx, int inst, const lbm_particle_desc* d, const double* seed,
                          int32_t* out_id) {
    using std::cos;
    using std::sin;
    const Geo& G = ctx->hinst[inst].G;
    const int room = cap_markers(ctx->cfg) - ctx->nmark;
    const size_t cap = (size_t)std::max(room, 0) + 1;
    std::vector<R> rb(2 * cap), nb(2 * cap), S(cap);
    const R dim[2] = {seeded<R>(d->dim[0], seed, 0), seeded<R>(d->dim[1], seed, 1)};
    ShapeOutT<R> so;
    if (make_shape_t<R>(*d, dim, ctx->icfg[inst].marker_spacing, rb.data(), nb.data(), S.data(), room, &so) < 0)
        return fail(ctx, LBM_EINVAL, "marker capacity exceeded");
    const int n = so.n;
    const R xc = seeded<R>(d->xc, seed, 2), yc = seeded<R>(d->yc, seed, 3);
    const R th = seeded<R>(d->theta, seed, 4), rho_s = seeded<R>(d->rho_s, seed, 5);
    const R c = cos(th), s = sin(th);
    // every marker and probe support must stay inside the walls
    for (int l = 0; l < n; ++l) {
        const double cv = value_of(c), sv = value_of(s);
        const double rx = value_of(rb[2 * l]), ry = value_of(rb[2 * l + 1]);
        const double nx0 = value_of(nb[2 * l]), ny0 = value_of(nb[2 * l + 1]);
        const double x = d->xc + cv * rx - sv * ry, y = d->yc + sv * rx + cv * ry;
        const double nx = cv * nx0 - sv * ny0, ny = sv * nx0 + cv * ny0;
        for (int pass = 0; pass < 2; ++pass) {
            const double px = x + pass * 1.2 * nx, py = y + pass * 1.2 * ny;
            const int i0 = (int)std::floor(px + 0.5), j0 = (int)std::floor(py + 0.5);
            if (!G.px && (i0 - 1 < 0 || i0 + 1 > G.nx - 1))
                return fail(ctx, LBM_EINVAL, "particle support crosses an x wall");
            if (!G.py && (j0 - 1 < 0 || j0 + 1 > G.ny - 1))
                return fail(ctx, LBM_EINVAL, "particle support crosses a y wall");
        }
    }
    DParticleT<R> P;
    std::memset(&P, 0, sizeof P);
    for (int h = 0; h < 2; ++h) {
        P.X[h][0] = xc;
        P.X[h][1] = yc;
        P.th[h] = th;
        P.cs[h][0] = c;
        P.cs[h][1] = s;
        P.U[h][0] = R(d->u0[0]);
        P.U[h][1] = R(d->u0[1]);
        P.W[h] = R(d->omega0);
    }
    P.area = so.area;
    P.rho_s = rho_s;
    P.mass = rho_s * so.area;
    P.inertia = P.mass * so.inertia_per_mass;
    P.inv_mass = R(1.0) / P.mass;
    P.inv_inertia = R(1.0) / P.inertia;
    P.m0 = ctx->nmark;
    P.nm = n;
    P.b0 = ctx->nblk;
    P.nblk = (n + MB - 1) / MB;
    P.inst = inst;
    if (P.b0 + P.nblk > cap_blocks(ctx->cfg)) return fail(ctx, LBM_EINVAL, "marker capacity exceeded");
    std::vector<int4> blocks(P.nblk);
    for (int k = 0; k < P.nblk; ++k)
        blocks[k] = make_int4(ctx->np, P.m0 + k * MB, std::min(MB, n - k * MB), inst);
    // the marker kernels' geometry in the compute type C
    static_assert(sizeof(MGeo<C>) == 4 * sizeof(C), "marker geometry is packed");
    std::vector<MGeo<C>> mg(n);
    std::vector<C> Sc(n);
    for (int l = 0; l < n; ++l) {
        mg[l] = MGeo<C>{C(rb[2 * l]), C(rb[2 * l + 1]), C(nb[2 * l]), C(nb[2 * l + 1])};
        Sc[l] = C(S[l]);
    }
    // the initial pose in C (both stored levels equal: no changes)
    PoseC<C> pc;
    std::memset(&pc, 0, sizeof pc);
    const double fx = std::floor(value_of(xc)), fy = std::floor(value_of(yc));
    pc.ix = (int)fx;
    pc.iy = (int)fy;
    pc.v[PC_XF] = C(xc - R(fx));
    pc.v[PC_YF] = C(yc - R(fy));
    pc.v[PC_C] = C(c);
    pc.v[PC_S] = C(s);
    pc.v[PC_U] = C(R(d->u0[0]));
    pc.v[PC_V] = C(R(d->u0[1]));
    pc.v[PC_W] = pc.v[PC_W1] = C(R(d->omega0));
    pc.v[PC_DU] = pc.v[PC_DV] = pc.v[PC_DW] = pc.v[PC_DC] = pc.v[PC_DS] = C(0.0f);
    CK(cudaMemcpyAsync(static_cast<MGeo<C>*>(ctx->mg) + P.m0, mg.data(), n * sizeof(MGeo<C>),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(static_cast<C*>(ctx->S) + P.m0, Sc.data(), n * sizeof(C), cudaMemcpyHostToDevice,
                       ctx->stream));
    for (int buf = 0; buf < 2; ++buf) {
        CK(cudaMemcpyAsync(state(ctx, buf) + (size_t)ctx->np * sizeof P, &P, sizeof P, cudaMemcpyHostToDevice,
                           ctx->stream));
        CK(cudaMemcpyAsync(pose(ctx, buf) + (size_t)ctx->np * sizeof pc, &pc, sizeof pc,
                           cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaMemcpyAsync(ctx->blk + P.b0, blocks.data(), P.nblk * sizeof(int4), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graphs(ctx);  // captured steps do not know this particle
    ctx->rc_max = std::max(ctx->rc_max, so.rcirc);
    ctx->hrc.push_back(so.rcirc);
    ctx->items_dirty = true;
    ctx->hdesc.push_back(*d);
    for (int l = 0; l < n; ++l) {
        const double g5[5] = {value_of(rb[2 * l]), value_of(rb[2 * l + 1]), value_of(nb[2 * l]),
                              value_of(nb[2 * l + 1]), value_of(S[l])};
        ctx->hgeo.insert(ctx->hgeo.end(), g5, g5 + 5);
        ctx->hmpart.push_back(ctx->np);
    }
    ctx->hblk.insert(ctx->hblk.end(), blocks.begin(), blocks.end());
    ctx->hpart.push_back(make_int4(P.m0, n, inst, box_tiles(so.rcirc)));
    ctx->halves_dirty = true;
    CK(cudaMemcpyAsync(ctx->ptab + ctx->np, &ctx->hpart.back(), sizeof(int4), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->nmark += n;
    ctx->nblk += P.nblk;
    if (out_id) *out_id = ctx->np;
    ctx->np += 1;
    return LBM_OK;
}

lbm_status add_particle(lbm_ctx* ctx, int inst, const lbm_particle_desc* d, const double* seed,
                        int32_t* out_id) {
    if (!ctx || !d) return LBM_EINVAL;
    if (inst < 0 || inst >= ctx->ninst) return fail(ctx, LBM_EINVAL, "no such instance");
    if (ctx->steps > 0) return fail(ctx, LBM_EINVAL, "particles must be added before the first step");
    if (ctx->np >= cap_particles(ctx->cfg)) return fail(ctx, LBM_EINVAL, "particle capacity exceeded");
    if (d->shape < LBM_SHAPE_CIRCLE || d->shape > LBM_SHAPE_TRIANGLE || !(d->dim[0] > 0) ||
        !(d->rho_s > 0))
        return fail(ctx, LBM_EINVAL, "bad particle shape, size or density");
    if ((d->shape == LBM_SHAPE_ELLIPSE || d->shape == LBM_SHAPE_RECT) && !(d->dim[1] > 0))
        return fail(ctx, LBM_EINVAL, "shape needs two dimensions");
    if (seed && ctx->prec != LBM_FP32_TANGENT)
        return fail(ctx, LBM_EINVAL, "tangent seeds need the LBM_FP32_TANGENT precision");
    if (ctx->prec == LBM_FP32_TANGENT) return add_particle_t<TD, TF>(ctx, inst, d, seed, out_id);
    if (ctx->prec == LBM_FP64) return add_particle_t<double, double>(ctx, inst, d, nullptr, out_id);
    return add_particle_t<double, float>(ctx, inst, d, nullptr, out_id);
}

lbm_status get_fields(lbm_ctx* ctx, int inst, double* rho, double* ux, double* uy,
                      double* drho = nullptr, double* dux = nullptr, double* duy = nullptr) {
    if (!ctx) return LBM_EINVAL;
    const bool tan = drho || dux || duy;
    if (tan && ctx->prec != LBM_FP32_TANGENT)
        return fail(ctx, LBM_EINVAL, "field tangents need the LBM_FP32_TANGENT precision");
    if (inst < 0 || inst >= ctx->ninst) return fail(ctx, LBM_EINVAL, "no such instance");
    lbm_status s = device_error(ctx);
    if (s != LBM_OK) return s;
    const Inst& I = ctx->hinst[inst];
    const int nx = I.G.nx, ny = I.G.ny;
    const size_t chunk = (size_t)ctx->scratch_rows * nx;
    for (int y0 = 0; y0 < ny; y0 += ctx->scratch_rows) {
        const int rows = std::min(ctx->scratch_rows, ny - y0);
        FieldArgs fa;
        fa.f = ctx->f[ctx->cur];
        fa.I = I;
        fa.y0 = y0;
        fa.rows = rows;
        fa.rho = ctx->scratch;
        fa.ux = ctx->scratch + chunk;
        fa.uy = ctx->scratch + 2 * chunk;
        fa.tan = tan ? ctx->scratch + 3 * chunk : nullptr;  // [3][KT][rows][nx]
        CK(launch_fields(ctx->prec, fa, ctx->stream));
        const size_t n = (size_t)rows * nx, off = (size_t)y0 * nx;
        if (rho) CK(cudaMemcpyAsync(rho + off, fa.rho, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
        if (ux) CK(cudaMemcpyAsync(ux + off, fa.ux, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
        if (uy) CK(cudaMemcpyAsync(uy + off, fa.uy, n * 8, cudaMemcpyDeviceToHost, ctx->stream));
        double* outs[3] = {drho, dux, duy};
        for (int q = 0; q < 3 && tan; ++q)
            for (int k = 0; k < KT && outs[q]; ++k)
                CK(cudaMemcpyAsync(outs[q] + (size_t)k * nx * ny + off, fa.tan + (size_t)(q * KT + k) * n, n * 8,
                                   cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return LBM_OK;
}

// rows of one population chunk through the staging area (9 planes of
// doubles per row)
int pop_rows(const lbm_ctx* ctx, int nx) {
    const size_t cap = (size_t)ctx->scratch_rows * ctx->scratch_cols * ctx->scratch_planes;
    return (int)std::max<size_t>(1, cap / (9 * (size_t)nx));
}

// populations host <-> device in chunks of rows through the staging area:
// one 2-D copy (9 plane segments) and one conversion kernel per chunk, in
// stream order; the host array is [9][ny][nx] doubles
lbm_status get_populations(lbm_ctx* ctx, int inst, double* f) {
    if (!ctx || !f) return LBM_EINVAL;
    if (inst < 0 || inst >= ctx->ninst) return fail(ctx, LBM_EINVAL, "no such instance");
    const Inst& I = ctx->hinst[inst];
    const int nx = I.G.nx, ny = I.G.ny, R = pop_rows(ctx, nx);
    for (int y0 = 0; y0 < ny; y0 += R) {
        const int rows = std::min(R, ny - y0);
        CK(launch_get_pops(ctx->prec, ctx->f[ctx->cur], I, y0, rows, ctx->scratch, ctx->stream));
        const size_t w = (size_t)rows * nx * sizeof(double);
        CK(cudaMemcpy2DAsync(f + (size_t)y0 * nx, (size_t)ny * nx * sizeof(double), ctx->scratch, w, w, 9,
                             cudaMemcpyDeviceToHost, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

lbm_status set_populations(lbm_ctx* ctx, int inst, const double* f) {
    if (!ctx || !f) return LBM_EINVAL;
    if (inst < 0 || inst >= ctx->ninst) return fail(ctx, LBM_EINVAL, "no such instance");
    const Inst& I = ctx->hinst[inst];
    const int nx = I.G.nx, ny = I.G.ny, R = pop_rows(ctx, nx);
    for (int y0 = 0; y0 < ny; y0 += R) {
        const int rows = std::min(R, ny - y0);
        const size_t w = (size_t)rows * nx * sizeof(double);
        CK(cudaMemcpy2DAsync(ctx->scratch, w, f + (size_t)y0 * nx, (size_t)ny * nx * sizeof(double), w, 9,
                             cudaMemcpyHostToDevice, ctx->stream));
        CK(launch_put_pops(ctx->prec, ctx->scratch, I, y0, rows, ctx->f[ctx->cur], ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return LBM_OK;
}

// the first m particles of the current state buffer: values into `out`,
// and in the tangent mode d(state)/dp_k into `tan` ([m][KT][LBM_TANGENT_FIELDS])
template <class R>
lbm_status read_particles(lbm_ctx* ctx, int m, lbm_particle_state* out, double* tan) {
    std::vector<DParticleT<R>> h(m);
    CK(cudaMemcpyAsync(h.data(), state(ctx, ctx->cur), m * sizeof(DParticleT<R>), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < m; ++i) {
        const DParticleT<R>& P = h[i];
        const R* q[LBM_TANGENT_FIELDS] = {&P.X[0][0], &P.X[0][1], &P.th[0], &P.U[0][0], &P.U[0][1],
                                          &P.W[0],    &P.F[0],    &P.F[1],  &P.M,       &P.wsum};
        if (out) {
            out[i].xc = value_of(*q[0]);
            out[i].yc = value_of(*q[1]);
            out[i].theta = value_of(*q[2]);
            out[i].u[0] = value_of(*q[3]);
            out[i].u[1] = value_of(*q[4]);
            out[i].omega = value_of(*q[5]);
            out[i].F[0] = value_of(*q[6]);
            out[i].F[1] = value_of(*q[7]);
            out[i].M = value_of(*q[8]);
            out[i].omega_sum = value_of(*q[9]);
        }
        if (tan)
            for (int k = 0; k < KT; ++k)
                for (int j = 0; j < LBM_TANGENT_FIELDS; ++j)
                    tan[((size_t)i * KT + k) * LBM_TANGENT_FIELDS + j] = derivative(*q[j], k);
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_workspace_bytes(const lbm_config* cfgs, int32_t n, size_t* bytes) {
    if (check_batch(cfgs, n) || !bytes) return LBM_EINVAL;
    *bytes = layout(cfgs, n).total;
    return LBM_OK;
}

lbm_status lbm_workspace_bytes(const lbm_config* cfg, size_t* bytes) {
    return lbm_batch_workspace_bytes(cfg, 1, bytes);
}

lbm_status lbm_init(const lbm_config* cfg, lbm_ctx** out) { return init_contexts(cfg, 1, out); }

lbm_status lbm_init_batch(const lbm_config* cfgs, int32_t n, lbm_ctx** out) {
    return init_contexts(cfgs, n, out);
}

int32_t lbm_instances(const lbm_ctx* ctx) { return ctx ? ctx->ninst : 0; }

lbm_status lbm_add_particle(lbm_ctx* ctx, const lbm_particle_desc* d, int32_t* out_id) {
    return add_particle(ctx, 0, d, nullptr, out_id);
}

lbm_status lbm_add_particle_to(lbm_ctx* ctx, int32_t instance, const lbm_particle_desc* d,
                               int32_t* out_id) {
    return add_particle(ctx, instance, d, nullptr, out_id);
}

lbm_status lbm_add_particle_tangent(lbm_ctx* ctx, int32_t instance, const lbm_particle_desc* d,
                                    const double* seed, int32_t* out_id) {
    if (!seed) return fail(ctx, LBM_EINVAL, "no tangent seeds");
    return add_particle(ctx, instance, d, seed, out_id);
}

lbm_status lbm_set_wall_tangents(lbm_ctx* ctx, int32_t instance, const double* dwall) {
    if (!ctx || !dwall) return LBM_EINVAL;
    if (ctx->prec != LBM_FP32_TANGENT) return fail(ctx, LBM_EINVAL, "wall tangents need LBM_FP32_TANGENT");
    if (instance < 0 || instance >= ctx->ninst) return fail(ctx, LBM_EINVAL, "no such instance");
    if (ctx->steps > 0) return fail(ctx, LBM_EINVAL, "wall tangents must be set before the first step");
    Inst& I = ctx->hinst[instance];
    for (int sd = 0; sd < 4; ++sd)
        for (int c = 0; c < 2; ++c)
            for (int k = 0; k < KT; ++k) {
                const double v = dwall[(sd * 2 + c) * KT + k];
                I.G.uwd[sd][c][k] = v;
                I.G.uwdf[sd][c][k] = (float)v;
            }
    CK(cudaMemcpyAsync(ctx->insts + instance, &I, sizeof(Inst), cudaMemcpyHostToDevice, ctx->stream));
    // the initial field (a Couette profile) follows the wall speeds
    CK(launch_init(ctx->prec, ctx->f[ctx->cur], I, ctx->icfg[instance].init, ctx->icfg[instance].init_u,
                   ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    drop_graphs(ctx);  // a single-lattice step carries the descriptor by value
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* ctx, int32_t nsteps) {
    if (!ctx || nsteps < 0) return LBM_EINVAL;
    if (fused(ctx) && ctx->items_dirty && nsteps > 0) {  // the work list, before any capture
        lbm_status s = build_items(ctx);
        if (s != LBM_OK) return s;
    }
    if (ctx->step_mode == LBM_STEP_OVERLAP && ctx->halves_dirty) {  // before any capture
        drop_graphs(ctx);
        plan_halves(ctx);
    }
    if (!ctx->tuned && nsteps > 0) {  // the first step picks the tile variant
        bool stepped = false;
        lbm_status s = tune_step(ctx, &stepped);
        if (s != LBM_OK) return s;
        if (stepped) nsteps -= 1;
    }
    if (ctx->stall_limit && nsteps > 0) {  // lbm_inject_stall: this step alone, launched directly
        lbm_status s = enqueue_step(ctx, ctx->stream, ctx->cur, ctx->steps, nullptr, true);
        ctx->stall_limit = 0;
        if (s != LBM_OK) return s;
        ctx->cur ^= 1;
        ctx->steps += 1;
        nsteps -= 1;
    }
    // long runs replay a captured graph of GRAPH_STEPS steps (launch-bound
    // small lattices), the remainder is launched directly
    while (nsteps >= GRAPH_STEPS && ctx->graphs_ok) {
        cudaGraphExec_t& ge = ctx->graph[ctx->cur][ctx->steps % ctx->check_every];
        if (!ge && !capture_graph(ctx, ctx->cur, ctx->steps)) {
            ctx->graphs_ok = false;
            break;
        }
        CK(cudaGraphLaunch(ge, ctx->stream));
        ctx->steps += GRAPH_STEPS;
        nsteps -= GRAPH_STEPS;
    }
    for (int32_t k = 0; k < nsteps; ++k) {
        lbm_status s = enqueue_step(ctx, ctx->stream, ctx->cur, ctx->steps, nullptr);
        if (s != LBM_OK) return s;
        ctx->cur ^= 1;
        ctx->steps += 1;
    }
    return LBM_OK;
}

lbm_status lbm_step_timed(lbm_ctx* ctx, int32_t nsteps, double* ms_step, double* ms_fluid) {
    if (!ctx || nsteps < 0) return LBM_EINVAL;
    for (auto& e : ctx->ev)
        if (!e) CK(cudaEventCreate(&e));
    double tot = 0, flu = 0;
    // the event before the fluid kernel only when its time is asked for: it
    // keeps the fluid kernel from starting before the forces are spread
    const bool mid = ms_fluid != nullptr;
    if (fused(ctx) && ctx->items_dirty && nsteps > 0) {
        lbm_status s = build_items(ctx);
        if (s != LBM_OK) return s;
    }
    if (!ctx->tuned && nsteps > 0) {  // the first step picks the tile variant (untimed)
        bool stepped = false;
        lbm_status s = tune_step(ctx, &stepped);
        if (s != LBM_OK) return s;
        if (stepped) nsteps -= 1;
    }
    for (int32_t k = 0; k < nsteps; ++k) {
        // each step is a replay of its captured one-step graph (as lbm_step
        // replays steps), with the timing events inside it
        cudaGraphExec_t& ge = (mid ? ctx->timed : ctx->timed0)[ctx->cur][watched(ctx, ctx->steps) ? 1 : 0];
        if (ctx->timed_ok && !ge && !capture_timed(ctx, ctx->cur, ctx->steps, mid)) ctx->timed_ok = false;
        if (ctx->timed_ok) {
            CK(cudaGraphLaunch(ge, ctx->stream));
        } else {
            CK(cudaEventRecord(ctx->ev[0], ctx->stream));
            lbm_status s = enqueue_step(ctx, ctx->stream, ctx->cur, ctx->steps, mid ? ctx->ev[1] : nullptr);
            if (s != LBM_OK) return s;
            CK(cudaEventRecord(ctx->ev[2], ctx->stream));
        }
        ctx->cur ^= 1;
        ctx->steps += 1;
        CK(cudaEventSynchronize(ctx->ev[2]));
        float a = 0, b = 0;
        CK(cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[2]));
        if (mid) CK(cudaEventElapsedTime(&b, ctx->ev[1], ctx->ev[2]));
        tot += a;
        flu += b;
    }
    if (ms_step) *ms_step += tot;
    if (ms_fluid) *ms_fluid += flu;
    return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* ctx) {
    if (!ctx) return LBM_EINVAL;
    return device_error(ctx);
}

lbm_status lbm_inject_stall(lbm_ctx* ctx, int64_t wait_cycles) {
    if (!ctx) return LBM_EINVAL;
    if (!FLUID_VARIANTS[ctx->variant].stages && !fused(ctx))
        return fail(ctx, LBM_EINVAL, "neither a staged tile variant nor the fused step: nothing to stall");
    if (wait_cycles < 1000000 || wait_cycles > WAIT_LIMIT)
        return fail(ctx, LBM_EINVAL, "wait_cycles must lie in [1e6, 2e9]");
    ctx->stall_limit = wait_cycles;
    return LBM_OK;
}

lbm_status lbm_inject_status(lbm_ctx* ctx, int32_t status) {
    if (!ctx) return LBM_EINVAL;
    unsigned bits = 0;
    if (status == LBM_EDOMAIN) bits = ERR_DOMAIN;
    else if (status == LBM_ENONFINITE) bits = ERR_NONFINITE;
    else if (status == LBM_ETIMEOUT) bits = ERR_TIMEOUT;
    else return fail(ctx, LBM_EINVAL, "only LBM_EDOMAIN, LBM_ENONFINITE and LBM_ETIMEOUT can be injected");
    CK(launch_raise(ctx->err, bits, ctx->stream));
    return LBM_OK;
}

lbm_status lbm_get_fields(lbm_ctx* ctx, double* rho, double* ux, double* uy) {
    return get_fields(ctx, 0, rho, ux, uy);
}

lbm_status lbm_get_instance_fields(lbm_ctx* ctx, int32_t instance, double* rho, double* ux, double* uy) {
    return get_fields(ctx, instance, rho, ux, uy);
}

lbm_status lbm_get_field_tangents(lbm_ctx* ctx, int32_t instance, double* drho, double* dux, double* duy) {
    if (!drho && !dux && !duy) return fail(ctx, LBM_EINVAL, "no output");
    return get_fields(ctx, instance, nullptr, nullptr, nullptr, drho, dux, duy);
}

lbm_status lbm_get_populations(lbm_ctx* ctx, double* f) { return get_populations(ctx, 0, f); }

lbm_status lbm_get_instance_populations(lbm_ctx* ctx, int32_t instance, double* f) {
    return get_populations(ctx, instance, f);
}

lbm_status lbm_set_populations(lbm_ctx* ctx, const double* f) { return set_populations(ctx, 0, f); }

lbm_status lbm_set_instance_populations(lbm_ctx* ctx, int32_t instance, const double* f) {
    return set_populations(ctx, instance, f);
}

lbm_status lbm_get_particles(lbm_ctx* ctx, lbm_particle_state* out, int32_t cap, int32_t* n) {
    if (!ctx) return LBM_EINVAL;
    lbm_status s = device_error(ctx);
    if (s != LBM_OK && s != LBM_EDOMAIN) return s;
    if (n) *n = ctx->np;
    if (ctx->np == 0 || !out || cap <= 0) return s;
    const int m = std::min<int>(cap, ctx->np);
    lbm_status r = ctx->prec == LBM_FP32_TANGENT ? read_particles<TD>(ctx, m, out, nullptr)
                                                 : read_particles<double>(ctx, m, out, nullptr);
    return r != LBM_OK ? r : s;
}

lbm_status lbm_get_particle_tangents(lbm_ctx* ctx, double* out, int32_t cap, int32_t* n) {
    if (!ctx) return LBM_EINVAL;
    if (ctx->prec != LBM_FP32_TANGENT) return fail(ctx, LBM_EINVAL, "particle tangents need LBM_FP32_TANGENT");
    lbm_status s = device_error(ctx);
    if (s != LBM_OK && s != LBM_EDOMAIN) return s;
    if (n) *n = ctx->np;
    if (ctx->np == 0 || !out || cap <= 0) return s;
    lbm_status r = read_particles<TD>(ctx, std::min<int>(cap, ctx->np), nullptr, out);
    return r != LBM_OK ? r : s;
}

lbm_status lbm_get_tile(const lbm_ctx* ctx, int32_t* variant, int32_t* cells_per_thread,
                        int32_t* rows_per_block) {
    if (!ctx) return LBM_EINVAL;
    if (variant) *variant = ctx->variant;
    if (cells_per_thread) *cells_per_thread = FLUID_VARIANTS[ctx->variant].cpt;
    if (rows_per_block) *rows_per_block = FLUID_VARIANTS[ctx->variant].by;
    return LBM_OK;
}

lbm_status lbm_tile_info(int32_t variant, int32_t precision, int32_t* cells_per_thread, int32_t* rows,
                         int32_t* stages) {
    if (variant < 0 || variant >= N_FLUID_VARIANTS) return LBM_EINVAL;
    const FluidVariant& fv = FLUID_VARIANTS[variant];
    if (cells_per_thread) *cells_per_thread = fv.cpt;
    if (rows) *rows = fv.by;
    if (stages) *stages = fv.stages;
    return variant_valid(precision, variant) ? LBM_OK : LBM_EINVAL;
}

lbm_status lbm_set_tile(lbm_ctx* ctx, int32_t variant) {
    if (!ctx) return LBM_EINVAL;
    if (variant < 0 || variant >= N_FLUID_VARIANTS) return fail(ctx, LBM_EINVAL, "no such tile variant");
    if (!ctx_variant_ok(ctx, variant))
        return fail(ctx, LBM_EINVAL, "the precision has no such tile variant");
    ctx->tuned = true;
    if (variant != ctx->variant) {
        ctx->variant = variant;
        drop_graphs(ctx);  // captured steps launch the old shape
    }
    return LBM_OK;
}

lbm_status lbm_set_step_mode(lbm_ctx* ctx, int32_t mode) {
    if (!ctx) return LBM_EINVAL;
    if (mode != LBM_STEP_SEPARATE && mode != LBM_STEP_FUSED && mode != LBM_STEP_OVERLAP)
        return fail(ctx, LBM_EINVAL, "no such step mode");
    if (mode == LBM_STEP_OVERLAP && ctx->ninst < 2)
        return fail(ctx, LBM_EINVAL, "the overlapped step is for batches of two or more instances");
    if (mode == LBM_STEP_FUSED && ctx->prec == LBM_FP32_TANGENT)
        return fail(ctx, LBM_EINVAL, "the fused step has no tangent mode");
    if (mode == LBM_STEP_FUSED && ctx->items_cap == 0)
        return fail(ctx, LBM_EINVAL, "the fused step is for batches (lbm_init_batch, two or more instances)");
    if (mode == ctx->step_mode) return LBM_OK;
    drop_graphs(ctx);
    ctx->step_mode = mode;
    if (mode == LBM_STEP_OVERLAP) ctx->halves_dirty = true;
    if (mode == LBM_STEP_FUSED) {
        ctx->items_dirty = true;
        ctx->variant = fused_fluid_variant();
        ctx->tuned = true;
        CK(cudaMemsetAsync(ctx->counters, 0, 2 * ctx->counter_words * sizeof(unsigned), ctx->stream));
    }
    return LBM_OK;
}

lbm_status lbm_get_step_mode(const lbm_ctx* ctx, int32_t* mode) {
    if (!ctx || !mode) return LBM_EINVAL;
    *mode = ctx->step_mode;
    return LBM_OK;
}

int64_t lbm_steps_done(const lbm_ctx* ctx) { return ctx ? ctx->steps : 0; }

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->msg.c_str() : "null context"; }

void lbm_destroy(lbm_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    drop_graphs(ctx);
    if (ctx->owns_ws) cudaFree(ctx->ws);
    delete ctx;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// lbm_adjoint: the reverse sweep (see include/lbib.h)
// ---------------------------------------------------------------------------
namespace {

constexpr int ADJ_LP = 13, ADJ_LG = 5, ADJ_LS = 4;  // the accumulators' lengths (adjoint.cu)

// device memory of one adjoint run, carved from one allocation
struct AdjMem {
    char* base = nullptr;
    size_t o = 0;
    template <class T>
    T* take(size_t n) {
        T* p = reinterpret_cast<T*>(base + o);
        o = up(o + n * sizeof(T));
        return p;
    }
};

lbm_status adjoint_run(lbm_ctx* ctx, int nsteps, int K, const double* seed, double* dpart, double* dwall) {
    const int np = ctx->np, nm = ctx->nmark, ni = ctx->ninst;
    const size_t popb = (size_t)ctx->pop_elems * sizeof(float);
    const size_t partb = (size_t)np * ctx->psz, poseb = (size_t)np * ctx->pcsz;
    const int nck = (nsteps + K - 1) / K;
    // sizes first (a null base), then one allocation
    AdjMem m;
    // the cell kernels' blocks over all instances
    std::vector<int4> cblk;
    const int ab = adjoint_block_rows();
    for (int i = 0; i < ni; ++i) {
        const Geo& G = ctx->hinst[i].G;
        const int fl = ctx->icfg[i].init == LBM_INIT_COUETTE ? 1 : 0;
        for (int by = 0; by < (G.ny + ab - 1) / ab; ++by)
            for (int bx = 0; bx < (G.nx + 31) / 32; ++bx) cblk.push_back(make_int4(i, bx, by, fl));
    }
    auto plan = [&](AdjMem& mm) {
        struct Ptrs {
            char *ckf, *cks, *ckp, *segf, *segs, *segp, *finf, *fins, *finp;
            float *lam_a, *lam_b, *lam_F;
            double *lp_a, *lp_b, *lfm, *lsh, *lmg, *lwall, *mgeo;
            int* mpart;
            float* zh;
            ProbePre* ppre;
            int4* cblk;
        } q;
        q.ckf = mm.take<char>(nck * popb);
        q.cks = mm.take<char>(nck * partb);
        q.ckp = mm.take<char>(nck * poseb);
        q.segf = mm.take<char>(K * popb);
        q.segs = mm.take<char>((K + 1) * partb);
        q.segp = mm.take<char>((K + 1) * poseb);
        q.finf = mm.take<char>(popb);
        q.fins = mm.take<char>(partb);
        q.finp = mm.take<char>(poseb);
        q.lam_a = mm.take<float>(2 * ctx->pop_elems);
        q.lam_b = mm.take<float>(2 * ctx->pop_elems);
        q.lam_F = mm.take<float>(4 * ctx->flb_elems);
        q.lp_a = mm.take<double>((size_t)np * 2 * ADJ_LP);
        q.lp_b = mm.take<double>((size_t)np * 2 * ADJ_LP);
        q.lfm = mm.take<double>((size_t)np * 2 * 3);
        q.lsh = mm.take<double>((size_t)np * 2 * ADJ_LS);
        q.lmg = mm.take<double>((size_t)nm * 2 * ADJ_LG);
        q.lwall = mm.take<double>((size_t)ni * 2 * 8);
        q.mgeo = mm.take<double>((size_t)nm * 5);
        q.mpart = mm.take<int>(nm);
        q.zh = mm.take<float>((size_t)ni * 2 * 81);
        q.ppre = mm.take<ProbePre>(nm);
        q.cblk = mm.take<int4>(cblk.size());
        return q;
    };
    plan(m);
    const size_t total = m.o;
    m.o = 0;
    if (cudaMalloc(&m.base, total) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, LBM_ENOMEM, "the adjoint's checkpoints and buffers do not fit on the device");
    }
    struct Free {
        char* p;
        ~Free() { cudaFree(p); }
    } guard{m.base};
    auto q = plan(m);
    cudaStream_t st = ctx->stream;
    CK(cudaMemsetAsync(m.base, 0, total, st));
    CK(cudaMemcpyAsync(q.mgeo, ctx->hgeo.data(), ctx->hgeo.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(q.mpart, ctx->hmpart.data(), ctx->hmpart.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(q.cblk, cblk.data(), cblk.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    auto save = [&](char* f, char* sp, char* pp) -> lbm_status {
        CK(cudaMemcpyAsync(f, ctx->f[ctx->cur], popb, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(sp, state(ctx, ctx->cur), partb, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(pp, pose(ctx, ctx->cur), poseb, cudaMemcpyDeviceToDevice, st));
        return LBM_OK;
    };
    auto load = [&](const char* f, const char* sp, const char* pp) -> lbm_status {
        ctx->cur = 0;
        CK(cudaMemcpyAsync(ctx->f[0], f, popb, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(state(ctx, 0), sp, partb, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(pose(ctx, 0), pp, poseb, cudaMemcpyDeviceToDevice, st));
        return LBM_OK;
    };
    lbm_status s = LBM_OK;
    // forward, with a checkpoint every K steps
    for (int c = 0; c < nck; ++c) {
        if ((s = save(q.ckf + c * popb, q.cks + c * partb, q.ckp + c * poseb)) != LBM_OK) return s;
        if ((s = lbm_step(ctx, std::min(K, nsteps - c * K))) != LBM_OK) return s;
    }
    const int fin_cur = ctx->cur;
    const int64_t fin_steps = ctx->steps;
    if ((s = save(q.finf, q.fins, q.finp)) != LBM_OK) return s;
    // the outputs' seeds: lambda of y_c (output 0) and of the omega sum (output 1)
    std::vector<double> lp0((size_t)np * 2 * ADJ_LP, 0.0);
    for (int p = 0; p < np; ++p) {
        lp0[((size_t)p * 2 + 0) * ADJ_LP + 1] = seed[2 * p];           // LY0
        lp0[((size_t)p * 2 + 1) * ADJ_LP + ADJ_LP - 1] = seed[2 * p + 1];  // LWS
    }
    CK(cudaMemcpyAsync(q.lp_a, lp0.data(), lp0.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    // lambda(g) of level n + 1 (zero above the last level: the outputs do
    // not depend on the final populations) and of level n
    float *lam_gp = q.lam_a, *lam_g = q.lam_b;
    double *lp_new = q.lp_a, *lp_old = q.lp_b;
    AdjArgs a;
    std::memset(&a, 0, sizeof a);
    a.flb = static_cast<long long*>(ctx->flb);
    a.flags = ctx->flags;
    a.insts = ctx->insts;
    a.mgeo = q.mgeo;
    a.marker_particle = q.mpart;
    a.ptab = ctx->ptab;
    a.np = np;
    a.nmark = nm;
    a.weight = ctx->cfg.weight;
    a.pop_elems = ctx->pop_elems;
    a.flb_elems = ctx->flb_elems;
    a.lam_F = q.lam_F;
    a.lamFM = q.lfm;
    a.lam_shape = q.lsh;
    a.lam_mgeo = q.lmg;
    a.lam_wall = q.lwall;
    a.zh = q.zh;
    a.ppre = q.ppre;
    a.cblk = q.cblk;
    a.ncblk = (int)cblk.size();
    a.err = ctx->err;
    CK(launch_adjoint_setup(a, ni, st));
    // a side stream for the probe Jacobians of each reverse level
    struct Side {
        cudaStream_t s = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr;
        ~Side() {
            if (s) {
                cudaStreamSynchronize(s);
                cudaStreamDestroy(s);
            }
            if (fork) cudaEventDestroy(fork);
            if (join) cudaEventDestroy(join);
        }
    } side;
    CK(cudaStreamCreateWithFlags(&side.s, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&side.fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&side.join, cudaEventDisableTiming));
    for (int c = nck - 1; c >= 0; --c) {
        const int n0 = c * K, mseg = std::min(K, nsteps - n0);
        if ((s = load(q.ckf + c * popb, q.cks + c * partb, q.ckp + c * poseb)) != LBM_OK) return s;
        for (int j = 0; j < mseg; ++j) {  // recompute the segment, keeping every level
            if ((s = save(q.segf + j * popb, q.segs + j * partb, q.segp + j * poseb)) != LBM_OK) return s;
            if ((s = enqueue_step(ctx, st, ctx->cur, n0 + j, nullptr)) != LBM_OK) return s;
            ctx->cur ^= 1;
        }
        // the bodies of level n0 + mseg (the last step's P(n+1))
        CK(cudaMemcpyAsync(q.segs + mseg * partb, state(ctx, ctx->cur), partb, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(q.segp + mseg * poseb, pose(ctx, ctx->cur), poseb, cudaMemcpyDeviceToDevice, st));
        for (int j = mseg - 1; j >= 0; --j) {
            // level n = n0 + j: its bodies in buffer 0, its f* read where it
            // was kept (population buffer 0 points there while the step's IB
            // kernels are launched); those kernels leave f_lb(n), its flags
            // and P(n+1) in buffer 1
            ctx->cur = 0;
            CK(cudaMemcpyAsync(state(ctx, 0), q.segs + j * partb, partb, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(pose(ctx, 0), q.segp + j * poseb, poseb, cudaMemcpyDeviceToDevice, st));
            void* const f0 = ctx->f[0];
            ctx->f[0] = q.segf + j * popb;
            s = enqueue_step_part(ctx, st, 0, n0 + j, true);
            ctx->f[0] = f0;
            if (s != LBM_OK) return s;
            a.f = reinterpret_cast<const float*>(q.segf + j * popb);
            a.Pn = reinterpret_cast<const DParticle*>(state(ctx, 0));
            a.Pn1 = reinterpret_cast<const DParticle*>(state(ctx, 1));
            a.lam_gp = lam_gp;
            a.lam_g = lam_g;
            a.lamP_new = lp_new;
            a.lamP_old = lp_old;
            // the probe Jacobians on the side stream, beside the cell, marker
            // and rigid-update kernels; joined before the probes finish
            CK(cudaEventRecord(side.fork, st));
            CK(cudaStreamWaitEvent(side.s, side.fork, 0));
            CK(launch_adjoint_probes_pre(a, side.s));
            CK(cudaEventRecord(side.join, side.s));
            CK(launch_adjoint_step(a, st));
            CK(cudaStreamWaitEvent(st, side.join, 0));
            CK(launch_adjoint_probes_fin(a, st));
            std::swap(lam_gp, lam_g);
            std::swap(lp_new, lp_old);
            CK(cudaMemsetAsync(lp_old, 0, (size_t)np * 2 * ADJ_LP * sizeof(double), st));
        }
    }
    // lambda(g(0)) is lam_gp, lambda(P(0)) is lp_new: the initial field's share
    a.lam_gp = lam_gp;
    CK(launch_adjoint_init(a, st));
    std::vector<double> lp((size_t)np * 2 * ADJ_LP), lsh((size_t)np * 2 * ADJ_LS), lmg((size_t)nm * 2 * ADJ_LG),
        lw((size_t)ni * 2 * 8);
    CK(cudaMemcpyAsync(lp.data(), lp_new, lp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(lsh.data(), q.lsh, lsh.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(lmg.data(), q.lmg, lmg.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(lw.data(), q.lwall, lw.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    // back to the forward run's final state
    ctx->cur = fin_cur;
    CK(cudaMemcpyAsync(ctx->f[fin_cur], q.finf, popb, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(state(ctx, fin_cur), q.fins, partb, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(pose(ctx, fin_cur), q.finp, poseb, cudaMemcpyDeviceToDevice, st));
    CK(cudaStreamSynchronize(st));
    ctx->steps = fin_steps;
    drop_graphs(ctx);
    if ((s = device_error(ctx)) != LBM_OK) return s;
    // the particles' inputs: the pose from both stored levels, the shape
    // through its markers and mass properties (dual numbers over the two
    // dimensions), the density through the mass properties
    for (int p = 0; p < np; ++p) {
        const lbm_particle_desc& d = ctx->hdesc[p];
        const int m0 = ctx->hpart[p].x, n = ctx->hpart[p].y;
        std::vector<TD> rb(2 * n + 2), nb(2 * n + 2), S(n + 1);
        TD dim[2] = {TD(d.dim[0]), TD(d.dim[1])};
        dim[0].d[0] = 1.0;
        dim[1].d[1] = 1.0;
        ShapeOutT<TD> so;
        if (make_shape_t<TD>(d, dim, ctx->icfg[ctx->hpart[p].z].marker_spacing, rb.data(), nb.data(), S.data(), n,
                             &so) != n)
            return fail(ctx, LBM_EINTERNAL, "adjoint: the particle's markers could not be rebuilt");
        const double area = value_of(so.area), ipm = value_of(so.inertia_per_mass), rs = d.rho_s;
        const double mass = rs * area, inertia = mass * ipm;
        for (int o = 0; o < 2; ++o) {
            const double* l = lp.data() + ((size_t)p * 2 + o) * ADJ_LP;
            const double* sh = lsh.data() + ((size_t)p * 2 + o) * ADJ_LS;
            double ldim[2] = {0.0, 0.0};
            for (int k = 0; k < n; ++k) {
                const double* g = lmg.data() + ((size_t)(m0 + k) * 2 + o) * ADJ_LG;
                for (int j = 0; j < 2; ++j)
                    ldim[j] += g[0] * rb[2 * k].d[j] + g[1] * rb[2 * k + 1].d[j] + g[2] * nb[2 * k].d[j] +
                               g[3] * nb[2 * k + 1].d[j] + g[4] * S[k].d[j];
            }
            // 1/m, 1/I -> m, I -> area, inertia per mass, rho_s
            const double lI = -sh[1] / (inertia * inertia);
            const double lm = -sh[0] / (mass * mass) + lI * ipm;
            const double lipm = lI * mass;
            const double larea = sh[2] + lm * rs, lrho = sh[3] + lm * area;
            for (int j = 0; j < 2; ++j) ldim[j] += larea * so.area.d[j] + lipm * so.inertia_per_mass.d[j];
            double* out = dpart + ((size_t)p * 2 + o) * 6;
            out[0] = ldim[0];
            out[1] = ldim[1];
            out[2] = l[0] + l[6];   // xc: both stored levels
            out[3] = l[1] + l[7];   // yc
            out[4] = l[2] + l[8];   // theta
            out[5] = lrho;
        }
    }
    for (size_t k = 0; k < lw.size(); ++k) dwall[k] = lw[k];
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_adjoint(lbm_ctx* ctx, int32_t nsteps, int32_t checkpoint_every, const double* seed,
                                  double* dparticle, double* dwall) {
    if (!ctx || !seed || !dparticle || !dwall || nsteps < 1 || checkpoint_every < 1) return LBM_EINVAL;
    if (ctx->prec != LBM_FP32) return fail(ctx, LBM_EINVAL, "the adjoint runs on LBM_FP32 contexts");
    if (ctx->steps != 0) return fail(ctx, LBM_EINVAL, "the adjoint starts from a context with no steps done");
    if (ctx->np < 1) return fail(ctx, LBM_EINVAL, "the adjoint needs a particle");
    if (ctx->step_mode == LBM_STEP_FUSED) return fail(ctx, LBM_EINVAL, "the adjoint does not run the fused step");
    for (const Inst& I : ctx->hinst)
        if (!I.G.px) return fail(ctx, LBM_EINVAL, "the adjoint needs periodic x sides (no x walls)");
    for (const Inst& I : ctx->hinst)
        if (9 * I.G.plane >= (long long)INT_MAX)
            return fail(ctx, LBM_EINVAL, "the adjoint's lattices must hold fewer than 2^31 / 9 nodes each");
    return adjoint_run(ctx, nsteps, checkpoint_every, seed, dparticle, dwall);
}

// ---------------------------------------------------------------------------
// lbm_step_static: the step with the immersed-boundary scratch in a static
// device array instead of the context's workspace (see include/lbib.h).
// ---------------------------------------------------------------------------
namespace {

// Scratch shared by every lbm_step_static call in the process, on every
// device that loads this library, until the process exits.
static __device__ __align__(256) unsigned char g_ib_scratch[LBM_STATIC_SCRATCH_BYTES];

// the limits of the header hold in every precision: the per-block sums of
// the widest particle type and the widest spreading record fit
static_assert(3 * ((size_t)LBM_STATIC_MAX_MARKERS / MB + LBM_STATIC_MAX_PARTICLES + 1) * sizeof(TD) + 256 +
                      (size_t)LBM_STATIC_MAX_PARTICLES * (sizeof(unsigned) + sizeof(int4)) + 512 +
                      (size_t)LBM_STATIC_MAX_MARKERS * sizeof(Rec<TF>) <=
                  LBM_STATIC_SCRATCH_BYTES,
              "the static scratch must hold the largest context the header allows");

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of g_ib_scratch on the current device (host code only sees
// a host-side stand-in under that name).  Looked up once per device.
cudaError_t static_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_ib_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_step_static(lbm_ctx* ctx, int32_t nsteps) {
    if (!ctx || nsteps < 0) return LBM_EINVAL;
    if (ctx->np > LBM_STATIC_MAX_PARTICLES || ctx->nmark > LBM_STATIC_MAX_MARKERS)
        return fail(ctx, LBM_EINVAL,
                    "lbm_step_static: more than " + std::to_string(LBM_STATIC_MAX_PARTICLES) +
                        " particles or " + std::to_string(LBM_STATIC_MAX_MARKERS) +
                        " markers do not fit its static scratch");
    // layout of this context's scratch inside the static array
    size_t o = 0;
    const size_t o_partial = o; o = up(o + 3 * (size_t)ctx->nblk * ctx->rsz);
    const size_t o_count = o;   o = up(o + (size_t)ctx->np * sizeof(unsigned));
    const size_t o_boxes = o;   o = up(o + (size_t)ctx->np * sizeof(int4));
    const size_t o_recs = o;    o = up(o + (size_t)ctx->nmark * rec_bytes(ctx->prec));
    if (o > LBM_STATIC_SCRATCH_BYTES)
        return fail(ctx, LBM_EINVAL, "lbm_step_static: scratch needs exceed LBM_STATIC_SCRATCH_BYTES");
    void* base = nullptr;
    CK(static_scratch(&base));
    char* sb = static_cast<char*>(base);
    // the per-particle completion counters must start at zero (each step's
    // last probe block resets them, but the array keeps whatever an earlier
    // call left); the boxes are reset by the probe kernel and every other
    // entry is written before it is read
    if (ctx->np > 0) CK(cudaMemsetAsync(sb + o_count, 0, (size_t)ctx->np * sizeof(unsigned), ctx->stream));
    for (int32_t k = 0; k < nsteps; ++k) {
        if (ctx->np > 0) {
            ParticleArgs pa = particle_args(ctx, ctx->cur);
            pa.partial = sb + o_partial;
            pa.count = reinterpret_cast<unsigned*>(sb + o_count);
            pa.recs = sb + o_recs;
            pa.boxes = reinterpret_cast<int4*>(sb + o_boxes);
            CK(launch_probes(ctx->prec, pa, ctx->nblk, ctx->stream));
            CK(launch_markers(ctx->prec, pa, ctx->nblk, ctx->stream));
            if (!markers_spread(ctx->prec))
                CK(launch_spread(ctx->prec, spread_args(ctx, pa), ctx->np, spread_tiles(ctx), ctx->stream));
        }
        lbm_status s = launch_fluid_step(ctx, ctx->stream, ctx->cur, ctx->variant, ctx->np > 0,
                                         watched(ctx, ctx->steps));
        if (s != LBM_OK) return s;
        ctx->cur ^= 1;
        ctx->steps += 1;
    }
    // a context in the fused step mode: its next fused step finds its counters cleared
    if (ctx->step_mode == LBM_STEP_FUSED && nsteps > 0)
        CK(cudaMemsetAsync(ctx->counters, 0, 2 * ctx->counter_words * sizeof(unsigned), ctx->stream));
    return LBM_OK;
}
