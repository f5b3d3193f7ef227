// step_fused.cu -- one persistent launch per time step for a batch of
// lattices (the screening use case): every stage of the step, for every
// instance, as items of one work list that the CTAs take in ticket order.
//
// Items (built on the host, uploaded once): probes (8 marker blocks, one
// warp each, the particle's last block doing the rigid-body update),
// markers (8 blocks), spreading tiles (32 x 8 cells), fluid tiles (4 cells
// x 32 lanes x 8 rows).  Within one instance each stage needs the one
// before it: markers wait for the particle's update, spreading tiles for all
// of the particle's marker blocks, fluid tiles for every spreading tile of
// their instance.  Instances never wait on each other, so the list runs the
// stages of instance r + 3D, r + 2D, r + D and the fluid tiles of instance
// r side by side (D instances apart): the FP64-bound particle work of some
// instances overlaps the bandwidth-bound fluid work of others, and a wait
// is rarely long.  A CTA takes the next ticket only after finishing its
// item, and every item waits only for items of smaller tickets, so the
// item of the smallest unfinished ticket can always proceed: the launch
// completes whatever the number of resident CTAs.  Every wait is bounded:
// on expiry it sets ERR_TIMEOUT and an abort word that ends every other wait
// at once (the step's results are then not usable).
//
// Counters live in two sets used by alternate steps (the population buffer
// parity); each launch clears the other set for the next step.
#include "fluid_core.cuh"
#include "ib_core.cuh"

namespace lbib {

namespace {

constexpr int FTHREADS = 256;   // 8 warps
constexpr int FUSED_TY = 8;     // spreading tile rows
constexpr int FUSED_CPT = 4;    // fluid tile: cells per thread (rows: one per warp)

// counter set: [0, np) particle updated, [np, 2 np) marker blocks done,
// [2 np, 2 np + ninst) spreading tiles done per instance, then the ticket
// and the abort word
struct Counters {
    unsigned *upd, *mdone, *sdone, *ticket, *abort;
};
__device__ __forceinline__ Counters counters(unsigned* base, int np, int ninst) {
    return Counters{base, base + np, base + 2 * np, base + 2 * np + ninst, base + 2 * np + ninst + 1};
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// CTA-wide bounded wait until *c >= target (thread 0 spins); false when the
// step was aborted or the wait ran out (which aborts it)
__device__ __forceinline__ bool wait_count(const unsigned* c, unsigned target, const FusedArgs& f,
                                           const Counters& k, int* s_ok) {
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_acquire(c) < target) {
            const long long t0 = clock64();
            while (ld_acquire(c) < target) {
                if (ld_acquire(k.abort)) {
                    ok = 0;
                    break;
                }
                if (clock64() - t0 > f.wait_limit) {
                    atomicOr(f.fa.err, ERR_TIMEOUT);
                    atomicExch(k.abort, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// A fluid item's wait for its instance's spreading tiles, per warp and
// after the warp's population loads (the hook of fluid_tile): lane 0 spins
// (bounded), the warp then reads the flags and forces.
struct SpreadWait {
    static constexpr bool LATE = true;
    const unsigned* c;
    unsigned target;
    long long limit;
    unsigned *err, *abort;
    __device__ __forceinline__ void operator()() const {
        if ((threadIdx.x & 31) == 0 && ld_acquire(c) < target) {
            const long long t0 = clock64();
            while (ld_acquire(c) < target) {
                if (ld_acquire(abort)) break;
                if (clock64() - t0 > limit) {
                    atomicOr(err, ERR_TIMEOUT);
                    atomicExch(abort, 1u);
                    break;
                }
                __nanosleep(64);
            }
        }
        __syncwarp();
    }
};

template <class S, class C, class R>
__global__ void __launch_bounds__(FTHREADS, 2) k_step_fused(FusedArgs f) {
    __shared__ SpreadSmem<C, FUSED_TY> sm;
    __shared__ int s_ticket, s_ok;
    const int warp = threadIdx.x >> 5;
    const Counters k = counters(f.counters[f.parity], f.np, f.ninst);
    if (blockIdx.x == 0) {  // clear the other set for the next step
        unsigned* o = f.counters[f.parity ^ 1];
        for (int i = threadIdx.x; i < 2 * f.np + f.ninst + 2; i += FTHREADS) o[i] = 0;
    }
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(k.ticket, 1u);
    __syncthreads();
    for (;;) {
        const int t = s_ticket;
        __syncthreads();  // every thread has read the ticket
        if (t >= f.nitems) break;
        // the next ticket is taken now and published at the item's end, so
        // that the atomic's round trip overlaps the item (a CTA then holds
        // two tickets, the later one not started: every wait still points
        // to smaller tickets than the waiter's)
        int next = 0;
        if (threadIdx.x == 0) next = (int)atomicAdd(k.ticket, 1u);
        const int4 it = f.items[t];
        switch (it.x) {
            case FI_PROBES:  // it = (kind, first block, blocks, particle)
                if (warp < it.z) probe_block<S, C, R, false, true>(f.pa, it.y + warp, k.upd);
                break;
            case FI_MARKERS:
                if (wait_count(k.upd + it.w, 1u, f, k, &s_ok) && warp < it.z)
                    marker_block<S, C, R, false, true>(f.pa, it.y + warp, k.mdone);
                break;
            case FI_SPREAD: {  // it = (kind, tile, particle, tile bound)
                const int4 pr = f.sa.ptab[it.z];
                const unsigned nblk = (unsigned)(pr.y + MB - 1) / MB;
                if (wait_count(k.mdone + it.z, nblk, f, k, &s_ok)) {
                    spread_tile<C, R, false, true, FUSED_TY>(f.sa, it.y, it.z, it.w, sm);
                    __syncthreads();
                    if (threadIdx.x == 0) {  // the tile's forces and flags visible first
                        __threadfence();
                        atomicAdd(k.sdone + pr.z, 1u);
                    }
                }
                break;
            }
            default: {  // FI_FLUID: it = (kind, task, instance, spreading tiles of the instance)
                unsigned target = (unsigned)it.w;
                if (f.stall && t == f.stall_ticket) target += 1;  // lbm_inject_stall: never reached
                const Task task = f.fa.tasks[it.y];
                const Inst& I = f.fa.insts[task.inst];
                const S* fin = static_cast<const S*>(f.fa.fin) + task.f_off;
                const GlobalSrc<S, C, FUSED_CPT> src{fin, (long long)task.pitch * task.ny, task.pitch, task.ny};
                const SpreadWait w{k.sdone + it.z, target, f.wait_limit, f.fa.err, k.abort};
                fluid_tile<S, C, FUSED_CPT>(src, I.G, fin, static_cast<S*>(f.fa.fout) + task.f_off,
                                            static_cast<ForceT<C>*>(f.fa.flb) + I.flb_off, f.fa.flags + I.flags_off,
                                            task.tx, task.ty * FUSED_TY + warp, f.fa.check, f.fa.err, 0, w);
                break;
            }
        }
        if (threadIdx.x == 0) s_ticket = next;
        __syncthreads();  // the next ticket is published; s_ok and the spreading list are free again
    }
}

template <class S, class C, class R>
cudaError_t launch_t(const FusedArgs& f, int sms, cudaStream_t s) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_fused<S, C, R>, FTHREADS, 0);
    if (e != cudaSuccess) return e;
    per_sm = per_sm < 1 ? 1 : per_sm;
    const int grid = f.nitems < per_sm * sms ? f.nitems : per_sm * sms;
    k_step_fused<S, C, R><<<grid > 0 ? grid : 1, FTHREADS, 0, s>>>(f);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_fused(int prec, const FusedArgs& f, int sms, cudaStream_t s) {
    if (prec == LBM_FP32) return launch_t<float, float, double>(f, sms, s);
    if (prec == LBM_FP16_SHIFTED) return launch_t<__half, float, double>(f, sms, s);
    if (prec == LBM_FP64) return launch_t<double, double, double>(f, sms, s);
    return cudaErrorInvalidValue;
}

int fused_spread_rows() { return FUSED_TY; }
int fused_fluid_variant() { return 0; }  // the 4 x 8 task list

}  // namespace lbib
