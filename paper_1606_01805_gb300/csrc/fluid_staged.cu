// fluid_staged.cu -- persistent fused fluid kernel that stages each tile's
// streamed rows in shared memory with tensor memory-access (TMA) copies.
//
// A CTA of 8 warps owns the tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// of a lattice (or of the task list of a batch).  A tile is 32 N cells of 8
// rows; for each population plane i it needs the source rows y0 - cy(i) ..
// y0 - cy(i) + 7 over the columns x0 - 1 .. x0 + 32 N (Eq. 4 in pull form).
// Nine lanes of warp 0 each copy one plane's box of those rows (widened by
// 16 bytes on each side, so that its first column stays 16-byte aligned)
// with one cp.async.bulk.tensor copy of the lattice's tensor map into one
// of ST shared-memory stages, completing on the stage's mbarrier, ST tiles
// ahead of the tile the CTA computes; the 8 warps then compute the tile from
// shared memory (the same per-cell step as the direct kernels, fluid_tile)
// and store the results straight to global memory.  So the loads of ST - 1
// tiles are in flight without holding registers, and a CTA never waits on a
// launch.  Rows and columns outside the lattice arrive as zeros: their
// cells take the per-cell general path (walls, corners, periodic edges),
// which reads global memory.  Every wait on an mbarrier is bounded: on
// expiry the CTA sets ERR_TIMEOUT, waits (bounded again) for the copies it
// still has in flight, and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "fluid_core.cuh"

namespace lbib {

namespace {

constexpr int STH = 8;             // rows per staged tile (one warp each)
constexpr int STHREADS = 32 * STH;

template <class S, int N>
struct Staged {
    static constexpr int TW = 32 * N;                           // tile width (cells)
    static constexpr int H = 16 / (int)sizeof(S);               // halo copied on each side
    static constexpr int SW = TW + 2 * H;                       // stage row (elements) = box width
    static constexpr int BOX = STH * SW;                        // elements of one plane's box
    static constexpr int STAGE = 9 * BOX;                       // elements per stage
    static constexpr size_t STAGE_BYTES = (size_t)STAGE * sizeof(S);
    static_assert(SW * sizeof(S) % 16 == 0, "stage rows keep 16-byte alignment");
    static_assert(BOX * sizeof(S) % 128 == 0, "every plane's box starts on a 128-byte boundary");
    static_assert(SW <= 256, "a tensor copy's box is at most 256 elements wide");
};

// dynamic shared memory of a CTA: ST stages, then (batches) ST instance
// descriptors, ST tile records and ST mbarriers
template <class S, int N, int ST, bool ONE>
struct StagedSmem {
    static constexpr size_t inst = ST * Staged<S, N>::STAGE_BYTES;  // from a 128-byte aligned base
    static constexpr size_t slot = inst + (ONE ? 0 : ST * sizeof(Inst));
    static constexpr size_t bar = slot + ST * sizeof(int4);
    static constexpr size_t bytes = bar + ST * sizeof(uint64_t) + 128;  // + alignment of the base
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return done != 0;
}
// wait for the phase of parity `parity` of b; false after `limit` cycles
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, long long limit) {
    if (mbar_test(b, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(b, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
// box (x, y, z) of the 3-D tensor map tmap (generic address of a
// CUtensorMap in parameter or global memory) into shared dst (128-byte
// aligned), completing as transaction bytes on b; coordinates outside the
// tensor read zeros
__device__ __forceinline__ void tensor_copy(void* dst, const void* tmap, int x, int y, int z, uint64_t* b) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(smem_u32(b))
        : "memory");
}

// (instance, tile x, tile y) of tile t
template <bool ONE>
__device__ __forceinline__ int4 tile_of(const FluidArgs& a, int t, int ntx) {
    if (ONE) return make_int4(0, t % ntx, t / ntx, 0);
    const Task& k = a.tasks[t];
    return make_int4(k.inst, k.tx, k.ty, 0);
}

// Warp 0: copy the rows tile t needs into stage s and arm its barrier.
// tmap: the tensor map of the single lattice (ONE), else the array of the
// instances' maps (of the population buffer read).
template <class S, int N, bool ONE>
__device__ __forceinline__ void issue_tile(const FluidArgs& a, const void* tmap, int t, int ntx, S* stage,
                                           uint64_t* bar, int4* slot, Inst* sinst) {
    using Sh = Staged<S, N>;
    const int lane = threadIdx.x & 31;
    int4 tk = make_int4(0, 0, 0, 0);
    if (lane == 0) tk = tile_of<ONE>(a, t, ntx);
    tk.x = __shfl_sync(0xffffffffu, tk.x, 0);
    tk.y = __shfl_sync(0xffffffffu, tk.y, 0);
    tk.z = __shfl_sync(0xffffffffu, tk.z, 0);
    const void* map = tmap;
    if constexpr (!ONE) {  // the descriptor travels with the tile (the consumers read it from shared memory)
        static_assert(sizeof(Inst) % 16 == 0 && sizeof(Inst) <= 32 * 16, "one 16-byte piece per lane");
        const Inst* ip = a.insts + tk.x;
        if (lane < (int)(sizeof(Inst) / 16))
            reinterpret_cast<int4*>(sinst)[lane] = reinterpret_cast<const int4*>(ip)[lane];
        map = static_cast<const CUtensorMap*>(tmap) + tk.x;
    }
    if (lane == 0) *slot = tk;
    unsigned bytes = 9u * Sh::BOX * sizeof(S);  // full boxes, zero-filled where outside
    // test hook (lbm_inject_stall): the first CTA's first tile waits for 16
    // bytes that no copy brings, so that its bounded wait runs out
    if (a.stall && blockIdx.x == 0 && t == 0) bytes += 16;
    __syncwarp();  // the tile record and descriptor are written before the arrival
    if (lane == 0) mbar_arrive_expect(bar, bytes);
    __syncwarp();
    if (lane < 9)  // plane i = lane: source rows y0 - cy(i) .., columns x0 - H ..
        tensor_copy(stage + lane * Sh::BOX, map, tk.y * Sh::TW - Sh::H, tk.z * STH - cy(lane), lane, bar);
}

template <class S, class C, int N, int ST, bool ONE>
__global__ void __launch_bounds__(STHREADS, 2)
    k_fluid_staged(FluidArgs a, Inst one, const __grid_constant__ CUtensorMap tmap_one, int ntiles, int ntx,
                   long long wait_limit) {
    using Sh = Staged<S, N>;
    using L = StagedSmem<S, N, ST, ONE>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    S* stages = reinterpret_cast<S*>(smem);
    const void* tmap = ONE ? static_cast<const void*>(&tmap_one) : a.tmaps;
    Inst* sinst = reinterpret_cast<Inst*>(smem + L::inst);
    int4* slot = reinterpret_cast<int4*>(smem + L::slot);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L::bar);
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) mbar_init(bar + s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    // prologue: the first ST tiles (populations only: the kernel before this
    // one in the stream writes none of them)
    if (warp == 0)
        for (int s = 0; s < ST; ++s) {
            const int t = blockIdx.x + s * gridDim.x;
            if (t < ntiles)
                issue_tile<S, N, ONE>(a, tmap, t, ntx, stages + s * Sh::STAGE, bar + s, slot + s, sinst + s);
        }
    pdl_wait();  // forces and flags come from the kernel before this one
    pdl_trigger();
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = k % ST;
        const unsigned parity = (unsigned)(k / ST) & 1u;
        const bool ok = mbar_wait(bar + s, parity, wait_limit);
        if (__syncthreads_or(!ok)) {
            // a copy never completed: report, let the copies still in flight
            // land (bounded), and leave
            // (the copies complete within microseconds; the drain waits at
            // least a millisecond)
            if (threadIdx.x == 0) {
                atomicOr(a.err, ERR_TIMEOUT);
                const long long drain = wait_limit > 2000000 ? wait_limit : 2000000;
                for (int j = 0; j < ST; ++j) {
                    const int kk = k + j;
                    if (blockIdx.x + kk * gridDim.x < ntiles)
                        mbar_wait(bar + kk % ST, (unsigned)(kk / ST) & 1u, drain);
                }
            }
            return;
        }
        const int4 tk = slot[s];
        const int x0 = tk.y * Sh::TW, y0 = tk.z * STH;
        const int pitch = ONE ? one.G.pitch : sinst[s].G.pitch, ny = ONE ? one.G.ny : sinst[s].G.ny;
        const StageSrc<S, C, N> src{stages + s * Sh::STAGE, Sh::SW, STH, y0, x0 - Sh::H, pitch, ny};
        if constexpr (ONE) {
            const S* fin = static_cast<const S*>(a.fin) + one.f_off;
            fluid_tile<S, C, N>(src, one.G, fin, static_cast<S*>(a.fout) + one.f_off,
                                       static_cast<ForceT<C>*>(a.flb) + one.flb_off, a.flags + one.flags_off, tk.y,
                                       y0 + warp, a.check, a.err, a.keep, NoWait{});
        } else {
            const Inst& I = sinst[s];
            const S* fin = static_cast<const S*>(a.fin) + I.f_off;
            fluid_tile<S, C, N>(src, I.G, fin, static_cast<S*>(a.fout) + I.f_off,
                                       static_cast<ForceT<C>*>(a.flb) + I.flb_off, a.flags + I.flags_off, tk.y,
                                       y0 + warp, a.check, a.err, a.keep, NoWait{});
        }
        __syncthreads();  // stage s is free again
        const int tn = t + ST * gridDim.x;
        if (warp == 0 && tn < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_tile<S, N, ONE>(a, tmap, tn, ntx, stages + s * Sh::STAGE, bar + s, slot + s, sinst + s);
        }
    }
}

template <class S, class C, int N, int ST, bool ONE>
cudaError_t launch_staged_t(const FluidArgs& a, const Inst* one, int sms, cudaStream_t s, bool pdl,
                            long long wait_limit) {
    auto kern = k_fluid_staged<S, C, N, ST, ONE>;
    constexpr size_t smem = StagedSmem<S, N, ST, ONE>::bytes;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, STHREADS, smem);
    if (e != cudaSuccess) return e;
    per_sm = per_sm < 1 ? 1 : per_sm;
    using Sh = Staged<S, N>;
    int ntiles, ntx = 1;
    Inst I{};
    if (ONE) {
        I = *one;
        ntx = (I.G.nx + Sh::TW - 1) / Sh::TW;
        ntiles = ntx * ((I.G.ny + STH - 1) / STH);
    } else {
        ntiles = a.ntasks;
    }
    const int grid = ntiles < per_sm * sms ? ntiles : per_sm * sms;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(STHREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    CUtensorMap m{};
    if (ONE) m = *static_cast<const CUtensorMap*>(a.tmap_one);
    return cudaLaunchKernelEx(&cfg, kern, a, I, m, ntiles, ntx, wait_limit);
}

template <class S, class C, int N, int ST>
cudaError_t launch_staged_one_or_batch(const FluidArgs& a, const Inst* one, int sms, cudaStream_t s, bool pdl,
                                       long long wait_limit) {
    if (one) return launch_staged_t<S, C, N, ST, true>(a, one, sms, s, pdl, wait_limit);
    return launch_staged_t<S, C, N, ST, false>(a, one, sms, s, pdl, wait_limit);
}

}  // namespace

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

template <class S, int N>
cudaError_t encode_t(const void* fbuf, const Inst& I, CUtensorMapDataType dt, CUtensorMap* out) {
    using Sh = Staged<S, N>;
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)I.G.pitch, (cuuint64_t)I.G.ny, 9};
    const cuuint64_t strides[2] = {(cuuint64_t)I.G.pitch * sizeof(S), (cuuint64_t)I.G.plane * sizeof(S)};
    const cuuint32_t box[3] = {(cuuint32_t)Sh::SW, (cuuint32_t)STH, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    void* base = const_cast<S*>(static_cast<const S*>(fbuf) + I.f_off);
    const CUresult r = fn(out, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t encode_stage_map(int prec, int cpt, const void* fbuf, const Inst& I, void* out) {
    CUtensorMap* m = static_cast<CUtensorMap*>(out);
    if (prec == LBM_FP32)
        return cpt == 4 ? encode_t<float, 4>(fbuf, I, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, m)
                        : encode_t<float, 2>(fbuf, I, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, m);
    if (prec == LBM_FP16_SHIFTED)
        return cpt == 4 ? encode_t<__half, 4>(fbuf, I, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, m)
                        : encode_t<__half, 2>(fbuf, I, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, m);
    return cudaErrorInvalidValue;
}

cudaError_t launch_fluid_staged(int prec, int cpt, int stages, const FluidArgs& a, const Inst* one, int sms,
                                cudaStream_t s, bool pdl, long long wait_limit) {
    if (a.ntasks <= 0) return cudaSuccess;
    const int key = cpt * 10 + stages;
    if (prec == LBM_FP32) {
        switch (key) {
            case 42: return launch_staged_one_or_batch<float, float, 4, 2>(a, one, sms, s, pdl, wait_limit);
            case 43: return launch_staged_one_or_batch<float, float, 4, 3>(a, one, sms, s, pdl, wait_limit);
            case 23: return launch_staged_one_or_batch<float, float, 2, 3>(a, one, sms, s, pdl, wait_limit);
            case 24: return launch_staged_one_or_batch<float, float, 2, 4>(a, one, sms, s, pdl, wait_limit);
            default: break;
        }
    } else if (prec == LBM_FP16_SHIFTED) {
        switch (key) {
            case 42: return launch_staged_one_or_batch<__half, float, 4, 2>(a, one, sms, s, pdl, wait_limit);
            case 43: return launch_staged_one_or_batch<__half, float, 4, 3>(a, one, sms, s, pdl, wait_limit);
            case 23: return launch_staged_one_or_batch<__half, float, 2, 3>(a, one, sms, s, pdl, wait_limit);
            case 24: return launch_staged_one_or_batch<__half, float, 2, 4>(a, one, sms, s, pdl, wait_limit);
            default: break;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbib
