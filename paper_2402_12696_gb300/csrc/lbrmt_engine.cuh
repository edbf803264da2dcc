// lbrmt_engine.cuh -- launch sequences of the LBRMT kernels for one precision.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>

#include "lbrmt_batch.cuh"
#include "lbrmt_kernels.cuh"

namespace lbrmt {

struct LaunchInfo {
    int tmax;            // largest solid tile side
    int force_blocks;    // persistent grid of K3
    int force_blocks_ov; // the same in the overlapped step (fewer CTAs per SM)
    int rmt_smem;        // dynamic shared memory of K2
    int rmt_carve;       // K2's preferred shared-memory carveout (percent), or -1
    int force_carve_ov;  // the overlapped K3's preferred carveout (percent), or -1
    int force_smem;      // dynamic shared memory of K3
    int rmt_req = 0;      // requested K2 CTA width (0: chosen by configure)
    int rmt_threads = 256; // K2 CTA width in use: 256, or 1024 (FP32 arithmetic only)
    bool tma = false;    // tensor maps of the populations and density plane are valid
    bool use_tma = true; // K1 with TMA staging (else the direct-load kernel)
    int lb_blocks = 0, lb_smem = 0;
    CUtensorMap tm_f[2], tm_c;
    // Overlapped step: K1 of the regions without solid forcing runs on a side
    // stream of the lowest priority, concurrently with K2, K3 and K1 of the other
    // regions, which are launched with the highest priority.  The stream and the
    // fork / join events are owned by the simulation.
    bool split = true;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, flags = nullptr;
    cudaEvent_t done[2] = {nullptr, nullptr};  // free-region K1 of the step of each parity has finished
    int prio_hi = 0;
};

// Does a step run the overlapped schedule (K1 split into busy and free regions)?
inline bool step_overlaps(const SimParams &sp, const LaunchInfo &li) {
    return li.split && li.side && sp.nsolids > 0 && !(li.tma && li.use_tma);
}

// Kernel launches of one step (timed: the sequential schedule of lbrmt_step_timed).
inline int step_launches(const SimParams &sp, const LaunchInfo &li, bool timed = false) {
    if (sp.nsolids == 0) return 1;
    return step_overlaps(sp, li) && !timed ? 5 : 3;  // K2, classification, K3, K1 (busy and free regions)
}

// Steps of a chain: within one, the free-region K1 of a step runs beside the
// solid kernels of the next; the chain's last step joins it.
enum { CHAIN_FIRST = 1, CHAIN_LAST = 2, CHAIN_ONE = 3 };

// Launch with a scheduling priority (a launch attribute, kept by stream capture).
template <class... P, class... A>
inline cudaError_t launch_prio(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, int prio,
                               A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = prio;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// The same with a preferred shared-memory carveout (percent of the SM's
// largest; the driver rounds it up to a carveout it supports), or none (-1).
template <class... P, class... A>
inline cudaError_t launch_carve(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, int prio,
                                int carve, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = prio;
    at[1].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    at[1].val.sharedMemCarveout = carve < 0 ? 0u : (unsigned)carve;
    cfg.attrs = at;
    cfg.numAttrs = carve < 0 ? 1 : 2;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// Shared-memory carveout steps of this GPU family (KB): the SM's 256 KB of
// L1/shared storage not carved out for shared memory is L1 cache.
constexpr int CARVE_STEPS_KB[] = {8, 16, 32, 64, 100, 132, 164, 196, 228};
// The smallest step that holds need bytes (-1: none up to per_sm).
inline int carve_step(int need, int per_sm) {
    for (int kb : CARVE_STEPS_KB)
        if (kb * 1024 >= need) return kb * 1024 <= per_sm ? kb * 1024 : -1;
    return -1;
}
// A step as a launch's carveout preference: percent of the largest carveout,
// rounded down, so that the driver, which rounds up to its steps, lands on it.
inline int carve_percent(int step, int per_sm) { return step > 0 ? (int)(100.0 * step / per_sm) : -1; }
// The SM's largest carveout and the shared memory reserved per CTA.
inline void smem_limits(int *per_sm, int *resv) {
    int dev = 0;
    *per_sm = *resv = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
inline EncodeTiledFn encode_tiled_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}
template <class S> inline CUtensorMapDataType tma_dtype();
template <> inline CUtensorMapDataType tma_dtype<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> inline CUtensorMapDataType tma_dtype<double>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT64; }
template <> inline CUtensorMapDataType tma_dtype<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }
template <> inline CUtensorMapDataType tma_dtype<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }

// Launch shape of the batched kernels.
struct BatchLaunch {
    int rmt_blocks, rmt_smem;      // K2: persistent grid, dynamic shared memory (largest solid tile)
    int rmt_carve;                 // K2's preferred shared-memory carveout (percent), or -1
    int force_blocks, force_smem;  // K3 (widest tile shape)
    // Overlapped batch step, as a single simulation's: the classification and
    // K1 of every member's solid-free regions on a side stream of the lowest
    // priority, K2, K3 and K1 of the busy regions at the highest.  The stream
    // and the fork / join events are owned by the batch.
    bool split = false;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, flags = nullptr;
    int prio_hi = 0;
};

// Does a batch step overlap (and how many kernels does it launch)?
inline bool batch_overlaps(const BatchLaunch &bl, int n_rmt) { return bl.split && bl.side && n_rmt > 0; }
inline int batch_launches(const BatchLaunch &bl, int n_rmt, bool timed = false) {
    if (n_rmt == 0) return 1;
    return batch_overlaps(bl, n_rmt) && !timed ? 5 : 4;  // classification, K2, K3, K1 (busy and free regions)
}

struct EngineOps {
    cudaError_t (*configure)(const SimParams &, const DevState &, int tmax, LaunchInfo *);
    cudaError_t (*init)(const SimParams &, const DevState &, const LaunchInfo &, cudaStream_t);
    // tape (optional): per-node rho, ux, uy, Fx, Fy of the step (5 planes of reals)
    cudaError_t (*step)(const SimParams &, const DevState &, const LaunchInfo &, int parity, cudaStream_t,
                        cudaEvent_t *ev, void *tape, int chain);
    cudaError_t (*field)(const SimParams &, const DevState &, int cur, int lastreg, int kind, int solid,
                         double *out, cudaStream_t);
    cudaError_t (*stats)(const SimParams &, const DevState &, int cur, double *out, cudaStream_t);
    // per-tile FP64 sums of rho - rho_f of the current populations into d.mass_partials (ntx nty values)
    cudaError_t (*mass)(const SimParams &, const DevState &, int cur, cudaStream_t);
    cudaError_t (*set_pop)(const SimParams &, const DevState &, int cur, const double *src, cudaStream_t);
    // batches: descriptor of one simulation (host image of BatchSimDesc<R, S>)
    size_t desc_size;
    void (*fill_desc)(void *dst, const SimParams &, const DevState &);
    cudaError_t (*batch_configure)(int tmax, int force_smem_elems, int nitems_rmt, BatchLaunch *);
    // ev (optional): events before K2, before K3, before K1 and after K1
    cudaError_t (*batch_step)(const void *descs, int nsim, const int2 *rmt_items, int n_rmt, const int2 *lb_items,
                              int n_lb, const BatchLaunch &, int parity, cudaStream_t, cudaEvent_t *ev);
    int real_size, store_size;
    int launches_per_step;
};

extern const EngineOps engine_fp32;
extern const EngineOps engine_fp64;
extern const EngineOps engine_fp16;
extern const EngineOps engine_bf16;

template <class R, class S>
__global__ void set_pop_kernel(SimParams sp, const double *src, S *f, S *carry, const int *reg, R *pool,
                               unsigned *err) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= sp.P) return;
    const int i = (int)(c % sp.nx), j = (int)(c / sp.nx);
    const double base = rest_base_d<R>(sp, reg, pool, i, j);
    bool ov = false;
    for (int q = 0; q < 9; q++) {
        const R v = R(src[q * sp.P + c] - (double)wq<double>(q) * sp.rho_f - (q == 0 ? base : 0.0));
        ov = ov || store_overflow<S, R>(v, sp, q);
        stS<S, R>(f + q * sp.P + c, v, sp, q);
    }
    if (ov) atomicOr(err, ERR_OVERFLOW16);
    // no previous collision: a zero half-force term in the next step's moments
    stC<S, R>(carry + c, R(NAN), sp);
    const int tile = (j >> sp.ly) * sp.ntx + (i >> sp.lx);
    if (reg[tile] > 0) {
        R *po = pool + (long long)tile * POOL_STRIDE + (((j & (sp.ty - 1)) << sp.lx) + (i & (sp.tx - 1)));
        po[POOL_CX] = R(0);
        po[POOL_CY] = R(0);
    }
}

template <class R, class S>
struct Engine {
    // Tensor maps over the population buffers (nx x ny x 9) and the density
    // plane (nx x ny x 1) with one registry tile per box; needs rows of 16-byte multiples.
    static void configure_tma(const SimParams &sp, const DevState &d, LaunchInfo *li, int nsm) {
        li->tma = false;
        EncodeTiledFn enc = encode_tiled_fn();
        const size_t ss = sizeof(S);
        if (!enc || ((size_t)sp.nx * ss) % 16 != 0) return;
        const cuuint64_t dimf[3] = {(cuuint64_t)sp.nx, (cuuint64_t)sp.ny, 9};
        const cuuint64_t dimc[3] = {(cuuint64_t)sp.nx, (cuuint64_t)sp.ny, 1};
        const cuuint64_t str[2] = {(cuuint64_t)sp.nx * ss, (cuuint64_t)sp.P * ss};
        const cuuint32_t boxf[3] = {(cuuint32_t)sp.tx, (cuuint32_t)sp.ty, 9}, boxc[3] = {(cuuint32_t)sp.tx, (cuuint32_t)sp.ty, 1};
        const cuuint32_t es[3] = {1, 1, 1};
        bool ok = true;
        for (int k = 0; k < 2 && ok; k++)
            ok = enc(&li->tm_f[k], tma_dtype<S>(), 3, d.f[k], dimf, str, boxf, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
                 CUDA_SUCCESS;
        ok = ok && enc(&li->tm_c, tma_dtype<S>(), 3, d.carry, dimc, str, boxc, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        if (!ok) return;
        li->lb_smem = 2 * 10 * TILE_N * (int)ss + 128;  // + alignment of the stages
        if (cudaFuncSetAttribute(lb_tma_kernel<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, li->lb_smem) !=
            cudaSuccess)
            return;
        int per = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, lb_tma_kernel<R, S>, TILE_N, li->lb_smem) != cudaSuccess ||
            per < 1)
            return;
        li->lb_blocks = nsm * per;
        li->tma = true;
    }

    // K2's dynamic shared memory and carveout.  A CTA holds the byte labels of
    // its tile (tmax^2, padded) and the node lists; min_blocks CTAs on an SM
    // take min_blocks x (dynamic + static + reserved) of its carveout, and the
    // rest is L1 cache, which K2's gathers and stencils lean on.  When a lower
    // carveout step than the one that lists of 8 LIST_CAP bytes need holds
    // min_blocks CTAs with at least RMT_LIST_MIN_BYTES of lists, the lists take
    // all of the CTA's share of that step and each launch asks for it.
    // Otherwise: lists of 8 LIST_CAP bytes and the driver's choice (-1).
    template <class K>
    static void rmt_smem_carveout(K kernel, int tmax, int min_blocks, int *smem, int *carve) {
        const int labs = (tmax * tmax + 15) & ~15;
        *smem = labs + 8 * LIST_CAP;
        *carve = -1;
        int per_sm, resv;
        smem_limits(&per_sm, &resv);
        cudaFuncAttributes fa;
        if (per_sm <= 0 || cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        const int fixed = (int)fa.sharedSizeBytes + resv;
        const int need_base = min_blocks * (*smem + fixed);
        for (int kb : CARVE_STEPS_KB) {
            const int c = kb * 1024;
            if (c > per_sm || c >= need_base) break;
            const int dyn = std::min((c / min_blocks - fixed) & ~15, RMT_SMEM_MAX);
            if (dyn - labs < RMT_LIST_MIN_BYTES) continue;
            int per = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, RMT_THREADS, dyn) != cudaSuccess ||
                per < min_blocks) {
                cudaGetLastError();
                return;
            }
            *smem = dyn;
            *carve = carve_percent(c, per_sm);
            return;
        }
    }

    static cudaError_t configure(const SimParams &sp, const DevState &d, int tmax, LaunchInfo *li) {
        li->tmax = tmax;
        li->rmt_smem = ((tmax * tmax + 15) & ~15) + 8 * LIST_CAP;
        {
            cudaError_t e0 = upload_rinv_tables();
            if (e0 != cudaSuccess) return e0;
        }
        li->force_smem = force_smem_elems(sp.tx, sp.ty) * (int)sizeof(R);
        // the attribute is per kernel, shared by every simulation: set the largest any may need
        cudaError_t e = cudaFuncSetAttribute(rmt_solid_kernel<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             RMT_SMEM_MAX);
        if (e != cudaSuccess) return e;
        rmt_smem_carveout(rmt_solid_kernel<R, S>, tmax, sizeof(R) == 4 ? RMT_MIN_BLOCKS : 2, &li->rmt_smem,
                          &li->rmt_carve);
        int nsm0 = 0, dev0 = 0;
        cudaGetDevice(&dev0);
        cudaDeviceGetAttribute(&nsm0, cudaDevAttrMultiProcessorCount, dev0);
        // K2's CTA width: the request, else 1024 threads when the solids number at
        // most half the SMs (FP32 arithmetic: 64 registers hold it), else 256
        int w = li->rmt_req;
        if (w == 0) w = sizeof(R) == 4 && sp.nsolids > 0 && 2 * sp.nsolids <= nsm0 ? RMT_THREADS_BIG : RMT_THREADS;
        if (w == RMT_THREADS_BIG && sizeof(R) != 4) w = RMT_THREADS;
        li->rmt_threads = w;
        if (w == RMT_THREADS_BIG) {
            e = cudaFuncSetAttribute(rmt_solid_kernel_big<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, RMT_SMEM_MAX);
            // One CTA per solid and at most one per SM: room for node lists of a
            // tile's size, so that a large solid's advected nodes and layers are
            // listed instead of walked (its box) or scanned (its tile, per layer).
            li->rmt_smem = std::max(li->rmt_smem, std::min(((tmax * tmax + 15) & ~15) + 4 * tmax * tmax, RMT_SMEM_MAX));
            li->rmt_carve = -1;
        }
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(force_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 force_smem_max() * (int)sizeof(R));
        if (e != cudaSuccess) return e;
        int dev = 0, nsm = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, force_kernel<R>, K3_THREADS, li->force_smem);
        if (e != cudaSuccess) return e;
        li->force_blocks = nsm * (per > 0 ? per : 1);
        // In the overlapped step K3 runs beside the free regions' K1: three of its
        // CTAs per SM (of four that fit) leave the registers of two K1 CTAs, and
        // the step is shorter although K3 alone takes longer.
        li->force_blocks_ov = nsm * std::min(std::max(per, 1), 3);
        // With fewer CTAs per SM than fit, the overlapped K3 asks for the
        // carveout step that holds those only: more L1 beside them.
        li->force_carve_ov = -1;
        if (per > 3) {
            int per_sm, resv;
            smem_limits(&per_sm, &resv);
            cudaFuncAttributes fa;
            if (per_sm > 0 && cudaFuncGetAttributes(&fa, force_kernel<R>) == cudaSuccess)
                li->force_carve_ov =
                    carve_percent(carve_step(3 * (li->force_smem + (int)fa.sharedSizeBytes + resv), per_sm), per_sm);
            else
                cudaGetLastError();
        }
        configure_tma(sp, d, li, nsm);
        return cudaSuccess;
    }

    static RmtArgs<R, S> rmt_args(const DevState &d, int parity, int init) {
        RmtArgs<R, S> a;
        const int p = parity, q = 1 - parity;
        a.f = (const S *)d.f[p];
        a.carry = (const S *)d.carry;
        a.fbody = (const R *)d.fbody;
        a.bfield = (const R *)d.bfield;
        a.reg_prev = d.reg_count[q];
        a.pool_prev = (const R *)d.pool[q];
        a.xi_in = (const R *)d.xi[p];
        a.frame_in = d.frame[p];
        if (init) {
            a.xi_out = (R *)d.xi[0];
            a.frame_out = d.frame[0];
            a.frame_next = d.frame[1];
            a.stats = nullptr;
        } else {
            a.xi_out = (R *)d.xi[q];
            a.frame_out = d.frame[q];
            a.frame_next = d.frame[p];
            a.stats = d.stats_step;
        }
        const int r = init ? 1 : p;  // the initial registry takes slot 1 (step 0 reads it as "previous")
        a.reg_count = d.reg_count[r];
        a.reg_solids = d.reg_solids[r];
        a.reg_active = d.reg_active[r];
        a.reg_nactive = d.reg_nactive[r];
        a.solids = d.solids;
        a.order = d.order;
        a.err = d.err;
        a.init = init;
        return a;
    }

    static ForceArgs<R> force_args(const DevState &d, int xi_idx, int r) {
        ForceArgs<R> a;
        a.xi = (const R *)d.xi[xi_idx];
        a.frame = d.frame[xi_idx];
        a.reg_count = d.reg_count[r];
        a.reg_solids = d.reg_solids[r];
        a.reg_active = d.reg_active[r];
        a.reg_nactive = d.reg_nactive[r];
        a.pool = (R *)d.pool[r];
        a.solids = d.solids;
        a.lamtab = d.lamtab;
        a.err = d.err;
        return a;
    }

    static LbArgs<R, S> lb_args(const SimParams &sp, const DevState &d, int parity) {
        const int p = parity, q = 1 - parity;
        LbArgs<R, S> a;
        a.f_in = (const S *)d.f[p];
        a.f_out = (S *)d.f[q];
        for (int k = 0; k < 9; k++) {
            a.fin_q[k] = a.f_in + (long long)k * sp.P;
            // the push target of an interior node: the offset is positive for k >= 1 (P > nx + 1)
            a.fout_push[k] = a.f_out + (long long)k * sp.P + (long long)cyq(k) * sp.nx + cxq(k);
        }
        a.carry = (S *)d.carry;
        a.fbody = (const R *)d.fbody;
        a.bfield = (const R *)d.bfield;
        a.tape = nullptr;
        a.reg_count = d.reg_count[p];
        a.pool = (R *)d.pool[p];
        a.clr_count = d.reg_count[q];
        a.clr_nactive = d.reg_nactive[q];
        a.pool_prev = (const R *)d.pool[q];
        a.err = d.err;
        return a;
    }

    static void fill_desc(void *dst, const SimParams &sp, const DevState &d) {
        BatchSimDesc<R, S> b;
        std::memset(&b, 0, sizeof(b));
        b.sp = sp;
        for (int p = 0; p < 2; p++) {
            b.rmt[p] = rmt_args(d, p, 0);
            b.frc[p] = force_args(d, 1 - p, p);
            b.lb[p] = lb_args(sp, d, p);
            b.reg_count[p] = d.reg_count[p];
            b.busy[p] = d.busy[p];
        }
        b.err = d.err;
        std::memcpy(dst, &b, sizeof(b));
    }

    static cudaError_t batch_configure(int tmax, int fs_elems, int nitems_rmt, BatchLaunch *bl) {
        int dev = 0, nsm = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        bl->rmt_smem = ((tmax * tmax + 15) & ~15) + 8 * LIST_CAP;
        bl->force_smem = fs_elems * (int)sizeof(R);
        cudaError_t e = cudaFuncSetAttribute(rmt_batch_kernel<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             RMT_SMEM_MAX);
        if (e != cudaSuccess) return e;
        rmt_smem_carveout(rmt_batch_kernel<R, S>, tmax, sizeof(R) == 4 ? RMT_MIN_BLOCKS : 2, &bl->rmt_smem,
                          &bl->rmt_carve);
        e = cudaFuncSetAttribute(force_batch_kernel<R, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 force_smem_max() * (int)sizeof(R));
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, rmt_batch_kernel<R, S>, RMT_THREADS, bl->rmt_smem);
        if (e != cudaSuccess) return e;
        bl->rmt_blocks = std::max(1, std::min(nitems_rmt, nsm * std::max(per, 1)));
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, force_batch_kernel<R, S>, K3_THREADS, bl->force_smem);
        if (e != cudaSuccess) return e;
        bl->force_blocks = nsm * std::max(per, 1);
        return cudaSuccess;
    }

    static cudaError_t batch_step(const void *descs, int nsim, const int2 *rmt_items, int n_rmt, const int2 *lb_items,
                                  int n_lb, const BatchLaunch &bl, int parity, cudaStream_t st, cudaEvent_t *ev) {
        const BatchSimDesc<R, S> *ds = static_cast<const BatchSimDesc<R, S> *>(descs);
        const bool overlap = batch_overlaps(bl, n_rmt) && !ev;
        const int prio = overlap ? bl.prio_hi : 0;
        if (overlap) {  // fork: classification and K1 of the free regions on the side stream
            cudaEventRecord(bl.fork, st);
            cudaStreamWaitEvent(bl.side, bl.fork, 0);
            busy_batch_kernel<R, S><<<(n_lb + 255) / 256, 256, 0, bl.side>>>(ds, lb_items, n_lb, parity);
            cudaEventRecord(bl.flags, bl.side);
            lb_batch_kernel<R, S, 2><<<n_lb, TILE_N, 0, bl.side>>>(ds, lb_items, parity);
            cudaEventRecord(bl.join, bl.side);
        } else if (n_rmt > 0) {
            busy_batch_kernel<R, S><<<(n_lb + 255) / 256, 256, 0, st>>>(ds, lb_items, n_lb, parity);
        }
        if (ev) cudaEventRecord(ev[0], st);
        if (n_rmt > 0)
            launch_carve(rmt_batch_kernel<R, S>, dim3(bl.rmt_blocks), dim3(RMT_THREADS), bl.rmt_smem, st, prio,
                         bl.rmt_carve, ds, rmt_items, n_rmt, parity);
        if (ev) cudaEventRecord(ev[1], st);
        if (n_rmt > 0)
            launch_prio(force_batch_kernel<R, S>, dim3(bl.force_blocks), dim3(K3_THREADS), bl.force_smem, st, prio, ds,
                        nsim, parity);
        if (ev) cudaEventRecord(ev[2], st);
        if (n_lb > 0) {
            if (overlap) {
                cudaStreamWaitEvent(st, bl.flags, 0);  // the classification is done
                launch_prio(lb_batch_kernel<R, S, 1>, dim3(n_lb), dim3(TILE_N), 0, st, prio, ds, lb_items, parity);
            } else
                lb_batch_kernel<R, S, 0><<<n_lb, TILE_N, 0, st>>>(ds, lb_items, parity);
        }
        if (ev) cudaEventRecord(ev[3], st);
        if (overlap) cudaStreamWaitEvent(st, bl.join, 0);  // join
        return cudaGetLastError();
    }

    static void launch_rmt(const SimParams &sp, const LaunchInfo &li, const RmtArgs<R, S> &a, cudaStream_t st,
                           int prio = 0) {
        if (li.rmt_threads == RMT_THREADS_BIG)
            launch_prio(rmt_solid_kernel_big<R, S>, dim3(sp.nsolids), dim3(RMT_THREADS_BIG), li.rmt_smem, st, prio, sp, a);
        else
            launch_carve(rmt_solid_kernel<R, S>, dim3(sp.nsolids), dim3(RMT_THREADS), li.rmt_smem, st, prio, li.rmt_carve,
                         sp, a);
    }

    static cudaError_t init(const SimParams &sp, const DevState &d, const LaunchInfo &li, cudaStream_t st) {
        if (sp.nsolids > 0) {
            launch_rmt(sp, li, rmt_args(d, 0, 1), st);
            force_kernel<R><<<li.force_blocks, K3_THREADS, li.force_smem, st>>>(sp, force_args(d, 0, 1));
        }
        dim3 grid(sp.ntx, sp.nty), blk(TILE_N);
        init_f_kernel<R, S><<<grid, blk, 0, st>>>(sp, (S *)d.f[0], (S *)d.carry);
        return cudaGetLastError();
    }

    // ev (optional): four events recorded before K2, before K3, before K1 and after
    // K1; the step then takes the sequential schedule (one K1 over every region,
    // on st after K3), so each kernel is timed alone.
    // Overlapped schedule of step n (chain: CHAIN_FIRST / CHAIN_LAST bits):
    //   st:   K2(n), classification(n), K3(n), [wait free K1(n-1)], K1 busy(n)
    //   side: [wait classification(n)] K1 free(n)
    // The free K1 of step n reads f^n and writes f^{n+1} outside the solids'
    // reach, so it runs beside K3(n), the busy K1(n) and the solid kernels of step
    // n + 1; the busy K1 of step n + 1 waits for it (pushes cross into busy
    // regions, and it overwrites f^n).  The first step of a chain has no free K1
    // before it in flight; the last joins its own.
    static cudaError_t step(const SimParams &sp, const DevState &d, const LaunchInfo &li, int parity,
                            cudaStream_t st, cudaEvent_t *ev, void *tape, int chain) {
        const int p = parity, q = 1 - parity;
        const bool overlap = step_overlaps(sp, li) && !ev;
        const int prio = overlap ? li.prio_hi : 0;
        const dim3 grid(sp.nrx, sp.nty), blk(TILE_N);
        LbArgs<R, S> la = lb_args(sp, d, p);
        la.tape = static_cast<R *>(tape);
        const int nreg = sp.nrx * sp.nty;
        if (ev) cudaEventRecord(ev[0], st);
        if (sp.nsolids > 0) launch_rmt(sp, li, rmt_args(d, p, 0), st, prio);
        if (overlap) {  // exact classification, then the free regions' K1 on the side stream
            lb_classify_kernel<<<(nreg + 255) / 256, 256, 0, st>>>(sp, d.reg_count[p], d.reg_count[q], d.busy[p],
                                                                   d.reg_nactive[q]);
            cudaEventRecord(li.flags, st);
            cudaStreamWaitEvent(li.side, li.flags, 0);
            lb_step_kernel<R, S, 2><<<grid, blk, 0, li.side>>>(sp, la, d.busy[p]);
            cudaEventRecord(li.done[p], li.side);
        }
        if (ev) cudaEventRecord(ev[1], st);
        if (sp.nsolids > 0)
            launch_carve(force_kernel<R>, dim3(overlap ? li.force_blocks_ov : li.force_blocks), dim3(K3_THREADS),
                         li.force_smem, st, prio, overlap ? li.force_carve_ov : -1, sp, force_args(d, q, p));
        if (ev) cudaEventRecord(ev[2], st);
        if (li.tma && li.use_tma)
            lb_tma_kernel<R, S><<<li.lb_blocks, TILE_N, li.lb_smem, st>>>(sp, la, li.tm_f[p], li.tm_c, sp.ntx * sp.nty);
        else if (overlap) {
            if (!(chain & CHAIN_FIRST)) cudaStreamWaitEvent(st, li.done[q], 0);  // free K1 of step n - 1
            launch_prio(lb_step_kernel<R, S, 1>, grid, blk, 0, st, prio, sp, la, (const unsigned char *)d.busy[p]);
        } else
            lb_step_kernel<R, S, 0><<<grid, blk, 0, st>>>(sp, la, nullptr);
        if (ev) cudaEventRecord(ev[3], st);
        if (overlap && (chain & CHAIN_LAST)) cudaStreamWaitEvent(st, li.done[p], 0);  // join
        return cudaGetLastError();
    }

    static cudaError_t field(const SimParams &sp, const DevState &d, int cur, int lastreg, int kind, int solid,
                             double *out, cudaStream_t st) {
        dim3 grid(sp.ntx, sp.nty), blk(TILE_N);
        if (kind >= 10 && kind <= 15 && kind != 13) {
            solid_field_kernel<R><<<64, 256, 0, st>>>(sp, (const R *)d.xi[cur], d.frame[cur], d.solids, solid,
                                                      kind - 10, out);
            return cudaGetLastError();
        }
        const int r = lastreg;
        field_kernel<R, S><<<grid, blk, 0, st>>>(sp, (const S *)d.f[cur], (const S *)d.carry, (const R *)d.fbody,
                                                 (const R *)d.bfield,
                                                 d.reg_count[r], (const R *)d.pool[r], kind, out);
        return cudaGetLastError();
    }

    static cudaError_t stats(const SimParams &sp, const DevState &d, int cur, double *out, cudaStream_t st) {
        if (sp.nsolids == 0) return cudaSuccess;
        solid_stats_kernel<R, S><<<sp.nsolids, STATS_THREADS, 0, st>>>(sp, (const S *)d.f[cur], (const S *)d.carry,
                                                             (const R *)d.fbody, (const R *)d.bfield,
                                                             d.reg_count[1 - cur], d.reg_solids[1 - cur],
                                                             (const R *)d.pool[1 - cur], (const R *)d.xi[cur],
                                                             d.frame[cur], d.solids, d.order, out);
        return cudaGetLastError();
    }

    static cudaError_t mass(const SimParams &sp, const DevState &d, int cur, cudaStream_t st) {
        mass_tile_kernel<R, S><<<dim3(sp.ntx, sp.nty), TILE_N, 0, st>>>(sp, (const S *)d.f[cur], d.reg_count[1 - cur],
                                                                     (const R *)d.pool[1 - cur], d.mass_partials);
        return cudaGetLastError();
    }

    static cudaError_t set_pop(const SimParams &sp, const DevState &d, int cur, const double *src, cudaStream_t st) {
        const int nb = (int)((sp.P + 255) / 256);
        set_pop_kernel<R, S><<<nb, 256, 0, st>>>(sp, src, (S *)d.f[cur], (S *)d.carry, d.reg_count[1 - cur],
                                                 (R *)d.pool[1 - cur], d.err);
        return cudaGetLastError();
    }

    static EngineOps ops() {
        EngineOps o;
        o.configure = &configure;
        o.init = &init;
        o.step = &step;
        o.field = &field;
        o.stats = &stats;
        o.mass = &mass;
        o.set_pop = &set_pop;
        o.desc_size = sizeof(BatchSimDesc<R, S>);
        o.fill_desc = &fill_desc;
        o.batch_configure = &batch_configure;
        o.batch_step = &batch_step;
        o.real_size = sizeof(R);
        o.store_size = sizeof(S);
        o.launches_per_step = 3;
        return o;
    }
};

}  // namespace lbrmt
