// lbrmt_batch.cuh -- persistent kernels that advance many independent
// simulations (of any grid size, solid count and tile shape) in one launch per
// step phase.  Each simulation is described by a BatchSimDesc in device memory
// (its parameters and the argument blocks of K2, K3 and K1 for both step
// parities); the kernels walk work lists of (simulation, item) pairs and run
// the same per-solid / per-tile device functions as the single-simulation
// kernels, so a batched simulation computes bit-identical fields.
#pragma once

#include "lbrmt_kernels.cuh"

namespace lbrmt {

constexpr int BATCH_MAX = 1024;  // simulations per batch

template <class R, class S>
struct BatchSimDesc {
    SimParams sp;
    RmtArgs<R, S> rmt[2];  // by step parity
    ForceArgs<R> frc[2];
    LbArgs<R, S> lb[2];
    const int *reg_count[2];  // tile registries, by step parity (classification of the overlapped step)
    unsigned char *busy[2];   // K1 region flags, by step parity
    unsigned *err;
};

// K2 over every solid of every simulation: item = (simulation, solid).
// Same launch bounds as the single-simulation kernel: the same register budget
// gives the same instruction selection, so batch members stay bit-identical to
// single runs.
template <class R, class S>
__global__ void __launch_bounds__(RMT_THREADS, sizeof(R) == 4 ? RMT_MIN_BLOCKS : 2)
    rmt_batch_kernel(const BatchSimDesc<R, S> *sims, const int2 *items, int nitems, int parity) {
    __shared__ SimParams sp;
    __shared__ RmtArgs<R, S> ra;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int2 w = items[it];
        __syncthreads();
        if (threadIdx.x == 0) {
            sp = sims[w.x].sp;
            ra = sims[w.x].rmt[parity];
        }
        __syncthreads();
        rmt_solid<R, S>(sp, ra, w.y);
    }
}

// K3 over the registered tiles of every simulation.  The work list is the
// concatenation of the simulations' active-tile lists, whose lengths K2 has
// just written; each CTA forms their prefix sums and walks the list with a
// grid stride.
template <class R, class S>
__global__ void __launch_bounds__(K3_THREADS, sizeof(R) == 4 ? 4 : 1) force_batch_kernel(const BatchSimDesc<R, S> *sims, int nsim, int parity) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ForceShared<R> fs;
    __shared__ int pre[BATCH_MAX + 1];
    __shared__ SimParams sp;
    __shared__ ForceArgs<R> fa;
    for (int k = threadIdx.x; k < nsim; k += blockDim.x) pre[k + 1] = *sims[k].frc[parity].reg_nactive;
    __syncthreads();
    if (threadIdx.x == 0) {
        pre[0] = 0;
        for (int k = 0; k < nsim; k++) pre[k + 1] += pre[k];
    }
    __syncthreads();
    const int total = pre[nsim];
    int cur = -1;
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        int lo = 0, hi = nsim;  // largest lo with pre[lo] <= it
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (pre[mid] <= it) lo = mid;
            else hi = mid;
        }
        if (lo != cur) {
            __syncthreads();
            if (threadIdx.x == 0) {
                sp = sims[lo].sp;
                fa = sims[lo].frc[parity];
            }
            __syncthreads();
            cur = lo;
        }
        force_tile<R>(sp, fa, fa.reg_active[it - pre[lo]], fs, reinterpret_cast<R *>(smem));
    }
}

// K1 over the regions of every simulation: one CTA per item (simulation,
// ry << 16 | rx) of the simulation-major list.  MODE 0: every region; 1: the
// busy regions of the overlapped step; 2: the free ones (no registry reads).
template <class R, class S, int MODE>
__global__ void __launch_bounds__(TILE_N, LB_MIN_BLOCKS<R, S> - 1) lb_batch_kernel(const BatchSimDesc<R, S> *sims,
                                                                             const int2 *items, int parity) {
    const int2 w = items[blockIdx.x];
    const BatchSimDesc<R, S> *d = sims + w.x;  // uniform, L1-resident reads
    const int rx = w.y & 0xffff, ry = w.y >> 16;
    if (MODE != 0) {
        const bool b = d->busy[parity][ry * d->sp.nrx + rx] != 0;
        if (b != (MODE == 1)) return;  // uniform over the CTA, before any barrier
    }
    lb_region<R, S, MODE != 2>(d->sp, d->lb[parity], rx, ry);
}

// Classification of every simulation's K1 regions for the overlapped batch
// step, one thread per region item, as in a single simulation's step.
template <class R, class S>
__global__ void busy_batch_kernel(const BatchSimDesc<R, S> *sims, const int2 *items, int nitems, int parity) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nitems) return;
    const int2 w = items[k];
    const BatchSimDesc<R, S> *d = sims + w.x;
    const int q = 1 - parity;
    classify_region(d->sp, (w.y >> 16) * d->sp.nrx + (w.y & 0xffff), d->reg_count[q], d->busy[q], d->busy[parity],
                    d->err);
}

}  // namespace lbrmt
