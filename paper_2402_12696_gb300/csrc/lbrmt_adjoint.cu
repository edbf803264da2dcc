// lbrmt_adjoint.cu -- checkpointed forward run and adjoint (reverse) sweep.
//
// lbrmt_forward_checkpointed returns the simulation to its initial state, runs
// T steps and keeps a copy of the whole device state every K steps (and of
// the final state).  lbrmt_backward then walks the checkpoints backwards: for
// each segment it restores the checkpoint and recomputes the segment's steps,
// recording per step the moments and force density (a tape written by the LB
// kernel), the new reference-map tiles and frames, and the registry; it then
// applies the reverse kernels step by step, from the last to the first.  The
// adjoint variables carried between steps are those of the populations, of
// the stored half-force and of the reference map; the gradients with respect
// to each solid's G and rho_s / rho_f and to the body force field are
// accumulated on the way.  The initial populations depend on rho_s through
// Delta rho^0 (f_0 = w_0 rho_f + Delta rho^0), the last term of the sweep.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "lbrmt.h"
#include "lbrmt_adjoint.cuh"
#include "lbrmt_engine.cuh"
#include "lbrmt_sim.cuh"

using namespace lbrmt;

struct AdjointStore {
    int T = 0, K = 0, ncp = 0;
    bool valid = false;
    std::vector<std::pair<void *, size_t>> bufs;  // the device state, buffer by buffer
    size_t state_bytes = 0;
    std::vector<void *> cps;                      // ncp checkpoints, then the final state
    size_t tape_k = 0;                            // steps the recording buffers hold
    void *tape = nullptr;                         // 5 planes per step
    void *xi_tape = nullptr;                      // K + 1 reference-map snapshots
    Frame *fr_tape = nullptr;
    int *reg_tape = nullptr;                      // K + 1 registries
    void *fb[2] = {nullptr, nullptr}, *cb[2] = {nullptr, nullptr};
    void *Fb = nullptr, *Db = nullptr, *xib[2] = {nullptr, nullptr};
    double *Gb = nullptr, *dLdc = nullptr;
};

void lbrmt_internal_adjoint_free(lbrmt_sim *s) {
    delete s->adj;  // its device memory is owned by the simulation's allocation list
    s->adj = nullptr;
}

static void collect_state(lbrmt_sim *s, AdjointStore &A) {
    const DevState &d = s->d;
    const size_t P = (size_t)s->sp.P, ntiles = (size_t)s->sp.ntx * s->sp.nty;
    const size_t rs = s->eng->real_size, ss = s->eng->store_size, S = s->solids.size();
    A.bufs.clear();
    for (int k = 0; k < 2; k++) {
        A.bufs.push_back({d.f[k], 9 * P * ss});
        A.bufs.push_back({d.xi[k], (size_t)s->xi_total * rs});
        A.bufs.push_back({d.frame[k], S * sizeof(Frame)});
        A.bufs.push_back({d.reg_count[k], ntiles * 4});
        A.bufs.push_back({d.reg_solids[k], ntiles * KMAX * 4});
        A.bufs.push_back({d.reg_active[k], ntiles * 4});
        A.bufs.push_back({d.reg_nactive[k], 16});
        A.bufs.push_back({d.pool[k], ntiles * POOL_STRIDE * rs});
        A.bufs.push_back({d.busy[k], (size_t)s->sp.nrx * s->sp.nty});
    }
    A.bufs.push_back({d.carry, P * ss});
    A.bufs.push_back({d.stats_step, S * 64});
    A.state_bytes = 0;
    for (auto &b : A.bufs) A.state_bytes += (b.second + 255) & ~(size_t)255;
}

static cudaError_t save_state(lbrmt_sim *s, const AdjointStore &A, void *blob) {
    size_t off = 0;
    for (auto &b : A.bufs) {
        if (b.second && b.first) {
            cudaError_t e = cudaMemcpyAsync((char *)blob + off, b.first, b.second, cudaMemcpyDeviceToDevice, s->stream);
            if (e != cudaSuccess) return e;
        }
        off += (b.second + 255) & ~(size_t)255;
    }
    return cudaSuccess;
}

static cudaError_t load_state(lbrmt_sim *s, const AdjointStore &A, const void *blob) {
    size_t off = 0;
    for (auto &b : A.bufs) {
        if (b.second && b.first) {
            cudaError_t e = cudaMemcpyAsync(b.first, (const char *)blob + off, b.second, cudaMemcpyDeviceToDevice, s->stream);
            if (e != cudaSuccess) return e;
        }
        off += (b.second + 255) & ~(size_t)255;
    }
    return cudaSuccess;
}

extern "C" lbrmt_status lbrmt_forward_checkpointed(lbrmt_sim *s, int nsteps, int checkpoint_every,
                                                   double *centroids_out) {
    if (!s || nsteps < 1 || checkpoint_every < 1) return LBRMT_ERR_ARG;
    if (s->cfg.precision != LBRMT_FP32 && s->cfg.precision != LBRMT_FP64)
        return lbrmt_internal_fail(s, LBRMT_ERR_ARG, "the adjoint needs FP32 or FP64 storage");
    if (s->in_batch) return lbrmt_internal_fail(s, LBRMT_ERR_STATE, "a batch member is stepped by its batch");
    if (s->cfg.force_mode != LBRMT_FORCE_MODE_LITERAL)
        return lbrmt_internal_fail(s, LBRMT_ERR_ARG, "the adjoint supports force_mode 0 (rho F in the Guo term) only");
    for (const SolidHost &h : s->solids)
        if (h.shape != LBRMT_SHAPE_DISK) return lbrmt_internal_fail(s, LBRMT_ERR_ARG, "the adjoint supports disks only");
    lbrmt_status st = s->inited ? lbrmt_reset(s) : lbrmt_init(s);
    if (st != LBRMT_OK) return st;
    if (!s->adj) s->adj = new AdjointStore();
    AdjointStore &A = *s->adj;
    A.valid = false;
    collect_state(s, A);
    const int ncp = (nsteps + checkpoint_every - 1) / checkpoint_every;
    while ((int)A.cps.size() < ncp + 1) {
        void *p = lbrmt_internal_alloc(s, A.state_bytes);
        if (!p) return lbrmt_internal_fail(s, LBRMT_ERR_CUDA, "out of device memory for checkpoints");
        A.cps.push_back(p);
    }
    A.T = nsteps;
    A.K = checkpoint_every;
    A.ncp = ncp;
    for (int c = 0; c < ncp; c++) {
        cudaError_t e = save_state(s, A, A.cps[c]);
        if (e != cudaSuccess) return lbrmt_internal_fail(s, LBRMT_ERR_CUDA, "checkpoint");
        st = lbrmt_step(s, std::min(checkpoint_every, nsteps - c * checkpoint_every));
        if (st != LBRMT_OK) return st;
    }
    cudaError_t e = save_state(s, A, A.cps[ncp]);
    if (e != cudaSuccess) return lbrmt_internal_fail(s, LBRMT_ERR_CUDA, "checkpoint");
    const int S = (int)s->solids.size();
    std::vector<double> stt((size_t)std::max(S, 1) * STATS_COLS);
    st = lbrmt_solid_stats(s, 0, stt.data());
    if (st != LBRMT_OK) return st;
    if (centroids_out)
        for (int k = 0; k < S; k++) {
            centroids_out[2 * k] = stt[STATS_COLS * k + 1];
            centroids_out[2 * k + 1] = stt[STATS_COLS * k + 2];
        }
    A.valid = true;
    return LBRMT_OK;
}

namespace lbrmt {
template <class R>
__global__ void to_double_kernel(const R *src, double *dst, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        dst[k] = (double)src[k];
}
}  // namespace lbrmt

template <class R>
static lbrmt_status backward_impl(lbrmt_sim *s, const double *dLdc, double *dLdG, double *dLdratio, double *bodyb,
                                  double *df0) {
    AdjointStore &A = *s->adj;
    const SimParams &sp = s->sp;
    DevState &d = s->d;
    const int S = (int)s->solids.size();
    const long long P = sp.P;
    const size_t ntiles = (size_t)sp.ntx * sp.nty;
    const size_t reg_slot = ntiles * (KMAX + 2) + 4;  // count, solids, active, nactive
    const int K = A.K, T = A.T;
    cudaStream_t st = s->stream;
    // recording and adjoint buffers
    if (A.tape_k < (size_t)K || !A.tape) {
        A.tape = lbrmt_internal_alloc(s, (size_t)K * 5 * P * sizeof(R));
        A.xi_tape = lbrmt_internal_alloc(s, (size_t)(K + 1) * s->xi_total * sizeof(R));
        A.fr_tape = (Frame *)lbrmt_internal_alloc(s, (size_t)(K + 1) * std::max(S, 1) * sizeof(Frame));
        A.reg_tape = (int *)lbrmt_internal_alloc(s, (size_t)(K + 1) * reg_slot * 4);
        if (!A.tape || !A.xi_tape || !A.fr_tape || !A.reg_tape)
            return lbrmt_internal_fail(s, LBRMT_ERR_CUDA, "out of device memory for the adjoint tape");
        A.tape_k = K;
    }
    if (!A.Fb) {
        for (int k = 0; k < 2; k++) {
            A.fb[k] = lbrmt_internal_alloc(s, 9 * P * sizeof(R));
            A.cb[k] = lbrmt_internal_alloc(s, 2 * P * sizeof(R));
            A.xib[k] = lbrmt_internal_alloc(s, std::max<long long>(s->xi_total, 1) * sizeof(R));
        }
        A.Fb = lbrmt_internal_alloc(s, 2 * P * sizeof(R));
        A.Db = lbrmt_internal_alloc(s, P * sizeof(R));
        A.Gb = (double *)lbrmt_internal_alloc(s, (size_t)std::max(S, 1) * 2 * 8);
        A.dLdc = (double *)lbrmt_internal_alloc(s, (size_t)std::max(S, 1) * 2 * 8);
        if (!A.fb[0] || !A.fb[1] || !A.cb[0] || !A.cb[1] || !A.xib[0] || !A.xib[1] || !A.Fb || !A.Db || !A.Gb || !A.dLdc)
            return lbrmt_internal_fail(s, LBRMT_ERR_CUDA, "out of device memory for the adjoint");
    }
    double *Gb = A.Gb, *Rb = A.Gb + std::max(S, 1);
    R *xib[2] = {(R *)A.xib[0], (R *)A.xib[1]};
    R *fb[2] = {(R *)A.fb[0], (R *)A.fb[1]}, *cb[2] = {(R *)A.cb[0], (R *)A.cb[1]};
    const size_t xib_bytes = (size_t)s->xi_total * sizeof(R);
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    ok(upload_rinv_tables());  // this unit's copy of the 1/|d| tables of the directional weights
    ok(cudaMemsetAsync(A.Gb, 0, (size_t)std::max(S, 1) * 16, st));
    ok(cudaMemcpyAsync(A.dLdc, dLdc, (size_t)S * 16, cudaMemcpyHostToDevice, st));
    for (int k = 0; k < 2; k++) ok(cudaMemsetAsync(xib[k], 0, xib_bytes, st));
    ok(cudaMemsetAsync(fb[T & 1], 0, 9 * P * sizeof(R), st));
    ok(cudaMemsetAsync(cb[T & 1], 0, 2 * P * sizeof(R), st));
    if (bodyb) ok(cudaMemsetAsync(bodyb, 0, 2 * P * 8, st));
    // the loss: adjoint of xi^T from dL/dc on the final state
    ok(load_state(s, A, A.cps[A.ncp]));
    if (S > 0)
        centroid_seed_kernel<R><<<S, 256, 0, st>>>(sp, (const R *)d.xi[T & 1], d.frame[T & 1], d.solids, A.dLdc, xib[T & 1]);
    ok(cudaGetLastError());
    int nsm = 0, dev = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int fsm = force_adj_smem_elems(sp.tx, sp.ty) * (int)sizeof(R);
    ok(cudaFuncSetAttribute(force_adjoint_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            force_adj_smem_max() * (int)sizeof(R)));
    ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, force_adjoint_kernel<R>, TILE_N, fsm));
    const int fblocks = nsm * std::max(per, 1);
    const int rsm = ((s->li.tmax * s->li.tmax + 15) & ~15) + 8 * LIST_CAP;  // labels and layer lists
    ok(cudaFuncSetAttribute(rmt_adjoint_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, RMT_SMEM_MAX));
    // the forward's choice: 1024-thread CTAs for FP32 arithmetic and few solids
    constexpr bool can_big = sizeof(R) == 4;
    const bool big = can_big && s->li.rmt_threads == RMT_THREADS_BIG;
    if constexpr (can_big)
        if (big) ok(cudaFuncSetAttribute(rmt_adjoint_kernel_big<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, RMT_SMEM_MAX));
    const int lblocks = (int)std::min<long long>((P + 255) / 256, (long long)nsm * 8);
    if (e != cudaSuccess) return lbrmt_internal_fail(s, LBRMT_ERR_CUDA, std::string("adjoint setup: ") + cudaGetErrorString(e));

    R *tape = (R *)A.tape, *xit = (R *)A.xi_tape;
    auto xi_slot = [&](int m) { return xit + (size_t)m * s->xi_total; };
    auto fr_slot = [&](int m) { return A.fr_tape + (size_t)m * std::max(S, 1); };
    auto reg_slot_ptr = [&](int m) { return A.reg_tape + (size_t)m * reg_slot; };
    auto copy_registry = [&](int m, int r) {
        int *g = reg_slot_ptr(m);
        ok(cudaMemcpyAsync(g, d.reg_count[r], ntiles * 4, cudaMemcpyDeviceToDevice, st));
        ok(cudaMemcpyAsync(g + ntiles, d.reg_solids[r], ntiles * KMAX * 4, cudaMemcpyDeviceToDevice, st));
        ok(cudaMemcpyAsync(g + ntiles * (KMAX + 1), d.reg_active[r], ntiles * 4, cudaMemcpyDeviceToDevice, st));
        ok(cudaMemcpyAsync(g + ntiles * (KMAX + 2), d.reg_nactive[r], 4, cudaMemcpyDeviceToDevice, st));
    };
    auto force_args = [&](int m) {
        ForceAdjArgs<R> fa;
        const int *g = reg_slot_ptr(m);
        fa.xi = xi_slot(m);
        fa.frame = fr_slot(m);
        fa.reg_count = g;
        fa.reg_solids = g + ntiles;
        fa.reg_active = g + ntiles * (KMAX + 1);
        fa.reg_nactive = g + ntiles * (KMAX + 2);
        fa.solids = d.solids;
        fa.Fb = (const R *)A.Fb;
        fa.Db = (const R *)A.Db;
        fa.Gb = Gb;
        fa.Rb = Rb;
        return fa;
    };
    for (int seg = A.ncp - 1; seg >= 0 && e == cudaSuccess; seg--) {
        const int n0 = seg * K, n1 = std::min(T, n0 + K);
        // recompute the segment, recording it
        ok(load_state(s, A, A.cps[seg]));
        s->steps = n0;
        ok(cudaMemcpyAsync(xi_slot(0), d.xi[n0 & 1], xib_bytes, cudaMemcpyDeviceToDevice, st));
        if (S > 0) ok(cudaMemcpyAsync(fr_slot(0), d.frame[n0 & 1], S * sizeof(Frame), cudaMemcpyDeviceToDevice, st));
        copy_registry(0, (n0 & 1) ^ 1);
        for (int n = n0; n < n1 && e == cudaSuccess; n++) {
            const int m = n - n0;
            ok(s->eng->step(sp, d, s->li, n & 1, st, nullptr, tape + (size_t)m * 5 * P, CHAIN_ONE));
            s->steps++;
            ok(cudaMemcpyAsync(xi_slot(m + 1), d.xi[(n + 1) & 1], xib_bytes, cudaMemcpyDeviceToDevice, st));
            if (S > 0) ok(cudaMemcpyAsync(fr_slot(m + 1), d.frame[(n + 1) & 1], S * sizeof(Frame), cudaMemcpyDeviceToDevice, st));
            copy_registry(m + 1, n & 1);
        }
        // reverse sweep over the segment
        for (int n = n1 - 1; n >= n0 && e == cudaSuccess; n--) {
            const int m = n - n0, p = n & 1, q = p ^ 1;
            LbAdjArgs<R> la;
            la.tape = tape + (size_t)m * 5 * P;
            la.fb_next = fb[q];
            la.cb_next = cb[q];
            la.fb = fb[p];
            la.cb = cb[p];
            la.Fb = (R *)A.Fb;
            la.Db = (R *)A.Db;
            la.bodyb = bodyb;
            lb_adjoint_kernel<R><<<lblocks, 256, 0, st>>>(sp, la);
            if (S > 0) {
                ForceAdjArgs<R> fa = force_args(m + 1);
                fa.xib = xib[q];
                force_adjoint_kernel<R><<<fblocks, TILE_N, fsm, st>>>(sp, fa, 0);
                RmtAdjArgs<R> ra;
                ra.xi_in = xi_slot(m);
                ra.xi_out = xi_slot(m + 1);
                ra.frame_in = fr_slot(m);
                ra.frame_out = fr_slot(m + 1);
                ra.tape = la.tape;
                ra.xib_out = xib[q];
                ra.xib_in = xib[p];
                ra.fb = fb[p];
                ra.cb = cb[p];
                ra.solids = d.solids;
                bool launched = false;
                if constexpr (can_big)
                    if (big) {
                        rmt_adjoint_kernel_big<R><<<S, RMT_THREADS_BIG, rsm, st>>>(sp, ra);
                        launched = true;
                    }
                if (!launched) rmt_adjoint_kernel<R><<<S, RMT_THREADS, rsm, st>>>(sp, ra);
                ok(cudaMemsetAsync(xib[q], 0, xib_bytes, st));
            }
            ok(cudaGetLastError());
        }
        if (seg == 0 && S > 0 && e == cudaSuccess) {
            // f^0_0 = w_0 rho_f + Delta rho^0: the rest population's adjoint is that of Delta rho^0
            ForceAdjArgs<R> fa = force_args(0);
            fa.Fb = nullptr;
            fa.Db = fb[0];  // plane q = 0
            fa.xib = xib[1];
            force_adjoint_kernel<R><<<fblocks, TILE_N, fsm, st>>>(sp, fa, 1);
            ok(cudaGetLastError());
        }
    }
    if (df0) {
        to_double_kernel<R><<<256, 256, 0, st>>>(fb[0], df0, 9 * P);
        ok(cudaGetLastError());
    }
    std::vector<double> h((size_t)std::max(S, 1) * 2);
    ok(cudaMemcpyAsync(h.data(), A.Gb, h.size() * 8, cudaMemcpyDeviceToHost, st));
    ok(cudaStreamSynchronize(st));
    // back to the final forward state
    ok(load_state(s, A, A.cps[A.ncp]));
    s->steps = T;
    ok(cudaStreamSynchronize(st));
    if (e != cudaSuccess) return lbrmt_internal_fail(s, LBRMT_ERR_CUDA, std::string("adjoint: ") + cudaGetErrorString(e));
    for (int k = 0; k < S; k++) {
        if (dLdG) dLdG[k] = h[k];
        if (dLdratio) dLdratio[k] = h[std::max(S, 1) + k];
    }
    return lbrmt_internal_check_flags(s);
}

extern "C" lbrmt_status lbrmt_backward(lbrmt_sim *s, const double *dL_dcentroid, double *dL_dG, double *dL_dratio,
                                       double *dL_dbody_dev, double *dL_df0_dev) {
    if (!s || !dL_dcentroid) return LBRMT_ERR_ARG;
    if (!s->adj || !s->adj->valid)
        return lbrmt_internal_fail(s, LBRMT_ERR_STATE, "lbrmt_backward needs a preceding lbrmt_forward_checkpointed");
    if (dL_dbody_dev && s->cfg.force_kind != LBRMT_FORCE_FIELD)
        return lbrmt_internal_fail(s, LBRMT_ERR_ARG, "the body force gradient needs force_kind LBRMT_FORCE_FIELD");
    if (s->eng->real_size == 8) return backward_impl<double>(s, dL_dcentroid, dL_dG, dL_dratio, dL_dbody_dev, dL_df0_dev);
    return backward_impl<float>(s, dL_dcentroid, dL_dG, dL_dratio, dL_dbody_dev, dL_df0_dev);
}
