// lbrmt_batch.cu -- host runtime of a batch of independent simulations.
//
// Each member is an ordinary simulation (its own device state, created
// through lbrmt_create on the batch's stream).  The batch keeps a device array
// of member descriptors and two work lists: (member, solid) for K2 and
// (member, tile) for K1; K3 walks the members' active-tile lists.  A batch
// step is one persistent launch per phase; steps are replayed through CUDA
// graphs of 2 and of BATCH_GRAPH_STEPS steps.
//
// Tile-shape autotuner: the registry / LB tile (tile_x x 256/tile_x) changes
// how tightly the tiles cover the solids' blur zones (K3 and the solid path of
// K1 work per registered tile) and how many tiles a ragged grid edge wastes,
// but not the results.  Greedy per grid size: starting from the configured
// shapes, each group of members with the same (nx, ny) tries every shape with
// the others fixed, timing whole batch steps, and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "lbrmt.h"
#include "lbrmt_engine.cuh"
#include "lbrmt_sim.cuh"

using namespace lbrmt;

namespace {

constexpr int BATCH_GRAPH_STEPS = 20;
constexpr int TILE_CHOICES[4] = {16, 32, 64, 128};

struct SolidSpec {
    int shape;
    double cx, cy, a, b, rho_s, G;
};

struct Member {
    lbrmt_config cfg;
    std::vector<SolidSpec> solids;
    lbrmt_sim *sim = nullptr;
};

}  // namespace

struct lbrmt_batch {
    std::vector<Member> m;
    cudaStream_t stream = nullptr;
    const EngineOps *eng = nullptr;
    bool inited = false;
    long long steps = 0;
    void *descs = nullptr;
    int2 *rmt_items = nullptr, *lb_items = nullptr;
    int n_rmt = 0, n_lb = 0;
    BatchLaunch bl{};
    cudaGraphExec_t g2 = nullptr, gmany = nullptr;
    long long last_launches = 0;
    std::vector<void *> allocs;
    std::vector<int> tune_side_nx, tune_side_ny, tune_tile;
    std::vector<double> tune_ms;
    std::string err;
};

static lbrmt_status bfail(lbrmt_batch *b, lbrmt_status st, const std::string &msg) {
    if (b) b->err = msg;
    return st;
}

static lbrmt_status bcuda(lbrmt_batch *b, cudaError_t e, const char *where) {
    return bfail(b, LBRMT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static lbrmt_status member_fail(lbrmt_batch *b, int k, lbrmt_status st) {
    const char *msg = b->m[k].sim ? lbrmt_last_error(b->m[k].sim) : "";
    return bfail(b, st, "member " + std::to_string(k) + ": " + (msg ? msg : ""));
}

static void *balloc(lbrmt_batch *b, size_t bytes) {
    const lbrmt_config &c = b->m[0].cfg;
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (c.alloc) p = c.alloc(bytes, c.alloc_ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) b->allocs.push_back(p);
    return p;
}

static void bfree_all(lbrmt_batch *b) {
    const lbrmt_config &c = b->m[0].cfg;
    for (void *p : b->allocs) {
        if (c.free) c.free(p, c.alloc_ctx);
        else cudaFree(p);
    }
    b->allocs.clear();
    b->descs = nullptr;
    b->rmt_items = b->lb_items = nullptr;
}

static void drop_graphs(lbrmt_batch *b) {
    if (b->g2) cudaGraphExecDestroy(b->g2);
    if (b->gmany) cudaGraphExecDestroy(b->gmany);
    b->g2 = b->gmany = nullptr;
}

// (Re)create member k from its config and solids, and initialise it.
static lbrmt_status make_member(lbrmt_batch *b, int k) {
    Member &mb = b->m[k];
    if (mb.sim) {
        lbrmt_destroy(mb.sim);
        mb.sim = nullptr;
    }
    lbrmt_status st = lbrmt_create(&mb.cfg, b->stream, &mb.sim);
    if (st != LBRMT_OK) return bfail(b, st, "member " + std::to_string(k) + ": create");
    for (const SolidSpec &s : mb.solids) {
        st = lbrmt_add_solid_shape(mb.sim, s.shape, s.cx, s.cy, s.a, s.b, s.rho_s, s.G, nullptr);
        if (st != LBRMT_OK) return member_fail(b, k, st);
    }
    st = lbrmt_init(mb.sim);
    if (st != LBRMT_OK) return member_fail(b, k, st);
    mb.sim->in_batch = true;
    return LBRMT_OK;
}

// Descriptors, work lists and launch shapes for the current members.
static lbrmt_status build_lists(lbrmt_batch *b) {
    drop_graphs(b);
    bfree_all(b);
    const int n = (int)b->m.size();
    std::vector<unsigned char> desc((size_t)n * b->eng->desc_size);
    std::vector<int2> rmt, lb;
    std::vector<int> rmt_T;
    int tmax = 8, fs_elems = 0;
    for (int k = 0; k < n; k++) {
        lbrmt_sim *s = b->m[k].sim;
        b->eng->fill_desc(desc.data() + (size_t)k * b->eng->desc_size, s->sp, s->d);
        for (int q = 0; q < (int)s->solids.size(); q++) {
            rmt.push_back(make_int2(k, q));
            rmt_T.push_back(s->solids[q].T);
            tmax = std::max(tmax, s->solids[q].T);
        }
        if (s->sp.nrx >= 65536 || s->sp.nty >= 32768) return bfail(b, LBRMT_ERR_ARG, "member grid too large for a batch");
        for (int ry = 0; ry < s->sp.nty; ry++)
            for (int rx = 0; rx < s->sp.nrx; rx++) lb.push_back(make_int2(k, (ry << 16) | rx));
        fs_elems = std::max(fs_elems, force_smem_elems(s->sp.tx, s->sp.ty));
    }
    // largest solid tiles first: the persistent K2 grid then ends with the short items
    std::vector<int> order(rmt.size());
    for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return rmt_T[a] > rmt_T[c]; });
    std::vector<int2> rmt_sorted(rmt.size());
    for (size_t i = 0; i < order.size(); i++) rmt_sorted[i] = rmt[order[i]];
    b->n_rmt = (int)rmt_sorted.size();
    b->n_lb = (int)lb.size();
    b->descs = balloc(b, desc.size());
    b->rmt_items = (int2 *)balloc(b, std::max<size_t>(1, rmt_sorted.size()) * sizeof(int2));
    b->lb_items = (int2 *)balloc(b, lb.size() * sizeof(int2));
    if (!b->descs || !b->rmt_items || !b->lb_items) return bfail(b, LBRMT_ERR_CUDA, "out of device memory for the batch lists");
    cudaError_t e = cudaMemcpy(b->descs, desc.data(), desc.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && b->n_rmt)
        e = cudaMemcpy(b->rmt_items, rmt_sorted.data(), rmt_sorted.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->lb_items, lb.data(), lb.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(b, e, "upload batch lists");
    e = b->eng->batch_configure(tmax, fs_elems, b->n_rmt, &b->bl);
    if (e != cudaSuccess) return bcuda(b, e, "configure batch kernels");
    return LBRMT_OK;
}

static lbrmt_status direct_batch_step(lbrmt_batch *b, cudaEvent_t *ev) {
    cudaError_t e = b->eng->batch_step(b->descs, (int)b->m.size(), b->rmt_items, b->n_rmt, b->lb_items, b->n_lb, b->bl,
                                       (int)(b->steps & 1), b->stream, ev);
    if (e != cudaSuccess) return bcuda(b, e, "batch step launch");
    b->steps++;
    for (Member &mb : b->m) mb.sim->steps++;
    b->last_launches += batch_launches(b->bl, b->n_rmt, ev != nullptr);
    return LBRMT_OK;
}

static lbrmt_status capture(lbrmt_batch *b, int nsteps, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "begin capture");
    cudaError_t el = cudaSuccess;
    for (int k = 0; k < nsteps && el == cudaSuccess; k++)
        el = b->eng->batch_step(b->descs, (int)b->m.size(), b->rmt_items, b->n_rmt, b->lb_items, b->n_lb, b->bl, k & 1,
                                b->stream, nullptr);
    e = cudaStreamEndCapture(b->stream, &g);
    if (el != cudaSuccess) e = el;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, e, "capture");
    }
    // per-node priorities: the overlapped step runs K2, K3 and the busy K1 ahead of the free K1
    e = cudaGraphInstantiate(out, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return bcuda(b, e, "instantiate graph");
    }
    return LBRMT_OK;
}

static lbrmt_status check_members(lbrmt_batch *b) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "stream");
    for (int k = 0; k < (int)b->m.size(); k++) {
        lbrmt_status st = lbrmt_internal_check_flags(b->m[k].sim);
        if (st != LBRMT_OK) return member_fail(b, k, st);
    }
    return LBRMT_OK;
}

// Mean ms per batch step over `steps` direct steps (after 4 warm-up steps), best of two.
// A trial takes an even number of steps: members re-created between trials start
// at step 0, and every member's state must have the parity of the batch's count.
static lbrmt_status time_trial(lbrmt_batch *b, int steps, double *ms_out) {
    steps += steps & 1;
    for (int k = 0; k < 4; k++) {
        lbrmt_status st = direct_batch_step(b, nullptr);
        if (st != LBRMT_OK) return st;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e30;
    lbrmt_status st = LBRMT_OK;
    for (int rep = 0; rep < 2 && st == LBRMT_OK; rep++) {
        cudaEventRecord(e0, b->stream);
        for (int k = 0; k < steps && st == LBRMT_OK; k++) st = direct_batch_step(b, nullptr);
        cudaEventRecord(e1, b->stream);
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) st = bcuda(b, e, "trial");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, (double)ms / steps);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == LBRMT_OK) st = check_members(b);
    *ms_out = best;
    return st;
}

static lbrmt_status autotune(lbrmt_batch *b, int steps) {
    // groups of members with the same grid size
    std::map<std::pair<int, int>, std::vector<int>> groups;
    for (int k = 0; k < (int)b->m.size(); k++) groups[{b->m[k].cfg.nx, b->m[k].cfg.ny}].push_back(k);
    double base = 0.0;
    b->steps = 0;  // every member was just created
    lbrmt_status st = build_lists(b);
    if (st == LBRMT_OK) st = time_trial(b, steps, &base);
    if (st != LBRMT_OK) return st;
    for (auto &g : groups) {
        const int cur = b->m[g.second[0]].cfg.tile_x;
        b->tune_side_nx.push_back(g.first.first);
        b->tune_side_ny.push_back(g.first.second);
        b->tune_tile.push_back(cur);
        b->tune_ms.push_back(base);
        int best = cur;
        double best_ms = base;
        int live = cur;  // shape the group's members currently have
        for (int tx : TILE_CHOICES) {
            if (tx == cur) continue;
            for (int k : g.second) {
                b->m[k].cfg.tile_x = tx;
                st = make_member(b, k);
                if (st != LBRMT_OK) return st;
            }
            live = tx;
            double ms = 0.0;
            st = build_lists(b);
            if (st == LBRMT_OK) st = time_trial(b, steps, &ms);
            if (st != LBRMT_OK) return st;
            b->tune_side_nx.push_back(g.first.first);
            b->tune_side_ny.push_back(g.first.second);
            b->tune_tile.push_back(tx);
            b->tune_ms.push_back(ms);
            if (ms < best_ms) {
                best_ms = ms;
                best = tx;
            }
        }
        for (int k : g.second) b->m[k].cfg.tile_x = best;
        if (live != best)
            for (int k : g.second) {
                st = make_member(b, k);
                if (st != LBRMT_OK) return st;
            }
        base = best_ms;
    }
    return LBRMT_OK;
}

extern "C" lbrmt_status lbrmt_create_batch(const lbrmt_config *cfgs, int nsim, void *cuda_stream, lbrmt_batch **out) {
    if (!cfgs || !out || nsim < 1 || nsim > BATCH_MAX) return LBRMT_ERR_ARG;
    *out = nullptr;
    for (int k = 1; k < nsim; k++)
        if (cfgs[k].precision != cfgs[0].precision) return LBRMT_ERR_ARG;
    lbrmt_batch *b = new lbrmt_batch();
    b->stream = (cudaStream_t)cuda_stream;
    b->m.resize(nsim);
    for (int k = 0; k < nsim; k++) {
        b->m[k].cfg = cfgs[k];
        if (b->m[k].cfg.tile_x == 0) b->m[k].cfg.tile_x = 32;
        // validate now (the member is re-created at initialisation)
        lbrmt_status st = lbrmt_create(&b->m[k].cfg, b->stream, &b->m[k].sim);
        if (st != LBRMT_OK) {
            lbrmt_destroy_batch(b);
            return st;
        }
    }
    b->eng = b->m[0].sim->eng;
    // side stream (lowest priority) and fork / join events of the overlapped step
    int least = 0, greatest = 0;
    BatchLaunch &bl = b->bl;
    const bool ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
                    cudaStreamCreateWithPriority(&bl.side, cudaStreamNonBlocking, least) == cudaSuccess &&
                    cudaEventCreateWithFlags(&bl.fork, cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventCreateWithFlags(&bl.join, cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventCreateWithFlags(&bl.flags, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        lbrmt_destroy_batch(b);
        return LBRMT_ERR_CUDA;
    }
    bl.prio_hi = greatest;
    bl.split = true;
    *out = b;
    return LBRMT_OK;
}

extern "C" lbrmt_status lbrmt_batch_set_overlap(lbrmt_batch *b, int enable) {
    if (!b) return LBRMT_ERR_ARG;
    if (b->stream) cudaStreamSynchronize(b->stream);
    b->bl.split = enable != 0;
    drop_graphs(b);
    return LBRMT_OK;
}

extern "C" int lbrmt_batch_uses_overlap(const lbrmt_batch *b) {
    return b && b->inited && batch_overlaps(b->bl, b->n_rmt) ? 1 : 0;
}

extern "C" lbrmt_status lbrmt_batch_add_solid_shape(lbrmt_batch *b, int sim_index, int shape, double cx, double cy,
                                                    double a, double bb, double rho_s, double G, int *solid_id_out) {
    if (!b || sim_index < 0 || sim_index >= (int)b->m.size()) return LBRMT_ERR_ARG;
    if (b->inited) return bfail(b, LBRMT_ERR_STATE, "solids must be added before lbrmt_batch_init");
    Member &mb = b->m[sim_index];
    lbrmt_status st = lbrmt_add_solid_shape(mb.sim, shape, cx, cy, a, bb, rho_s, G, solid_id_out);
    if (st != LBRMT_OK) return member_fail(b, sim_index, st);
    mb.solids.push_back(SolidSpec{shape, cx, cy, a, shape == LBRMT_SHAPE_DISK ? a : bb, rho_s, G});
    return LBRMT_OK;
}

extern "C" lbrmt_status lbrmt_batch_add_solid(lbrmt_batch *b, int sim_index, int shape, double cx, double cy,
                                              double radius, double rho_s, double G, int *solid_id_out) {
    if (b && shape != LBRMT_SHAPE_DISK) return bfail(b, LBRMT_ERR_ARG, "lbrmt_batch_add_solid adds disks");
    return lbrmt_batch_add_solid_shape(b, sim_index, LBRMT_SHAPE_DISK, cx, cy, radius, radius, rho_s, G, solid_id_out);
}

extern "C" lbrmt_status lbrmt_batch_init(lbrmt_batch *b, int autotune_steps) {
    if (!b || autotune_steps < 0) return LBRMT_ERR_ARG;
    if (b->inited) return LBRMT_OK;
    lbrmt_status st = LBRMT_OK;
    for (int k = 0; k < (int)b->m.size() && st == LBRMT_OK; k++) st = make_member(b, k);
    if (st == LBRMT_OK && autotune_steps > 0) {
        st = autotune(b, autotune_steps);
        // the trials advanced the members: start every member again from its initial state
        for (int k = 0; k < (int)b->m.size() && st == LBRMT_OK; k++) st = make_member(b, k);
    }
    if (st == LBRMT_OK) st = build_lists(b);
    if (st != LBRMT_OK) return st;
    b->steps = 0;
    b->inited = true;
    return check_members(b);
}

extern "C" lbrmt_status lbrmt_batch_step(lbrmt_batch *b, int nsteps) {
    if (!b || nsteps < 0) return LBRMT_ERR_ARG;
    if (!b->inited) {
        lbrmt_status st = lbrmt_batch_init(b, 0);
        if (st != LBRMT_OK) return st;
    }
    b->last_launches = 0;
    int left = nsteps;
    lbrmt_status st = LBRMT_OK;
    if (b->stream && nsteps >= 2) {
        if (b->steps & 1) {
            st = direct_batch_step(b, nullptr);
            left--;
        }
        if (st == LBRMT_OK && left >= BATCH_GRAPH_STEPS && !b->gmany) st = capture(b, BATCH_GRAPH_STEPS, &b->gmany);
        while (st == LBRMT_OK && left >= BATCH_GRAPH_STEPS) {
            cudaError_t e = cudaGraphLaunch(b->gmany, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "graph launch");
            for (int k = 0; k < BATCH_GRAPH_STEPS; k++) {
                b->steps++;
                for (Member &mb : b->m) mb.sim->steps++;
            }
            b->last_launches += (long long)BATCH_GRAPH_STEPS * batch_launches(b->bl, b->n_rmt);
            left -= BATCH_GRAPH_STEPS;
        }
        if (st == LBRMT_OK && left >= 2 && !b->g2) st = capture(b, 2, &b->g2);
        while (st == LBRMT_OK && left >= 2) {
            cudaError_t e = cudaGraphLaunch(b->g2, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "graph launch");
            for (int k = 0; k < 2; k++) {
                b->steps++;
                for (Member &mb : b->m) mb.sim->steps++;
            }
            b->last_launches += 2 * batch_launches(b->bl, b->n_rmt);
            left -= 2;
        }
    }
    while (st == LBRMT_OK && left > 0) {
        st = direct_batch_step(b, nullptr);
        left--;
    }
    return st;
}

extern "C" lbrmt_status lbrmt_batch_step_timed(lbrmt_batch *b, int nsteps, float *ms_out) {
    if (!b || nsteps < 1 || !ms_out) return LBRMT_ERR_ARG;
    if (!b->inited) {
        lbrmt_status st = lbrmt_batch_init(b, 0);
        if (st != LBRMT_OK) return st;
    }
    std::vector<cudaEvent_t> ev(4 * (size_t)nsteps, nullptr);
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return bfail(b, LBRMT_ERR_CUDA, "event create");
    b->last_launches = 0;
    lbrmt_status st = LBRMT_OK;
    for (int n = 0; n < nsteps && st == LBRMT_OK; n++) st = direct_batch_step(b, &ev[4 * (size_t)n]);
    double acc[3] = {0, 0, 0};
    if (st == LBRMT_OK) {
        cudaError_t e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) st = bcuda(b, e, "timed sync");
        for (int n = 0; n < nsteps && st == LBRMT_OK; n++)
            for (int k = 0; k < 3; k++) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[4 * (size_t)n + k], ev[4 * (size_t)n + k + 1]);
                acc[k] += ms;
            }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    for (int k = 0; k < 3; k++) ms_out[k] = (float)(acc[k] / nsteps);
    if (st != LBRMT_OK) return st;
    return check_members(b);
}

extern "C" lbrmt_status lbrmt_batch_sync(lbrmt_batch *b) {
    if (!b) return LBRMT_ERR_ARG;
    return check_members(b);
}

extern "C" lbrmt_status lbrmt_batch_member(lbrmt_batch *b, int sim_index, lbrmt_sim **out) {
    if (!b || !out || sim_index < 0 || sim_index >= (int)b->m.size()) return LBRMT_ERR_ARG;
    if (!b->inited) return bfail(b, LBRMT_ERR_STATE, "members are available after lbrmt_batch_init");
    *out = b->m[sim_index].sim;
    return LBRMT_OK;
}

extern "C" int lbrmt_batch_size(const lbrmt_batch *b) { return b ? (int)b->m.size() : 0; }

extern "C" int lbrmt_batch_tile_x(const lbrmt_batch *b, int sim_index) {
    if (!b || sim_index < 0 || sim_index >= (int)b->m.size()) return 0;
    return b->m[sim_index].cfg.tile_x;
}

extern "C" int lbrmt_batch_tune_log(const lbrmt_batch *b, int *nx, int *ny, int *tile_x, double *ms, int cap) {
    if (!b) return 0;
    const int n = (int)b->tune_ms.size();
    for (int k = 0; k < n && k < cap; k++) {
        if (nx) nx[k] = b->tune_side_nx[k];
        if (ny) ny[k] = b->tune_side_ny[k];
        if (tile_x) tile_x[k] = b->tune_tile[k];
        if (ms) ms[k] = b->tune_ms[k];
    }
    return n;
}

extern "C" long long lbrmt_batch_steps_done(const lbrmt_batch *b) { return b ? b->steps : 0; }

extern "C" long long lbrmt_batch_last_launch_count(const lbrmt_batch *b) { return b ? b->last_launches : 0; }

extern "C" const char *lbrmt_batch_last_error(const lbrmt_batch *b) { return b ? b->err.c_str() : ""; }

extern "C" void lbrmt_destroy_batch(lbrmt_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->bl.side) cudaStreamSynchronize(b->bl.side);
    drop_graphs(b);
    for (cudaEvent_t ev : {b->bl.fork, b->bl.join, b->bl.flags})
        if (ev) cudaEventDestroy(ev);
    if (b->bl.side) cudaStreamDestroy(b->bl.side);
    if (!b->m.empty()) bfree_all(b);
    for (Member &mb : b->m)
        if (mb.sim) lbrmt_destroy(mb.sim);
    delete b;
}
