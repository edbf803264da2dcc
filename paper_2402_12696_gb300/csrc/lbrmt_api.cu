// lbrmt_api.cu -- host runtime behind the C ABI of include/lbrmt.h.
//
// Owns the device state of one simulation, builds the solid tiles at
// initialisation, enqueues the three kernels of a step on the caller's stream
// and replays them through a two-step CUDA graph (the state is double-buffered
// by step parity, so steps 2k and 2k+1 form a fixed launch sequence).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbrmt.h"
#include "lbrmt_engine.cuh"
#include "lbrmt_sim.cuh"

using namespace lbrmt;

namespace lbrmt {
__global__ void mass_reduce_kernel(const double *partials, int n, double base, double *out) {
    __shared__ double sh[1024];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = base + sh[0];
}
}  // namespace lbrmt

static void drop_graphs(lbrmt_sim *s) {
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    if (s->gexec_long) cudaGraphExecDestroy(s->gexec_long);
    s->gexec = s->gexec_long = nullptr;
}

static void release_streams(lbrmt_sim *s) {
    if (s->li.fork) cudaEventDestroy(s->li.fork);
    if (s->li.join) cudaEventDestroy(s->li.join);
    if (s->li.flags) cudaEventDestroy(s->li.flags);
    for (auto &e : s->li.done)
        if (e) cudaEventDestroy(e);
    s->li.done[0] = s->li.done[1] = nullptr;
    if (s->li.side) cudaStreamDestroy(s->li.side);
    s->li.fork = s->li.join = s->li.flags = nullptr;
    s->li.side = nullptr;
}

static lbrmt_status fail(lbrmt_sim *s, lbrmt_status st, const std::string &msg) {
    if (s) s->err = msg;
    return st;
}

static lbrmt_status cuda_fail(lbrmt_sim *s, cudaError_t e, const char *where) {
    return fail(s, LBRMT_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static void *dalloc(lbrmt_sim *s, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (s->cfg.alloc) p = s->cfg.alloc(bytes, s->cfg.alloc_ctx);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (p) s->allocs.push_back(p);
    return p;
}

static void dfree_all(lbrmt_sim *s) {
    for (void *p : s->allocs) {
        if (s->cfg.free) s->cfg.free(p, s->cfg.alloc_ctx);
        else cudaFree(p);
    }
    s->allocs.clear();
}

extern "C" void lbrmt_default_config(lbrmt_config *c) {
    std::memset(c, 0, sizeof(*c));
    c->nx = 64; c->ny = 64;
    c->bc_x = LBRMT_PERIODIC; c->bc_y = LBRMT_PERIODIC;
    c->tau = 1.0; c->rho_f = 1.0; c->lid_u = 0.0;
    c->eps = 1.5; c->n_layers = 11; c->eta = 1.0;
    c->gravity = 0.0; c->force_kind = LBRMT_FORCE_NONE;
    c->precision = LBRMT_FP32;
    c->max_solids_per_tile = KMAX;
    c->rmax = 11;
    c->tile_x = 32;
    c->deform_margin = 0.25;
}

extern "C" lbrmt_status lbrmt_create(const lbrmt_config *cfg, void *cuda_stream, lbrmt_sim **out) {
    if (!cfg || !out) return LBRMT_ERR_ARG;
    *out = nullptr;
    const lbrmt_config &c = *cfg;
    if (c.nx < 8 || c.ny < 8 || 9ll * c.nx * c.ny >= (1ll << 31)) return LBRMT_ERR_ARG;
    if ((c.bc_x != 0 && c.bc_x != 1) || (c.bc_y != 0 && c.bc_y != 1)) return LBRMT_ERR_ARG;
    if (!(c.tau > 0.5 && c.tau <= 1.0)) return LBRMT_ERR_PARAM_RANGE;  // Appendix A
    if (!(c.rho_f > 0) || !(c.eps > 0) || c.n_layers < 1 || c.n_layers > 20) return LBRMT_ERR_ARG;
    if (c.max_solids_per_tile < 1 || c.max_solids_per_tile > KMAX || c.rmax < 2 || c.rmax > 20) return LBRMT_ERR_ARG;
    if (c.lid_u != 0.0 && c.bc_y != LBRMT_WALL) return LBRMT_ERR_ARG;
    if (!(c.gravity >= 0) || c.force_kind < 0 || c.force_kind > LBRMT_FORCE_FIELD) return LBRMT_ERR_ARG;
    if (c.precision < LBRMT_FP32 || c.precision > LBRMT_BF16_STORE) return LBRMT_ERR_ARG;
    if (!(c.deform_margin >= 0.0) || c.deform_margin > 4.0) return LBRMT_ERR_ARG;
    if (c.force_mode != LBRMT_FORCE_MODE_LITERAL && c.force_mode != LBRMT_FORCE_MODE_CONSERVATIVE) return LBRMT_ERR_ARG;
    const int tx = c.tile_x == 0 ? 32 : c.tile_x;
    if (tx != 16 && tx != 32 && tx != 64 && tx != 128) return LBRMT_ERR_ARG;

    if (std::fabs(c.lid_u) / std::sqrt(1.0 / 3.0) > 0.3) return LBRMT_ERR_PARAM_RANGE;  // Ma* <= 0.3

    lbrmt_sim *s = new lbrmt_sim();
    s->cfg = c;
    if (cudaGetDevice(&s->device) != cudaSuccess) s->device = 0;
    s->stream = (cudaStream_t)cuda_stream;
    s->eng = c.precision == LBRMT_FP64 ? &engine_fp64
             : c.precision == LBRMT_FP16_STORE ? &engine_fp16
             : c.precision == LBRMT_BF16_STORE ? &engine_bf16
                                                : &engine_fp32;
    SimParams &sp = s->sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.nx = c.nx; sp.ny = c.ny; sp.wall_x = c.bc_x; sp.wall_y = c.bc_y;
    set_tile_params(sp, tx);
    sp.P = (long long)c.nx * c.ny;
    sp.tau = c.tau; sp.rho_f = c.rho_f; sp.lid_u = c.lid_u; sp.eps = c.eps; sp.eta = c.eta;
    sp.gravity = c.gravity; sp.force_kind = c.force_kind; sp.fa0 = c.force_a[0]; sp.fa1 = c.force_a[1];
    sp.force_mode = c.force_mode;
    sp.n_layers = c.n_layers; sp.rmax = c.rmax; sp.kmax = c.max_solids_per_tile; sp.nsolids = 0;
    sp.omega = 1.0 / c.tau; sp.kf = 1.0 - 0.5 / c.tau; sp.fy = c.force_kind == LBRMT_FORCE_CONST ? c.force_a[1] : 0.0;
    sp.omega_f = (float)sp.omega; sp.kf_f = (float)sp.kf; sp.rho_f_f = (float)c.rho_f; sp.lid_u_f = (float)c.lid_u;
    sp.eps_f = (float)c.eps; sp.eta_f = (float)c.eta; sp.fy_f = (float)sp.fy;
    {  // solid-fraction table grid: the largest power-of-two step with at most LAM_TAB_MAX entries
        int m = 0;
        while (2 * (int)std::ceil(c.eps * std::ldexp(1.0, m + 1)) + 1 <= LAM_TAB_MAX) m++;
        sp.lam_h = (float)std::ldexp(1.0, -m);
        sp.eps_lo = (float)(c.eps - (double)sp.eps_f);
        sp.lam_inv_h = (float)std::ldexp(1.0, m);
        sp.lam_k0 = (int)std::ceil(c.eps * std::ldexp(1.0, m));
    }

    // registry and pool sized for the largest tile count over the tile shapes, so
    // the shape can change later (lbrmt_set_tile_x) without reallocation
    size_t ntiles = 0, nparts = 0, nregions = 0;
    for (int w = 16; w <= 128; w *= 2) {
        SimParams t = sp;
        set_tile_params(t, w);
        ntiles = std::max(ntiles, (size_t)t.ntx * (size_t)t.nty);
        nparts = std::max(nparts, (size_t)t.ntx * (size_t)t.nty);  // one mass partial per registry tile
        nregions = std::max(nregions, (size_t)t.nrx * (size_t)t.nty);
    }
    s->ntiles_cap = (long long)ntiles;
    s->mass_parts_cap = (long long)nparts;
    s->nregions_cap = (long long)nregions;
    const size_t P = (size_t)sp.P;
    const size_t rs = s->eng->real_size, ss = s->eng->store_size;
    DevState &d = s->d;
    std::memset(&d, 0, sizeof(d));
    bool ok = true;
    for (int k = 0; k < 2; k++) {
        ok = ok && (d.f[k] = dalloc(s, 9 * P * ss));
        ok = ok && (d.reg_count[k] = (int *)dalloc(s, ntiles * 4));
        ok = ok && (d.reg_solids[k] = (int *)dalloc(s, ntiles * KMAX * 4));
        ok = ok && (d.reg_active[k] = (int *)dalloc(s, ntiles * 4));
        ok = ok && (d.reg_nactive[k] = (int *)dalloc(s, 16));
        ok = ok && (d.pool[k] = dalloc(s, ntiles * POOL_STRIDE * rs));
        ok = ok && (d.busy[k] = (unsigned char *)dalloc(s, nregions));
    }
    ok = ok && (d.carry = dalloc(s, P * ss));
    ok = ok && (d.fbody = dalloc(s, (size_t)c.ny * rs));
    if (c.force_kind == LBRMT_FORCE_FIELD) ok = ok && (d.bfield = dalloc(s, 2 * P * rs));
    ok = ok && (d.mass_partials = (double *)dalloc(s, nparts * 8));
    ok = ok && (d.err = (unsigned *)dalloc(s, 16));
    ok = ok && (d.lamtab = (LamEntry *)dalloc(s, (size_t)(2 * sp.lam_k0 + 1) * sizeof(LamEntry)));
    ok = ok && (s->scratch = (double *)dalloc(s, 128));  // one solid's statistics or the total mass
    // side stream (lowest priority) and fork / join events of the overlapped step
    if (ok) {
        int least = 0, greatest = 0;
        ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
             cudaStreamCreateWithPriority(&s->li.side, cudaStreamNonBlocking, least) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->li.fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->li.join, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->li.flags, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->li.done[0], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->li.done[1], cudaEventDisableTiming) == cudaSuccess;
        s->li.prio_hi = greatest;
    }
    if (!ok) {
        release_streams(s);
        dfree_all(s);
        delete s;
        return LBRMT_ERR_CUDA;
    }
    cudaStream_t st = s->stream;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
        e = cudaMemsetAsync(d.reg_count[k], 0, ntiles * 4, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(d.reg_nactive[k], 0, 16, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(d.pool[k], 0, ntiles * POOL_STRIDE * rs, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d.err, 0, 16, st);
    if (e == cudaSuccess && d.bfield) e = cudaMemsetAsync(d.bfield, 0, 2 * P * rs, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.mass_partials, 0, nparts * 8, st);
    // body force per row (x component), Sec. 4 forcing on all phases
    std::vector<double> fb(c.ny, 0.0);
    for (int j = 0; j < c.ny; j++) {
        if (c.force_kind == LBRMT_FORCE_CONST) fb[j] = c.force_a[0];
        else if (c.force_kind == LBRMT_FORCE_SINE_X) fb[j] = c.force_a[0] * std::sin(2.0 * M_PI * j / c.ny);
    }
    // solid-fraction table lambda = 1 - H_eps (Eq. 2_3_heaviside) with its Taylor
    // coefficients on phi_k = (k - k0) h, from the formula in double
    if (e == cudaSuccess) {
        const int n = 2 * sp.lam_k0 + 1;
        std::vector<LamEntry> tab(n);
        const double eps = c.eps, pi = M_PI;
        for (int k = 0; k < n; k++) {
            const double t = (double)(k - sp.lam_k0) * (double)sp.lam_h / eps;
            const double sn = std::sin(pi * t), cs = std::cos(pi * t);
            // lambda = 1 - (1 + t + sin(pi t)/pi)/2; for k >= 2 its k-th derivative in phi is
            // -(pi^(k-1) / (2 eps^k)) sin^(k-1)(pi t), with sin^(m) the m-th derivative of sin
            const double lam = 1.0 - 0.5 * (1.0 + t + sn / pi);
            const double l1 = -0.5 * (1.0 + cs) / eps;
            const double dsin[6] = {sn, cs, -sn, -cs, sn, cs};  // the m-th derivative of sin at pi t
            double lk[6] = {lam, l1, 0, 0, 0, 0}, fact = 1.0;
            for (int m = 2; m <= 5; m++) {
                fact *= m;
                lk[m] = -std::pow(pi, m - 1) / (2.0 * std::pow(eps, m)) * dsin[m] / fact;
            }
            LamEntry &q = tab[k];
            q.l0h = (float)lam; q.l0l = (float)(lam - (double)q.l0h);
            q.l1h = (float)l1; q.l1l = (float)(l1 - (double)q.l1h);
            q.l2 = (float)lk[2]; q.l3 = (float)lk[3]; q.l4 = (float)lk[4]; q.l5 = (float)lk[5];
        }
        e = cudaMemcpy(d.lamtab, tab.data(), n * sizeof(LamEntry), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        if (rs == 4) {
            std::vector<float> f32(fb.begin(), fb.end());
            e = cudaMemcpy(d.fbody, f32.data(), c.ny * 4, cudaMemcpyHostToDevice);
        } else {
            e = cudaMemcpy(d.fbody, fb.data(), c.ny * 8, cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) {
        dfree_all(s);
        delete s;
        return LBRMT_ERR_CUDA;
    }
    *out = s;
    return LBRMT_OK;
}

extern "C" lbrmt_status lbrmt_add_solid_shape(lbrmt_sim *s, int shape, double cx, double cy, double a, double b,
                                              double rho_s, double G, int *id_out) {
    if (!s) return LBRMT_ERR_ARG;
    if (s->inited) return fail(s, LBRMT_ERR_STATE, "solids must be added before the first step");
    if (shape < LBRMT_SHAPE_DISK || shape > LBRMT_SHAPE_RECT) return fail(s, LBRMT_ERR_ARG, "unknown shape");
    if (shape == LBRMT_SHAPE_DISK) b = a;
    if (!(a >= 1.0) || !(b >= 1.0) || !(rho_s > 0) || !(G >= 0) || !std::isfinite(cx) || !std::isfinite(cy))
        return fail(s, LBRMT_ERR_ARG, "bad solid parameters");
    // Appendix A: the solid's shear wave speed sqrt(G / rho_s) must not exceed one node per step
    if (G > rho_s) return fail(s, LBRMT_ERR_PARAM_RANGE, "shear wave speed sqrt(G/rho_s) above the lattice speed");
    const double radius = shape == LBRMT_SHAPE_DISK ? a : shape == LBRMT_SHAPE_ELLIPSE ? std::max(a, b) : std::hypot(a, b);
    const int margin = 4 + (int)std::ceil(radius * s->cfg.deform_margin);
    int T = 2 * (int)std::ceil(radius) + 2 * (s->cfg.n_layers + margin) + 1;
    T = (T + 7) & ~7;
    if (T > TILE_SIDE_MAX) return fail(s, LBRMT_ERR_ARG, "solid too large for a tile");
    if ((!s->cfg.bc_x && T >= s->cfg.nx) || (!s->cfg.bc_y && T >= s->cfg.ny))
        return fail(s, LBRMT_ERR_ARG, "solid tile wider than the periodic domain");
    SolidHost h{cx, cy, radius, rho_s, G, shape, a, b, T, 0};
    s->solids.push_back(h);
    if (id_out) *id_out = (int)s->solids.size() - 1;
    return LBRMT_OK;
}

extern "C" lbrmt_status lbrmt_add_solid(lbrmt_sim *s, int shape, double cx, double cy, double radius,
                                        double rho_s, double G, int *id_out) {
    if (s && shape != LBRMT_SHAPE_DISK) return fail(s, LBRMT_ERR_ARG, "lbrmt_add_solid adds disks; use lbrmt_add_solid_shape");
    return lbrmt_add_solid_shape(s, LBRMT_SHAPE_DISK, cx, cy, radius, radius, rho_s, G, id_out);
}

static lbrmt_status check_flags(lbrmt_sim *s) {
    unsigned h[4] = {0, 0, 0, 0};
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "stream");
    e = cudaMemcpy(h, s->d.err, 16, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "error flags");
    const unsigned f = h[0];
    if (!f) return LBRMT_OK;
    if (f & ERR_NAN) return fail(s, LBRMT_ERR_NUMERIC, "non-finite density or velocity");
    if (f & ERR_SLOT_OVERFLOW) return fail(s, LBRMT_ERR_OVERFLOW, "more solids on a tile than max_solids_per_tile");
    if (f & ERR_TILE_OVERFLOW) return fail(s, LBRMT_ERR_OVERFLOW, "a solid's band outgrew its tile");
    if (f & ERR_EXTRAP) return fail(s, LBRMT_ERR_EXTRAP, "extrapolation window exceeded rmax");
    if (f & ERR_STENCIL) return fail(s, LBRMT_ERR_EXTRAP, "advection stencil left the band");
    if (f & ERR_SINGULAR) return fail(s, LBRMT_ERR_NUMERIC, "singular reference-map Jacobian");
    if (f & ERR_OVERFLOW16) return fail(s, LBRMT_ERR_OVERFLOW, "a population exceeded the 16-bit storage range");
    if (f & ERR_TIMEOUT) return fail(s, LBRMT_ERR_TIMEOUT, "a bounded wait on a tensor copy gave up");
    if (f & ERR_ALIGN) return fail(s, LBRMT_ERR_CUDA, "misaligned shared-memory stage (tensor copies skipped)");
    if (f & ERR_FREE_REGION)
        return fail(s, LBRMT_ERR_NUMERIC, "an interface moved more than one node in a step (a region stepped as solid-free held a solid)");
    return fail(s, LBRMT_ERR_NUMERIC, "device error flag");
}

lbrmt_status lbrmt_internal_check_flags(lbrmt_sim *s) { return check_flags(s); }
void *lbrmt_internal_alloc(lbrmt_sim *s, size_t bytes) { return dalloc(s, bytes); }
lbrmt_status lbrmt_internal_fail(lbrmt_sim *s, lbrmt_status st, const std::string &msg) { return fail(s, st, msg); }

// Solid descriptors and initial frames from the host solids; configure and run
// the initialisation kernels (Algorithm 1, initialisation) on the allocated state.
// Power-of-two storage scales of the 16-bit variants, per population plane and
// for the density plane, from bounds of the stored values: with the
// velocity bounded by U = 0.3 (above the Mach limit of Appendix A), the density
// difference D = max |rho_s - rho_f|, a pressure deviation of 0.1 rho_f and
// rho_max = rho_f + D + 0.1 rho_f, a stored deviation of plane q is below
// w_q (0.1 rho_f + D + rho_max (3 sqrt2 U + 10.5 U^2)) (q >= 1), w_0 (0.1 rho_f + D
// + 1.5 rho_max U^2) (the rest plane, relative to Delta rho), and the density
// plane rho - rho_f below 0.1 rho_f + D.  Each bound is mapped
// below 2^15 (FP16's largest value is 65504).  FP32 / FP64 storage: scale 1.
static void set_store_scales(lbrmt_sim *s) {
    SimParams &sp = s->sp;
    for (int q = 0; q < 9; q++) sp.st_scale[q] = sp.st_inv[q] = 1.0f;
    sp.ct_scale = sp.ct_inv = 1.0f;
    if (s->eng->store_size != 2) return;
    const lbrmt_config &c = s->cfg;
    double D = 0.0;
    for (const SolidHost &h : s->solids) D = std::max(D, std::fabs(h.rho_s - c.rho_f));
    const double U = 0.3, rmax = c.rho_f * 1.1 + D;
    auto scale_for = [](double bound) {
        int k = (int)std::floor(std::log2(32768.0 / bound));
        k = std::max(0, std::min(k, 24));
        return (float)std::ldexp(1.0, k);
    };
    for (int q = 0; q < 9; q++) {
        const double w = q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        const double b = q == 0 ? w * (0.1 * c.rho_f + D + 1.5 * rmax * U * U)
                                : w * (0.1 * c.rho_f + D + rmax * (3.0 * std::sqrt(2.0) * U + 10.5 * U * U));
        sp.st_scale[q] = scale_for(b);
        sp.st_inv[q] = 1.0f / sp.st_scale[q];
    }
    sp.ct_scale = scale_for(0.1 * c.rho_f + D);
    sp.ct_inv = 1.0f / sp.ct_scale;
}

// After the solids' materials changed (a checkpoint's adopted): new scales, and
// the captured graphs (whose launch arguments carry them) are dropped.
void lbrmt_internal_refresh_scales(lbrmt_sim *s) {
    const SimParams old = s->sp;
    set_store_scales(s);
    if (std::memcmp(old.st_scale, s->sp.st_scale, sizeof(old.st_scale)) != 0 || old.ct_scale != s->sp.ct_scale) {
        if (s->stream) cudaStreamSynchronize(s->stream);
        drop_graphs(s);
    }
}

static lbrmt_status run_init(lbrmt_sim *s) {
    const int S = (int)s->solids.size();
    DevState &d = s->d;
    set_store_scales(s);
    int tmax = 8;
    for (auto &h : s->solids) tmax = std::max(tmax, h.T);
    std::vector<SolidDesc> sd(S);
    std::vector<Frame> org(S);
    for (int k = 0; k < S; k++) {
        const SolidHost &h = s->solids[k];
        // initial frame: centred on the solid, off = o - X_c on the 2^-14 grid (d = o - X_c - off)
        org[k].ox = (int)std::floor(h.xc) - h.T / 2;
        org[k].oy = (int)std::floor(h.yc) - h.T / 2;
        org[k].offx = (float)(std::rint(((double)org[k].ox - h.xc) * 16384.0) / 16384.0);
        org[k].offy = (float)(std::rint(((double)org[k].oy - h.yc) * 16384.0) / 16384.0);
        org[k].bx0 = org[k].by0 = 1; org[k].bx1 = org[k].by1 = 0;  // empty until initialised
        sd[k].xc = h.xc; sd[k].yc = h.yc; sd[k].R = h.R; sd[k].rho_s = h.rho_s; sd[k].G = h.G;
        sd[k].shape = h.shape; sd[k].a = h.a; sd[k].b = h.b; sd[k].eps = s->cfg.eps;
        sd[k].drho = h.rho_s - s->cfg.rho_f;
        sd[k].accel = -(1.0 - s->cfg.rho_f / h.rho_s) * s->cfg.gravity;
        const double r2 = h.R * h.R;
        sd[k].R_f = (float)h.R; sd[k].G_f = (float)h.G; sd[k].Rlo_f = (float)(h.R - (double)sd[k].R_f);
        sd[k].r2hi_f = (float)r2; sd[k].r2lo_f = (float)(r2 - (double)sd[k].r2hi_f); sd[k].r2lo = 0.0;
        sd[k].drho_f = (float)sd[k].drho; sd[k].accel_f = (float)sd[k].accel;
        sd[k].drho_lo_f = (float)(sd[k].drho - (double)sd[k].drho_f);
        sd[k].T = h.T; sd[k].off = h.off;
    }
    // solid kernel launch order: largest tiles first, so the last CTAs to start are short
    std::vector<int> order(S);
    for (int k = 0; k < S; k++) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return s->solids[a].T > s->solids[b].T; });
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess && S > 0) {
        e = cudaMemcpy(d.order, order.data(), S * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d.solids, sd.data(), S * sizeof(SolidDesc), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d.frame[0], org.data(), S * sizeof(Frame), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d.frame[1], org.data(), S * sizeof(Frame), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemsetAsync(d.stats_step, 0, (size_t)S * 64, s->stream);
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "upload solids");
    const bool use_tma = s->li.use_tma;
    e = s->eng->configure(s->sp, d, tmax, &s->li);
    s->li.use_tma = use_tma;
    if (e != cudaSuccess) return cuda_fail(s, e, "configure kernels");
    // both registries start empty; the initialisation registers into registry 1
    // (step 0 reads its Delta rho as the rest base of f^0 and clears it) and
    // step 0 registers into registry 0
    const size_t ntiles = (size_t)s->sp.ntx * s->sp.nty;
    for (int k = 0; k < 2 && e == cudaSuccess; k++) {
        e = cudaMemsetAsync(d.reg_count[k], 0, ntiles * 4, s->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(d.reg_nactive[k], 0, 16, s->stream);
    }
    // the pools' half-force planes of the initial registry must read zero (the
    // density plane is marked "no collision yet" by the initialisation kernel)
    const size_t rsz = s->eng->real_size;
    for (int k = 0; k < 2 && e == cudaSuccess; k++)
        e = cudaMemsetAsync(d.pool[k], 0, ntiles * POOL_STRIDE * rsz, s->stream);
    // the slots a tile shape's K1 does not write must hold zero (a previous shape may have written them)
    if (e == cudaSuccess) e = cudaMemsetAsync(d.mass_partials, 0, (size_t)s->mass_parts_cap * 8, s->stream);
    // every region counts as busy for the first step's check of the previous classification
    for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaMemsetAsync(d.busy[k], 1, (size_t)s->nregions_cap, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.err, 0, 16, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "clear registry");
    e = s->eng->init(s->sp, d, s->li, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "init kernels");
    e = cudaMemsetAsync(d.reg_count[0], 0, ntiles * 4, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.reg_nactive[0], 0, 16, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "clear registry");
    s->inited = true;
    s->steps = 0;
    return check_flags(s);
}

extern "C" lbrmt_status lbrmt_init(lbrmt_sim *s) {
    if (!s) return LBRMT_ERR_ARG;
    if (s->inited) return LBRMT_OK;
    const int S = (int)s->solids.size();
    s->sp.nsolids = S;
    DevState &d = s->d;
    long long total = 0;
    const long long planes = s->eng->real_size == 4 ? xi_planes<float>() : xi_planes<double>();
    for (auto &h : s->solids) {
        h.off = total;
        total += planes * h.T * h.T;  // eta_x, eta_y, phi (and in FP32 the low parts of eta)
    }
    s->xi_total = total;
    const size_t rs = s->eng->real_size;
    bool ok = true;
    for (int k = 0; k < 2; k++) {
        ok = ok && (d.xi[k] = dalloc(s, (size_t)total * rs));
        ok = ok && (d.frame[k] = (Frame *)dalloc(s, (size_t)S * sizeof(Frame)));
    }
    ok = ok && (d.solids = (SolidDesc *)dalloc(s, (size_t)S * sizeof(SolidDesc)));
    ok = ok && (d.order = (int *)dalloc(s, (size_t)std::max(S, 1) * sizeof(int)));
    ok = ok && (d.stats_step = (double *)dalloc(s, (size_t)S * 64));
    if ((size_t)S * STATS_COLS * 8 > 128) {
        double *sc = (double *)dalloc(s, (size_t)S * STATS_COLS * 8);
        ok = ok && sc;
        s->scratch = sc;
    }
    if (!ok) return fail(s, LBRMT_ERR_CUDA, "out of device memory for the solid tiles");
    return run_init(s);
}

extern "C" lbrmt_status lbrmt_reset(lbrmt_sim *s) {
    if (!s) return LBRMT_ERR_ARG;
    if (s->in_batch) return fail(s, LBRMT_ERR_STATE, "a batch member is stepped by its batch");
    if (!s->inited) return lbrmt_init(s);
    drop_graphs(s);
    return run_init(s);
}

static void set_tile_shape(lbrmt_sim *s, int tx) {
    SimParams &sp = s->sp;
    s->cfg.tile_x = tx;
    set_tile_params(sp, tx);
}

extern "C" lbrmt_status lbrmt_set_tile_x(lbrmt_sim *s, int tile_x) {
    if (!s) return LBRMT_ERR_ARG;
    if (tile_x == 0) tile_x = 32;
    if (tile_x != 16 && tile_x != 32 && tile_x != 64 && tile_x != 128) return fail(s, LBRMT_ERR_ARG, "tile_x must be 16, 32, 64 or 128");
    if (s->in_batch) return fail(s, LBRMT_ERR_STATE, "a batch member's tile shape is set by its batch");
    if (s->stream) cudaStreamSynchronize(s->stream);
    drop_graphs(s);
    if (s->adj) lbrmt_internal_adjoint_free(s);  // its recording buffers are sized by the tile count
    set_tile_shape(s, tile_x);
    if (!s->inited) return LBRMT_OK;
    return run_init(s);
}

extern "C" int lbrmt_tile_x(const lbrmt_sim *s) { return s ? s->sp.tx : 0; }

extern "C" lbrmt_status lbrmt_autotune_tile(lbrmt_sim *s, int steps, int *best_tile_x, int *best_tma, double *ms_out) {
    if (!s || steps < 1) return LBRMT_ERR_ARG;
    const int cand[4] = {16, 32, 64, 128};
    int best = s->sp.tx, best_t = s->li.use_tma ? 1 : 0;
    double best_ms = 1e30;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(s, LBRMT_ERR_CUDA, "event create");
    lbrmt_status st = LBRMT_OK;
    for (int k = 0; k < 8 && st == LBRMT_OK; k++) {
        const int tx = cand[k >> 1], tma = (k & 1) ? 0 : 1;
        double ms = 1e30;
        s->li.use_tma = tma != 0;
        st = lbrmt_set_tile_x(s, tx);
        if (st == LBRMT_OK && !s->inited) st = lbrmt_init(s);
        const bool runs = st == LBRMT_OK && (tma == 0 || s->li.tma);  // the tensor path may not apply
        if (runs) st = lbrmt_step(s, 4);  // warm-up (graph capture)
        for (int rep = 0; rep < 2 && runs && st == LBRMT_OK; rep++) {
            cudaEventRecord(e0, s->stream);
            st = lbrmt_step(s, steps);
            cudaEventRecord(e1, s->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(s, LBRMT_ERR_CUDA, "autotune");
            float f = 0.f;
            cudaEventElapsedTime(&f, e0, e1);
            ms = std::min(ms, (double)f / steps);
        }
        if (st == LBRMT_OK && runs) st = check_flags(s);
        if (ms_out) ms_out[k] = runs ? ms : -1.0;
        if (st == LBRMT_OK && runs && ms < best_ms) {
            best_ms = ms;
            best = tx;
            best_t = tma;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LBRMT_OK) return st;
    if (best_tile_x) *best_tile_x = best;
    if (best_tma) *best_tma = best_t;
    s->li.use_tma = best_t != 0;
    return lbrmt_set_tile_x(s, best);  // back to the initial state with the chosen variant
}

extern "C" lbrmt_status lbrmt_set_solid_params(lbrmt_sim *s, int solid_id, double rho_s, double G) {
    if (!s || solid_id < 0 || solid_id >= (int)s->solids.size()) return LBRMT_ERR_ARG;
    if (!(rho_s > 0) || !(G >= 0)) return fail(s, LBRMT_ERR_ARG, "bad solid parameters");
    s->solids[solid_id].rho_s = rho_s;
    s->solids[solid_id].G = G;
    if (!s->inited) return LBRMT_OK;
    return lbrmt_reset(s);
}

namespace lbrmt {
template <class R>
__global__ void body_field_kernel(const double *src, R *dst, long long n) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        dst[k] = R(src[k]);
}
}  // namespace lbrmt

extern "C" lbrmt_status lbrmt_set_body_force_field(lbrmt_sim *s, int sim_index, const double *dev_xy) {
    if (!s || !dev_xy || sim_index != 0) return LBRMT_ERR_ARG;
    if (s->cfg.force_kind != LBRMT_FORCE_FIELD) return fail(s, LBRMT_ERR_STATE, "force_kind is not LBRMT_FORCE_FIELD");
    const long long n = 2 * s->sp.P;
    if (s->eng->real_size == 8) body_field_kernel<double><<<256, 256, 0, s->stream>>>(dev_xy, (double *)s->d.bfield, n);
    else body_field_kernel<float><<<256, 256, 0, s->stream>>>(dev_xy, (float *)s->d.bfield, n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(s, e, "body force field");
    return LBRMT_OK;
}

static lbrmt_status direct_step(lbrmt_sim *s) {
    cudaError_t e = s->eng->step(s->sp, s->d, s->li, (int)(s->steps & 1), s->stream, nullptr, nullptr, CHAIN_ONE);
    if (e != cudaSuccess) return cuda_fail(s, e, "step launch");
    s->steps++;
    s->last_launches += step_launches(s->sp, s->li);
    return LBRMT_OK;
}

// Capture nsteps (even) steps from an even step count as one graph; the steps
// form one chain of the overlapped schedule.
static lbrmt_status build_graph(lbrmt_sim *s, int nsteps, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(s, e, "begin capture");
    cudaError_t es = cudaSuccess;
    for (int k = 0; k < nsteps; k++) {
        const int chain = (k == 0 ? CHAIN_FIRST : 0) | (k == nsteps - 1 ? CHAIN_LAST : 0);
        cudaError_t ek = s->eng->step(s->sp, s->d, s->li, k & 1, s->stream, nullptr, nullptr, chain);
        if (ek != cudaSuccess && es == cudaSuccess) es = ek;
    }
    e = cudaStreamEndCapture(s->stream, &g);
    if (es != cudaSuccess) e = es;
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(s, e, "capture");
    }
    // per-node priorities: the overlapped step runs K2, K3 and the busy K1 ahead of the free K1
    e = cudaGraphInstantiate(out, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *out = nullptr;
        return cuda_fail(s, e, "instantiate graph");
    }
    return LBRMT_OK;
}

extern "C" lbrmt_status lbrmt_step(lbrmt_sim *s, int nsteps) {
    if (!s || nsteps < 0) return LBRMT_ERR_ARG;
    if (s->in_batch) return fail(s, LBRMT_ERR_STATE, "a batch member is stepped by its batch");
    if (!s->inited) {
        lbrmt_status st = lbrmt_init(s);
        if (st != LBRMT_OK) return st;
    }
    s->last_launches = 0;
    int left = nsteps;
    const bool graphs = s->use_graphs && s->stream != nullptr && nsteps >= 2;
    if (graphs) {
        if (s->steps & 1) {
            lbrmt_status st = direct_step(s);
            if (st != LBRMT_OK) return st;
            left--;
        }
        if (left >= GRAPH_LONG && !s->gexec_long) {
            lbrmt_status st = build_graph(s, GRAPH_LONG, &s->gexec_long);
            if (st != LBRMT_OK) return st;
        }
        while (left >= GRAPH_LONG) {
            cudaError_t e = cudaGraphLaunch(s->gexec_long, s->stream);
            if (e != cudaSuccess) return cuda_fail(s, e, "graph launch");
            s->steps += GRAPH_LONG;
            s->last_launches += GRAPH_LONG * step_launches(s->sp, s->li);
            left -= GRAPH_LONG;
        }
        if (left >= 2 && !s->gexec) {
            lbrmt_status st = build_graph(s, 2, &s->gexec);
            if (st != LBRMT_OK) return st;
        }
        while (left >= 2) {
            cudaError_t e = cudaGraphLaunch(s->gexec, s->stream);
            if (e != cudaSuccess) return cuda_fail(s, e, "graph launch");
            s->steps += 2;
            s->last_launches += 2 * step_launches(s->sp, s->li);
            left -= 2;
        }
    }
    while (left > 0) {
        lbrmt_status st = direct_step(s);
        if (st != LBRMT_OK) return st;
        left--;
    }
    return LBRMT_OK;
}

extern "C" lbrmt_status lbrmt_step_timed(lbrmt_sim *s, int nsteps, float *ms_out) {
    if (!s || nsteps < 1 || !ms_out) return LBRMT_ERR_ARG;
    if (s->in_batch) return fail(s, LBRMT_ERR_STATE, "a batch member is stepped by its batch");
    if (!s->inited) {
        lbrmt_status st = lbrmt_init(s);
        if (st != LBRMT_OK) return st;
    }
    std::vector<cudaEvent_t> ev(4 * (size_t)nsteps, nullptr);
    for (auto &e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(s, LBRMT_ERR_CUDA, "event create");
    s->last_launches = 0;
    lbrmt_status status = LBRMT_OK;
    for (int n = 0; n < nsteps; n++) {
        cudaError_t e = s->eng->step(s->sp, s->d, s->li, (int)(s->steps & 1), s->stream, &ev[4 * (size_t)n], nullptr,
                                     CHAIN_ONE);
        if (e != cudaSuccess) { status = cuda_fail(s, e, "timed step"); break; }
        s->steps++;
        s->last_launches += step_launches(s->sp, s->li, true);
    }
    double acc[3] = {0, 0, 0};
    if (status == LBRMT_OK) {
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) status = cuda_fail(s, e, "timed sync");
        for (int n = 0; n < nsteps && status == LBRMT_OK; n++)
            for (int k = 0; k < 3; k++) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[4 * (size_t)n + k], ev[4 * (size_t)n + k + 1]);
                acc[k] += ms;
            }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    for (int k = 0; k < 3; k++) ms_out[k] = (float)(acc[k] / nsteps);
    if (status != LBRMT_OK) return status;
    return check_flags(s);
}

static bool field_ok(int f) { return (f >= 0 && f <= 5) || (f >= 10 && f <= 12) || f == 14 || f == 15 || (f >= 20 && f < 29); }

extern "C" lbrmt_status lbrmt_read_fields(lbrmt_sim *s, int sim_index, int field, int solid_id, double *dev_out) {
    if (!s || !dev_out || sim_index != 0 || !field_ok(field)) return LBRMT_ERR_ARG;
    if (!s->inited) {
        lbrmt_status st = lbrmt_init(s);
        if (st != LBRMT_OK) return st;
    }
    const int cur = (int)(s->steps & 1);
    const int lastreg = 1 - cur;  // registry of the step (or initialisation) that wrote the state
    if (field >= 10 && field <= 15) {
        if (solid_id < 0 || solid_id >= (int)s->solids.size()) return fail(s, LBRMT_ERR_ARG, "bad solid id");
        cudaError_t e = cudaMemsetAsync(dev_out, 0xFF, (size_t)s->sp.P * 8, s->stream);  // NaN
        if (e != cudaSuccess) return cuda_fail(s, e, "clear field");
    }
    cudaError_t e = s->eng->field(s->sp, s->d, cur, lastreg, field, solid_id, dev_out, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "field kernel");
    return LBRMT_OK;
}

// Device address of a page-locked (or registered) host buffer, which kernels
// read and write directly over the coherent CPU-GPU link; null for pageable
// memory, which goes through a device staging buffer and a copy instead.
static void *mapped_view(const void *host) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
        cudaGetLastError();  // not an error of the simulation
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

extern "C" lbrmt_status lbrmt_read_fields_host(lbrmt_sim *s, int sim_index, int field, int solid_id,
                                               double *host_out) {
    if (!s || !host_out) return LBRMT_ERR_ARG;
    // fields written at every node go straight into a page-locked buffer
    // (the per-solid fields are cleared first and written on the band only)
    if (void *dv = (field < 10 || field >= 20) ? mapped_view(host_out) : nullptr) {
        lbrmt_status st = lbrmt_read_fields(s, sim_index, field, solid_id, (double *)dv);
        if (st != LBRMT_OK) return st;
        return check_flags(s);
    }
    if (!s->staging) {
        s->staging = (double *)dalloc(s, (size_t)9 * s->sp.P * 8);
        if (!s->staging) return fail(s, LBRMT_ERR_CUDA, "out of device memory");
    }
    lbrmt_status st = lbrmt_read_fields(s, sim_index, field, solid_id, s->staging);
    if (st != LBRMT_OK) return st;
    cudaError_t e = cudaMemcpyAsync(host_out, s->staging, (size_t)s->sp.P * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "copy field");
    return check_flags(s);
}

extern "C" lbrmt_status lbrmt_set_populations_host(lbrmt_sim *s, const double *host_f) {
    if (!s || !host_f) return LBRMT_ERR_ARG;
    if (!s->inited) {
        lbrmt_status st = lbrmt_init(s);
        if (st != LBRMT_OK) return st;
    }
    // a page-locked buffer is read by the conversion kernel directly
    const double *src = (const double *)mapped_view(host_f);
    cudaError_t e = cudaSuccess;
    if (!src) {
        if (!s->staging) {
            s->staging = (double *)dalloc(s, (size_t)9 * s->sp.P * 8);
            if (!s->staging) return fail(s, LBRMT_ERR_CUDA, "out of device memory");
        }
        e = cudaMemcpyAsync(s->staging, host_f, (size_t)9 * s->sp.P * 8, cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "copy populations");
        src = s->staging;
    }
    e = s->eng->set_pop(s->sp, s->d, (int)(s->steps & 1), src, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "set populations");
    return check_flags(s);
}

extern "C" lbrmt_status lbrmt_solid_stats(lbrmt_sim *s, int sim_index, double *host_out) {
    if (!s || !host_out || sim_index != 0) return LBRMT_ERR_ARG;
    if (!s->inited) {
        lbrmt_status st = lbrmt_init(s);
        if (st != LBRMT_OK) return st;
    }
    const int S = (int)s->solids.size();
    if (S == 0) return LBRMT_OK;
    cudaError_t e = s->eng->stats(s->sp, s->d, (int)(s->steps & 1), s->scratch, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "stats kernel");
    e = cudaMemcpyAsync(host_out, s->scratch, (size_t)S * STATS_COLS * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "copy stats");
    return check_flags(s);
}

extern "C" lbrmt_status lbrmt_solid_stats_async(lbrmt_sim *s, int sim_index, double *host_out) {
    if (!s || !host_out || sim_index != 0) return LBRMT_ERR_ARG;
    if (!s->inited) return fail(s, LBRMT_ERR_STATE, "not initialised");
    const int S = (int)s->solids.size();
    if (S == 0) return LBRMT_OK;
    if (double *dv = (double *)mapped_view(host_out)) {  // page-locked: the kernel writes it
        cudaError_t e = s->eng->stats(s->sp, s->d, (int)(s->steps & 1), dv, s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "stats kernel");
        return LBRMT_OK;
    }
    cudaError_t e = s->eng->stats(s->sp, s->d, (int)(s->steps & 1), s->scratch, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "stats kernel");
    e = cudaMemcpyAsync(host_out, s->scratch, (size_t)S * STATS_COLS * 8, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "copy stats");
    return LBRMT_OK;
}

extern "C" lbrmt_status lbrmt_total_mass(lbrmt_sim *s, int sim_index, double *host_out) {
    if (!s || !host_out || sim_index != 0) return LBRMT_ERR_ARG;
    if (!s->inited) return fail(s, LBRMT_ERR_STATE, "the simulation is not initialised (lbrmt_init)");
    const int cur = (int)(s->steps & 1);
    cudaError_t e = s->eng->mass(s->sp, s->d, cur, s->stream);
    if (e == cudaSuccess) {
        mass_reduce_kernel<<<1, 1024, 0, s->stream>>>(s->d.mass_partials, s->sp.ntx * s->sp.nty,
                                                      s->sp.rho_f * (double)s->sp.P, s->scratch);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "mass kernel");
    e = cudaMemcpyAsync(host_out, s->scratch, 8, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "copy mass");
    return check_flags(s);
}

extern "C" lbrmt_status lbrmt_active_tiles(lbrmt_sim *s, int sim_index, long long *host_out) {
    if (!s || !host_out || sim_index != 0) return LBRMT_ERR_ARG;
    *host_out = 0;
    if (s->steps == 0 || s->sp.nsolids == 0) return LBRMT_OK;
    const int r = 1 - (int)(s->steps & 1);
    int n = 0;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&n, s->d.reg_nactive[r], 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(s, e, "active tiles");
    *host_out = n;
    return LBRMT_OK;
}

extern "C" lbrmt_status lbrmt_sync(lbrmt_sim *s) {
    if (!s) return LBRMT_ERR_ARG;
    return check_flags(s);
}

extern "C" long long lbrmt_steps_done(const lbrmt_sim *s) { return s ? s->steps : -1; }
extern "C" int lbrmt_num_solids(const lbrmt_sim *s) { return s ? (int)s->solids.size() : -1; }
extern "C" long long lbrmt_last_launch_count(const lbrmt_sim *s) { return s ? s->last_launches : -1; }

extern "C" lbrmt_status lbrmt_set_use_graphs(lbrmt_sim *s, int enable) {
    if (!s) return LBRMT_ERR_ARG;
    s->use_graphs = enable != 0;
    return LBRMT_OK;
}

extern "C" lbrmt_status lbrmt_set_use_tma(lbrmt_sim *s, int enable) {
    if (!s) return LBRMT_ERR_ARG;
    s->li.use_tma = enable != 0;
    if (s->gexec || s->gexec_long) {
        cudaStreamSynchronize(s->stream);
        drop_graphs(s);
    }
    return LBRMT_OK;
}

extern "C" int lbrmt_uses_tma(const lbrmt_sim *s) { return s && s->inited && s->li.tma && s->li.use_tma ? 1 : 0; }

extern "C" const char *lbrmt_last_error(const lbrmt_sim *s) { return s ? s->err.c_str() : "null handle"; }

extern "C" lbrmt_status lbrmt_set_overlap(lbrmt_sim *s, int enable) {
    if (!s) return LBRMT_ERR_ARG;
    if (s->in_batch) return fail(s, LBRMT_ERR_STATE, "a batch member is stepped by its batch");
    if (s->stream) cudaStreamSynchronize(s->stream);
    s->li.split = enable != 0;
    drop_graphs(s);
    return LBRMT_OK;
}

extern "C" int lbrmt_uses_overlap(const lbrmt_sim *s) { return s && s->inited && step_overlaps(s->sp, s->li) ? 1 : 0; }

extern "C" lbrmt_status lbrmt_set_rmt_threads(lbrmt_sim *s, int threads) {
    if (!s) return LBRMT_ERR_ARG;
    if (threads != 0 && threads != RMT_THREADS && threads != RMT_THREADS_BIG)
        return fail(s, LBRMT_ERR_ARG, "reference-map CTA width must be 0, 256 or 1024");
    if (s->in_batch) return fail(s, LBRMT_ERR_STATE, "a batch member is stepped by its batch");
    if (s->stream) cudaStreamSynchronize(s->stream);
    s->li.rmt_req = threads;
    if (s->inited) {  // choose again (configure keeps the tensor-memory choice)
        const bool use_tma = s->li.use_tma;
        cudaError_t e = s->eng->configure(s->sp, s->d, s->li.tmax, &s->li);
        s->li.use_tma = use_tma;
        if (e != cudaSuccess) return cuda_fail(s, e, "configure kernels");
    }
    drop_graphs(s);
    return LBRMT_OK;
}

extern "C" int lbrmt_rmt_threads(const lbrmt_sim *s) { return s && s->inited ? s->li.rmt_threads : 0; }

extern "C" lbrmt_status lbrmt_check_bounded_wait(lbrmt_sim *s) {
    if (!s) return LBRMT_ERR_ARG;
    lbrmt_status st = check_flags(s);  // a pending error is reported, not overwritten
    if (st != LBRMT_OK) return st;
    bounded_wait_check_kernel<<<1, 32, 0, s->stream>>>(s->d.err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(s, e, "bounded wait check");
    st = check_flags(s);
    e = cudaMemsetAsync(s->d.err, 0, 16, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "clear error flags");
    return st;
}

extern "C" void lbrmt_destroy(lbrmt_sim *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    if (s->li.side) cudaStreamSynchronize(s->li.side);
    drop_graphs(s);
    release_streams(s);
    if (s->adj) lbrmt_internal_adjoint_free(s);
    dfree_all(s);
    delete s;
}
