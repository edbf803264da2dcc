// lbrmt_checkpoint.cu -- checkpoint and resume of a simulation (lbrmt_save /
// lbrmt_load): the whole state that Algorithm 1 carries from step n to n+1.
//
// The state is every persistent device buffer of the simulation, both halves
// of each ping-pong pair: the populations f and the density plane of the
// last collision (with the pools' half-force planes, the term rho F / 2 of
// Sec. 3.4's moments), the reference-map tiles xi with the level-set
// plane and their frames (Sec. 3.1-3.2), the tile registries with the force
// pools of the last step (Sec. 3.3), the regions' busy flags of the overlapped
// schedule, the body-force rows or field, the per-solid descriptors and
// statistics, and the lattice Boltzmann kernel's mass partial sums.  Restoring
// all of them and the step counter makes the resumed run the same, bit for bit,
// as the run that was saved.
//
// Blob layout (a caller-owned device buffer): a fixed header, one record per
// solid, then the sections, each starting on a 256-byte boundary, in the order
// of sections().  The header fixes what must agree for the bytes to mean the
// same thing in the loading simulation: grid, walls, precision, the method's
// parameters, the tile shape and the solids' geometry and tile sides.

#include <cstdint>
#include <cstring>

#include "lbrmt_sim.cuh"

using namespace lbrmt;

namespace {

constexpr char CK_MAGIC[8] = {'L', 'B', 'R', 'M', 'T', 'C', 'K', '1'};
constexpr uint32_t CK_VERSION = 1;
constexpr int CK_MAX_SECTIONS = 40;
constexpr size_t CK_ALIGN = 256;

struct CkHeader {
    char magic[8];
    uint32_t version, nsections;
    uint64_t total_bytes, header_bytes;  // header_bytes: header + solid records, before alignment
    int32_t precision, nx, ny, bc_x, bc_y, force_kind, n_layers, rmax, kmax, tile_x, nsolids, pad0;
    int64_t steps, xi_total, ntiles_cap, mass_parts_cap, nregions_cap;
    double tau, rho_f, lid_u, eps, eta, gravity, fa0, fa1, deform_margin;
    uint64_t section_bytes[CK_MAX_SECTIONS];
};

struct CkSolid {
    int32_t shape, T;
    double xc, yc, R, a, b, rho_s, G;
};

struct Section {
    void *ptr;
    size_t bytes;
};

inline size_t align_up(size_t n) { return (n + CK_ALIGN - 1) & ~(CK_ALIGN - 1); }

// Every persistent buffer of the simulation with its allocated size.
int sections(const lbrmt_sim *s, Section *out) {
    const DevState &d = s->d;
    const size_t P = (size_t)s->sp.P, rs = s->eng->real_size, ss = s->eng->store_size;
    const size_t nt = (size_t)s->ntiles_cap, S = s->solids.size();
    int n = 0;
    auto add = [&](void *p, size_t b) {
        if (p && b > 0) out[n++] = {p, b};
    };
    for (int k = 0; k < 2; k++) {
        add(d.f[k], 9 * P * ss);
        add(d.reg_count[k], nt * 4);
        add(d.reg_solids[k], nt * KMAX * 4);
        add(d.reg_active[k], nt * 4);
        add(d.reg_nactive[k], 16);
        add(d.pool[k], nt * POOL_STRIDE * rs);
        add(d.busy[k], (size_t)s->nregions_cap);
        add(d.xi[k], (size_t)s->xi_total * rs);
        add(d.frame[k], S * sizeof(Frame));
    }
    add(d.carry, P * ss);
    add(d.fbody, (size_t)s->sp.ny * rs);
    if (s->cfg.force_kind == LBRMT_FORCE_FIELD) add(d.bfield, 2 * P * rs);
    add(d.mass_partials, (size_t)s->mass_parts_cap * 8);
    add(d.stats_step, S * 64);
    add(d.solids, S * sizeof(SolidDesc));
    add(d.order, S * sizeof(int));
    return n;
}

void fill_header(const lbrmt_sim *s, CkHeader &h, std::vector<CkSolid> &recs, const Section *sec, int nsec) {
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, CK_MAGIC, 8);
    h.version = CK_VERSION;
    h.nsections = (uint32_t)nsec;
    const lbrmt_config &c = s->cfg;
    h.precision = c.precision; h.nx = c.nx; h.ny = c.ny; h.bc_x = c.bc_x; h.bc_y = c.bc_y;
    h.force_kind = c.force_kind; h.n_layers = c.n_layers; h.rmax = c.rmax; h.kmax = c.max_solids_per_tile;
    h.tile_x = s->sp.tx; h.nsolids = (int32_t)s->solids.size();
    h.steps = s->steps; h.xi_total = s->xi_total;
    h.ntiles_cap = s->ntiles_cap; h.mass_parts_cap = s->mass_parts_cap; h.nregions_cap = s->nregions_cap;
    h.tau = c.tau; h.rho_f = c.rho_f; h.lid_u = c.lid_u; h.eps = c.eps; h.eta = c.eta; h.gravity = c.gravity;
    h.fa0 = c.force_a[0]; h.fa1 = c.force_a[1]; h.deform_margin = c.deform_margin;
    recs.resize(s->solids.size());
    for (size_t k = 0; k < recs.size(); k++) {
        const SolidHost &o = s->solids[k];
        recs[k] = {o.shape, o.T, o.xc, o.yc, o.R, o.a, o.b, o.rho_s, o.G};
    }
    h.header_bytes = sizeof(CkHeader) + recs.size() * sizeof(CkSolid);
    size_t total = align_up(h.header_bytes);
    for (int k = 0; k < nsec; k++) {
        h.section_bytes[k] = sec[k].bytes;
        total += align_up(sec[k].bytes);
    }
    h.total_bytes = total;
}

lbrmt_status mismatch(lbrmt_sim *s, const char *what) {
    return lbrmt_internal_fail(s, LBRMT_ERR_ARG, std::string("checkpoint does not match this simulation: ") + what);
}

}  // namespace

extern "C" lbrmt_status lbrmt_save(lbrmt_sim *s, void *dev_blob, size_t *bytes) {
    if (!s || !bytes) return LBRMT_ERR_ARG;
    if (s->in_batch) return lbrmt_internal_fail(s, LBRMT_ERR_STATE, "a batch member is saved with its batch");
    if (!s->inited) return lbrmt_internal_fail(s, LBRMT_ERR_STATE, "lbrmt_save needs an initialised simulation");
    Section sec[CK_MAX_SECTIONS];
    const int nsec = sections(s, sec);
    CkHeader h;
    std::vector<CkSolid> recs;
    fill_header(s, h, recs, sec, nsec);
    if (!dev_blob) {  // size query
        *bytes = (size_t)h.total_bytes;
        return LBRMT_OK;
    }
    if (*bytes < h.total_bytes) return lbrmt_internal_fail(s, LBRMT_ERR_ARG, "checkpoint buffer too small");
    // a state with a raised error flag is not worth resuming
    lbrmt_status st = lbrmt_internal_check_flags(s);
    if (st != LBRMT_OK) return st;
    std::vector<unsigned char> head(h.header_bytes);
    std::memcpy(head.data(), &h, sizeof(h));
    if (!recs.empty()) std::memcpy(head.data() + sizeof(h), recs.data(), recs.size() * sizeof(CkSolid));
    unsigned char *dst = (unsigned char *)dev_blob;
    cudaError_t e = cudaMemcpyAsync(dst, head.data(), head.size(), cudaMemcpyHostToDevice, s->stream);
    size_t off = align_up(h.header_bytes);
    for (int k = 0; k < nsec && e == cudaSuccess; k++) {
        e = cudaMemcpyAsync(dst + off, sec[k].ptr, sec[k].bytes, cudaMemcpyDeviceToDevice, s->stream);
        off += align_up(sec[k].bytes);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess)
        return lbrmt_internal_fail(s, LBRMT_ERR_CUDA, std::string("checkpoint copy: ") + cudaGetErrorString(e));
    *bytes = (size_t)h.total_bytes;
    return LBRMT_OK;
}

extern "C" lbrmt_status lbrmt_load(lbrmt_sim *s, const void *dev_blob, size_t bytes) {
    if (!s || !dev_blob) return LBRMT_ERR_ARG;
    if (s->in_batch) return lbrmt_internal_fail(s, LBRMT_ERR_STATE, "a batch member is loaded with its batch");
    if (bytes < sizeof(CkHeader)) return mismatch(s, "buffer shorter than the header");
    if (s->stream) cudaStreamSynchronize(s->stream);
    CkHeader h;
    cudaError_t e = cudaMemcpy(&h, dev_blob, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return lbrmt_internal_fail(s, LBRMT_ERR_CUDA, std::string("checkpoint header: ") + cudaGetErrorString(e));
    if (std::memcmp(h.magic, CK_MAGIC, 8) != 0 || h.version != CK_VERSION) return mismatch(s, "not a checkpoint");
    if (h.total_bytes > bytes) return mismatch(s, "buffer shorter than the checkpoint");
    const lbrmt_config &c = s->cfg;
    if (h.precision != c.precision) return mismatch(s, "precision");
    if (h.nx != c.nx || h.ny != c.ny || h.bc_x != c.bc_x || h.bc_y != c.bc_y) return mismatch(s, "grid or walls");
    if (h.force_kind != c.force_kind || h.n_layers != c.n_layers || h.rmax != c.rmax ||
        h.kmax != c.max_solids_per_tile || h.tau != c.tau || h.rho_f != c.rho_f || h.lid_u != c.lid_u ||
        h.eps != c.eps || h.eta != c.eta || h.gravity != c.gravity || h.fa0 != c.force_a[0] ||
        h.fa1 != c.force_a[1] || h.deform_margin != c.deform_margin)
        return mismatch(s, "method parameters");
    if (h.nsolids != (int)s->solids.size()) return mismatch(s, "number of solids");
    if (h.header_bytes != sizeof(CkHeader) + (uint64_t)h.nsolids * sizeof(CkSolid)) return mismatch(s, "header size");
    std::vector<CkSolid> recs(h.nsolids);
    if (h.nsolids > 0) {
        e = cudaMemcpy(recs.data(), (const unsigned char *)dev_blob + sizeof(CkHeader), recs.size() * sizeof(CkSolid),
                       cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            return lbrmt_internal_fail(s, LBRMT_ERR_CUDA, std::string("checkpoint solids: ") + cudaGetErrorString(e));
    }
    for (int k = 0; k < h.nsolids; k++) {
        const SolidHost &o = s->solids[k];
        const CkSolid &r = recs[k];
        if (r.shape != o.shape || r.T != o.T || r.xc != o.xc || r.yc != o.yc || r.R != o.R || r.a != o.a ||
            r.b != o.b)
            return mismatch(s, "solid geometry");
    }
    // the tile shape of the saved registries (their layout depends on it)
    if (s->sp.tx != h.tile_x) {
        lbrmt_status st = lbrmt_set_tile_x(s, h.tile_x);
        if (st != LBRMT_OK) return st;
    }
    // material parameters as saved (lbrmt_set_solid_params may have changed them)
    for (int k = 0; k < h.nsolids; k++) {
        s->solids[k].rho_s = recs[k].rho_s;
        s->solids[k].G = recs[k].G;
    }
    if (!s->inited) {
        lbrmt_status st = lbrmt_init(s);
        if (st != LBRMT_OK) return st;
    } else {
        lbrmt_internal_refresh_scales(s);  // 16-bit storage scales follow the materials
    }
    Section sec[CK_MAX_SECTIONS];
    const int nsec = sections(s, sec);
    if ((int)h.nsections != nsec || h.xi_total != s->xi_total || h.ntiles_cap != s->ntiles_cap ||
        h.mass_parts_cap != s->mass_parts_cap || h.nregions_cap != s->nregions_cap)
        return mismatch(s, "buffer sizes");
    for (int k = 0; k < nsec; k++)
        if (h.section_bytes[k] != sec[k].bytes) return mismatch(s, "buffer sizes");
    const unsigned char *src = (const unsigned char *)dev_blob;
    size_t off = align_up(h.header_bytes);
    for (int k = 0; k < nsec && e == cudaSuccess; k++) {
        e = cudaMemcpyAsync(sec[k].ptr, src + off, sec[k].bytes, cudaMemcpyDeviceToDevice, s->stream);
        off += align_up(sec[k].bytes);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d.err, 0, 16, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess)
        return lbrmt_internal_fail(s, LBRMT_ERR_CUDA, std::string("checkpoint restore: ") + cudaGetErrorString(e));
    // the step counter fixes which half of each ping-pong pair is current; the
    // captured graph reads the same buffers, so it stays valid
    s->steps = h.steps;
    return LBRMT_OK;
}
