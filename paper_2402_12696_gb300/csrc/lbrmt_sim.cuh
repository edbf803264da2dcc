// lbrmt_sim.cuh -- the simulation handle behind the C ABI (host side).
#pragma once

#include <string>
#include <vector>

#include "lbrmt.h"
#include "lbrmt_engine.cuh"

struct SolidHost {
    double xc, yc, R, rho_s, G;  // R: disk radius, circumscribed radius of other shapes
    int shape;
    double a, b;
    int T;
    long long off;
};

struct AdjointStore;

constexpr int GRAPH_LONG = 16;

struct lbrmt_sim {
    lbrmt_config cfg;
    int device = 0;
    cudaStream_t stream = nullptr;
    lbrmt::SimParams sp;
    const lbrmt::EngineOps *eng = nullptr;
    lbrmt::LaunchInfo li;
    lbrmt::DevState d;
    std::vector<SolidHost> solids;
    long long xi_total = 0;         // reals in one xi buffer (all solid tiles)
    long long ntiles_cap = 0;       // registry / pool capacity in tiles (largest over the tile shapes)
    long long mass_parts_cap = 0;  // K1 mass partial slots allocated (max over tile shapes)
    long long nregions_cap = 0;    // K1 regions (busy flags) allocated (max over tile shapes)
    bool inited = false;
    long long steps = 0;
    bool use_graphs = true;
    bool in_batch = false;          // stepped by a batch: lbrmt_step is refused
    cudaGraphExec_t gexec = nullptr;       // two steps (one of each parity)
    cudaGraphExec_t gexec_long = nullptr;  // GRAPH_LONG steps: the overlap runs across their joins less often
    long long last_launches = 0;
    std::vector<void *> allocs;
    double *scratch = nullptr;      // device: S*8 stats or 1 mass value
    double *staging = nullptr;      // device: 9*P doubles for set_populations
    std::string err;
    AdjointStore *adj = nullptr;    // checkpoints and buffers of the adjoint (lbrmt_adjoint.cu)
};

// Wait for the simulation's stream and map its device error flags to a status.
lbrmt_status lbrmt_internal_check_flags(lbrmt_sim *s);

// Device allocation owned by the simulation (freed with it), and error recording.
void *lbrmt_internal_alloc(lbrmt_sim *s, size_t bytes);
lbrmt_status lbrmt_internal_fail(lbrmt_sim *s, lbrmt_status st, const std::string &msg);
void lbrmt_internal_adjoint_free(lbrmt_sim *s);
// Recompute the 16-bit storage scales from the solids' materials (drops stale graphs).
void lbrmt_internal_refresh_scales(lbrmt_sim *s);
