/*
 * lbrmt.h -- C ABI of the GB300 (sm_103a) LBRMT time step.
 *
 * The lattice Boltzmann reference map technique (Sun & Rycroft, arXiv
 * 2402.12696) couples a D2Q9 lattice Boltzmann fluid with finite-strain
 * neo-Hookean solids tracked by a reference map on one fixed grid.  One call
 * of lbrmt_step advances every node by Algorithm 1 of the paper:
 *   reference-map advection (Sec. 3.1), extrapolation into a band of layers
 *   (Sec. 3.2), relabelling with phi = phi_0(xi), divergence of the blended
 *   solid stress with contact (Secs. 3.3, 3.6, Eq. 2_4_F_divs), SFC
 *   equilibrium (Eq. 2_3_feq_sfc), Guo forcing (Eq. 2_2_Fi / 3_4_Fi), BGK
 *   collision (Eq. 2_2_bgk_force), wall conditions (Sec. 3.5), streaming and
 *   the half-force moments (Sec. 3.4).
 *
 * Conventions for every entry point:
 *   - Lattice units: dx = dt = 1.  Grid node (i, j) has linear index
 *     j * nx + i; "field" outputs are nx*ny doubles in that order.
 *   - The library owns all simulation state.  It allocates device memory
 *     through the config's alloc/free callbacks when they are set (the
 *     Python binding routes them to the PyTorch caching allocator), else
 *     with cudaMalloc.  Pointers passed by the caller stay caller-owned.
 *   - All work is enqueued asynchronously on the CUDA stream given to
 *     lbrmt_create.  Calls named *_host copy to/from host memory and return
 *     after the copy completed.  A page-locked (or registered) host buffer is
 *     read or written by the kernels directly over the coherent CPU-GPU link;
 *     a pageable one goes through a device staging buffer and a copy.
 *   - Every call returns an lbrmt_status and never aborts.  Device-side
 *     error flags (non-finite density, registry overflow, extrapolation
 *     failure, tile overflow) are raised asynchronously and reported by the
 *     next lbrmt_sync, read or stats call; lbrmt_last_error() gives text.
 *   - A sim handle is not thread-safe; use one handle per host thread.
 */
#ifndef LBRMT_H
#define LBRMT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbrmt_sim lbrmt_sim;

typedef enum {
    LBRMT_OK = 0,
    LBRMT_ERR_ARG = -1,         /* invalid argument */
    LBRMT_ERR_CUDA = -2,        /* a CUDA runtime call failed */
    LBRMT_ERR_NUMERIC = -3,     /* non-finite density or velocity */
    LBRMT_ERR_OVERFLOW = -4,    /* solids-per-tile registry or solid tile overflow */
    LBRMT_ERR_EXTRAP = -5,      /* extrapolation window exceeded rmax or stencil left the band */
    LBRMT_ERR_TIMEOUT = -6,     /* a bounded device wait gave up */
    LBRMT_ERR_PARAM_RANGE = -7, /* parameter outside the limits of Appendix A (1/2 < tau <= 1, ...) */
    LBRMT_ERR_STATE = -8        /* call not valid in the current state */
} lbrmt_status;

enum { LBRMT_PERIODIC = 0, LBRMT_WALL = 1 };
enum { LBRMT_FP32 = 0, LBRMT_FP64 = 1, LBRMT_FP16_STORE = 2, LBRMT_BF16_STORE = 3 };
enum { LBRMT_FORCE_NONE = 0, LBRMT_FORCE_CONST = 1, LBRMT_FORCE_SINE_X = 2, LBRMT_FORCE_FIELD = 3 };
enum { LBRMT_SHAPE_DISK = 0, LBRMT_SHAPE_ELLIPSE = 1, LBRMT_SHAPE_RECT = 2 };
enum { LBRMT_FORCE_MODE_LITERAL = 0, LBRMT_FORCE_MODE_CONSERVATIVE = 1 };

/* Field ids for lbrmt_read_fields.  RHO/UX/UY are the moments of the current
 * populations (Sec. 3.4); FX/FY/DRHO are the force density F of Eq. 2_4_F_divs
 * and the density difference of Eq. 2_3_drho used by the last step; XI_X,
 * XI_Y, PHI are the reference map (absolute reference coordinates) and level
 * set of one solid on its solid + band nodes (NaN elsewhere); DET_F_DEV and
 * VON_MISES are det F - 1 (F = J^-1, J = d xi / dx by central differences over
 * the 4-neighbours; the volumetric deviation of Sec. 4.1) and the von Mises
 * stress of the neo-Hookean stress of Eq. 3_3_solid_stress in plane strain, on
 * the solid's nodes (phi < 0; NaN elsewhere); POP0 + q is the population f_q. */
enum {
    LBRMT_FIELD_RHO = 0, LBRMT_FIELD_UX = 1, LBRMT_FIELD_UY = 2,
    LBRMT_FIELD_FX = 3, LBRMT_FIELD_FY = 4, LBRMT_FIELD_DRHO = 5,
    LBRMT_FIELD_XI_X = 10, LBRMT_FIELD_XI_Y = 11, LBRMT_FIELD_PHI = 12,
    LBRMT_FIELD_DET_F_DEV = 14, LBRMT_FIELD_VON_MISES = 15,
    LBRMT_FIELD_POP0 = 20
};

typedef void *(*lbrmt_alloc_fn)(size_t bytes, void *ctx);
typedef void (*lbrmt_free_fn)(void *ptr, void *ctx);

typedef struct {
    int nx, ny;                 /* grid nodes; nx, ny >= 8 and 9 nx ny < 2^31 */
    int bc_x, bc_y;             /* LBRMT_PERIODIC or LBRMT_WALL (halfway bounce-back, Sec. 3.5) */
    double tau;                 /* BGK relaxation time; 1/2 < tau <= 1 (Appendix A) */
    double rho_f;               /* fluid density (1 in the paper) */
    double lid_u;               /* speed of the top (y = ny-1/2) wall in +x; needs bc_y = WALL */
    double eps;                 /* blur-zone half-width (1.5 in the paper) */
    int n_layers;               /* extrapolation layers (11 in the paper), 1..20 */
    double eta;                 /* contact constant of Eq. 3_6_collision_stress */
    double gravity;             /* g >= 0 acting in -y on solids: a = (1 - rho_f/rho_s) g (Sec. 4.3) */
    int force_kind;             /* LBRMT_FORCE_*: body force on all phases */
    double force_a[2];          /* (fx, fy) for CONST, (A, 0) for f_x = A sin(2 pi y / ny);
                                   FIELD: a per-node field set by lbrmt_set_body_force_field (0 at creation) */
    int precision;              /* LBRMT_FP32 / LBRMT_FP64 arithmetic and storage; LBRMT_FP16_STORE /
                                   LBRMT_BF16_STORE: FP32 arithmetic, populations and the density
                                   plane stored in 16 bits (times power-of-two scales per plane,
                                   chosen at initialisation from bounds of the values) */
    int max_solids_per_tile;    /* registry slots per tile, 1..8 */
    int rmax;                   /* largest extrapolation window half-width (>= 2) */
    int tile_x;                 /* registry / LB tile width: 16, 32, 64 or 128 nodes (height 256 /
                                   tile_x); 0 selects 32.  Results do not depend on it. */
    double deform_margin;       /* room a solid's tile leaves for deformation beyond its band, as a
                                   fraction of its (circumscribed) radius (default 0.25; a band that
                                   reaches the tile edge raises LBRMT_ERR_OVERFLOW) */
    int force_mode;             /* LBRMT_FORCE_MODE_LITERAL (0, default): the Guo term and the
                                   half-force moments carry rho F for the whole force density, as the
                                   expanded Eq. 3_4_Fi prints it (F an acceleration, Sec. 3.4);
                                   LBRMT_FORCE_MODE_CONSERVATIVE (1): the divergence of the solid and
                                   contact stresses (Eqs. 3_3_div_solid_stress, 3_6_global_stress)
                                   enters without rho, the accelerations keep it, so the stress
                                   forces sum to zero over a periodic box.  The adjoint supports
                                   mode 0 only (LBRMT_ERR_ARG). */
    lbrmt_alloc_fn alloc;       /* optional device allocator */
    lbrmt_free_fn free;
    void *alloc_ctx;
} lbrmt_config;

/* Fill a config with the paper's defaults (eps 1.5, 11 layers, rho_f 1,
 * eta 1, tau 1, periodic 64x64, FP32, 8 slots, rmax 11, 32x8 tiles). */
void lbrmt_default_config(lbrmt_config *cfg);

/* Create a simulation on the current CUDA device.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream; then no CUDA graph is used).
 * Checks the Appendix A limit 1/2 < tau <= 1 (LBRMT_ERR_PARAM_RANGE). */
lbrmt_status lbrmt_create(const lbrmt_config *cfg, void *cuda_stream, lbrmt_sim **out);

/* Add a solid before the first step (Sec. 3.6: material and shape per
 * object).  shape = LBRMT_SHAPE_DISK: level set phi_0(X) = |X - c| - radius
 * (phi < 0 inside, Sec. 2.4); (cx, cy) in lattice units, rho_s > 0, G >= 0
 * the small-strain shear modulus of Eq. 2_4_solid_const.  Returns the solid
 * id (0, 1, ...) in *solid_id_out (may be NULL). */
lbrmt_status lbrmt_add_solid(lbrmt_sim *sim, int shape, double cx, double cy, double radius,
                             double rho_s, double G, int *solid_id_out);

/* Add a solid of any shape: LBRMT_SHAPE_DISK (radius a; b ignored),
 * LBRMT_SHAPE_ELLIPSE (semi-axes a along x, b along y) or LBRMT_SHAPE_RECT
 * (half-sides a, b), axis-aligned, centred at (cx, cy); its level set phi_0 is
 * the signed distance to the boundary (negative inside; Sec. 3 uses phi < 0
 * for the solid).  a, b >= 1; G <= rho_s (the shear wave speed sqrt(G/rho_s)
 * within one node per step, Appendix A; else LBRMT_ERR_PARAM_RANGE).  The
 * adjoint supports disks only. */
lbrmt_status lbrmt_add_solid_shape(lbrmt_sim *sim, int shape, double cx, double cy, double a, double b,
                                   double rho_s, double G, int *solid_id_out);

/* Body force field f(x) of Eq. 2_4_F_divs for force_kind LBRMT_FORCE_FIELD:
 * dev_xy is a device array of 2*nx*ny doubles (x components, then y
 * components, row-major), copied (and rounded to the arithmetic precision);
 * caller-owned.  Acts on all phases from the next step on.  Set between steps,
 * it also replaces the previous step's body force in the half-force term
 * rho F / 2 of the next step's moments wherever no solid was registered
 * (that term is rebuilt from the stored density and the current field); the
 * method holds the field constant, and so do the adjoint and its gradient.
 * sim_index must be 0. */
lbrmt_status lbrmt_set_body_force_field(lbrmt_sim *sim, int sim_index, const double *dev_xy);

/* Change a solid's density and shear modulus.  After initialisation this
 * also returns the simulation to its initial state (lbrmt_reset). */
lbrmt_status lbrmt_set_solid_params(lbrmt_sim *sim, int solid_id, double rho_s, double G);

/* Return to the initial state of Algorithm 1 with the current parameters
 * (keeps the allocations and the body force field). */
lbrmt_status lbrmt_reset(lbrmt_sim *sim);

/* Checkpoint and resume: the whole state that Algorithm 1 carries from one
 * step to the next (populations and the density plane of the half-force term,
 * both halves of every ping-pong pair of reference-map tiles, frames, tile
 * registries and force pools, the body force, the solids' descriptors and
 * statistics, and the step count).  lbrmt_save with dev_blob NULL stores the size needed in *bytes;
 * with a caller-owned device buffer of *bytes >= that size it waits for the
 * simulation's stream, checks the device error flags (a raised flag is
 * returned as its status and nothing is written), copies the state into the
 * buffer and stores the size written in *bytes.  Needs an initialised
 * simulation (LBRMT_ERR_STATE otherwise).
 * lbrmt_load restores a saved state into a simulation created with the same
 * configuration and solids (same order, shape, position, size and tile side;
 * densities and shear moduli are taken from the checkpoint) and initialises it
 * first if needed; it adopts the checkpoint's tile shape.  A buffer that is not
 * a checkpoint of a matching simulation gives LBRMT_ERR_ARG and leaves the
 * state as it was.  Stepping on from a loaded state gives the same results,
 * bit for bit, as stepping on from the state that was saved.  The buffer stays
 * caller-owned and is not referenced after the call. */
lbrmt_status lbrmt_save(lbrmt_sim *sim, void *dev_blob, size_t *bytes);
lbrmt_status lbrmt_load(lbrmt_sim *sim, const void *dev_blob, size_t bytes);

/* Registry / lattice Boltzmann tile shape: tile_x in {16, 32, 64, 128} (0:
 * 32), height 256 / tile_x.  After initialisation this returns the
 * simulation to its initial state.  The results do not depend on it. */
lbrmt_status lbrmt_set_tile_x(lbrmt_sim *sim, int tile_x);
int lbrmt_tile_x(const lbrmt_sim *sim);

/* Autotuner of the tile shape and of the lattice Boltzmann loads: time
 * `steps` graph-replayed steps (best of two, after 4 warm-up steps) for each
 * tile_x in {16, 32, 64, 128} with tensor-memory staging and with direct
 * loads, keep the fastest and return to the initial state with it.  The
 * results do not depend on the choice.  best_tile_x / best_tma (may be NULL)
 * receive the choice; ms_out (8 doubles, may be NULL) the ms per step of
 * (16, staged), (16, direct), (32, staged), ... (-1 where not applicable). */
lbrmt_status lbrmt_autotune_tile(lbrmt_sim *sim, int steps, int *best_tile_x, int *best_tma, double *ms_out);

/* Initialise (Algorithm 1, initialisation): xi = x on each solid and its
 * band, phi = phi_0(xi), rho = rho_t, v = 0, f = f^eq,SFC(rho_t, 0).  Called
 * implicitly by the first step or read; allocates the solid tiles. */
lbrmt_status lbrmt_init(lbrmt_sim *sim);

/* Advance nsteps >= 0 time steps of Algorithm 1 (asynchronous). */
lbrmt_status lbrmt_step(lbrmt_sim *sim, int nsteps);

/* Write one field (ids above) as nx*ny doubles to the device buffer dev_out
 * (caller-owned, nx*ny*8 bytes).  solid_id selects the solid for XI_X, XI_Y
 * and PHI; sim_index must be 0. */
lbrmt_status lbrmt_read_fields(lbrmt_sim *sim, int sim_index, int field, int solid_id,
                               double *dev_out);

/* Same as lbrmt_read_fields but into host memory (nx*ny doubles); waits for
 * the stream.  A page-locked (or registered) buffer receives the fields written
 * at every node (RHO .. DRHO, POP0 + q) from the field kernel directly, over
 * the coherent CPU-GPU link; other buffers and the per-solid fields go through
 * a device staging buffer and a copy. */
lbrmt_status lbrmt_read_fields_host(lbrmt_sim *sim, int sim_index, int field, int solid_id,
                                    double *host_out);

/* Overwrite the populations from host memory (9 planes of nx*ny doubles,
 * plane q = f_q) and reset the half-force term of the next step's moments to
 * zero (as at initialisation); waits for the
 * stream.  A page-locked (or registered) buffer is read by the conversion
 * kernel directly; other buffers are copied to a device staging buffer
 * (9*nx*ny doubles, allocated on first use) first. */
lbrmt_status lbrmt_set_populations_host(lbrmt_sim *sim, const double *host_f);

/* Per-solid FP64 statistics of the current state, S x 10 doubles into host
 * memory: lambda-weighted area sum, centroid x, centroid y (unwrapped frame),
 * mass sum(lambda rho), momentum sum(lambda rho u), sum(lambda rho v), the
 * maximum of |det F - 1| over the solid nodes (phi < 0) and its lambda-weighted
 * mean over them; lambda = 1 - H_eps(phi) on domain nodes; and the net contact
 * force (x, y) on the solid: the divergence (Eq. 3_3_div_solid_stress) of the
 * contact stresses of Eq. 3_6_collision_stress between it and each other solid,
 * summed over the domain nodes nearer to it than to the other (phi_s < phi_t,
 * half where equal), so the forces of one contact are equal and opposite in a
 * periodic box.  Sums are FP64 over compensated per-thread sums of FP32 node
 * terms (FP32 arithmetic) or FP64 throughout (FP64). */
lbrmt_status lbrmt_solid_stats(lbrmt_sim *sim, int sim_index, double *host_out);

/* The same statistics, enqueued on the simulation's stream without waiting:
 * host_out (S x 10 doubles, page-locked host memory owned by the caller) is
 * written by the statistics kernel directly when the stream reaches it (a
 * pageable buffer is filled by a copy from device memory instead), so the
 * caller keeps it alive and
 * unread until lbrmt_sync returns; device error flags surface there.  Needs
 * an initialised simulation (LBRMT_ERR_STATE otherwise).  Lets a caller read
 * every step's statistics without stalling the stream between steps. */
lbrmt_status lbrmt_solid_stats_async(lbrmt_sim *sim, int sim_index, double *host_out);

/* Total mass sum_x rho of the current populations (every node's rho - rho_f
 * formed in FP64 from its stored values and rest base, summed per registry
 * tile and then in a fixed order; Appendix C: conserved to round-off in a
 * periodic or walled box), into host memory.  Needs an initialised
 * simulation (LBRMT_ERR_STATE otherwise). */
lbrmt_status lbrmt_total_mass(lbrmt_sim *sim, int sim_index, double *host_out);

/* Number of registry tiles (tile_x x 256/tile_x nodes) that the last step
 * registered for the stress/force kernel (tiles touched by a blur zone), into
 * host memory; 0 before the first step. */
lbrmt_status lbrmt_active_tiles(lbrmt_sim *sim, int sim_index, long long *host_out);

/* Total mass sum_x rho of the current populations, written as one double to
 * dev_out (caller-owned device memory), enqueued on the simulation's stream;
 * the library allocates no device memory for it.  The paper has no
 * counterpart: this is for callers that cannot allocate device memory where
 * they need the diagnostic (a frozen memory pool, a device handed to another
 * allocator, a real-time loop that allows no allocation).  Its partial sums
 * live in one file-scope device array of 2048 doubles (16 KiB) that every GPU
 * loading the library holds until exit; simulations of more than 33,554,432
 * nodes are rejected with LBRMT_ERR_ARG.  The first call on a device (and the
 * first after the device's context changed, e.g. after cudaDeviceReset) looks
 * up that array's address, so make it before any stream capture.  The
 * simulation's device must be current and the simulation initialised
 * (LBRMT_ERR_STATE otherwise).  All calls share the array, which keeps the
 * last call's partial sums (each call overwrites the ones it uses): calls that
 * overlap on the GPU (other streams of the same device) race and give wrong
 * results. */
lbrmt_status lbrmt_total_mass_noalloc(lbrmt_sim *sim, int sim_index, double *dev_out);

/* Wait for the stream and turn device error flags into a status. */
lbrmt_status lbrmt_sync(lbrmt_sim *sim);

/* Number of time steps taken, number of solids, kernel launches issued by
 * the last lbrmt_step call (graph launches count their kernels). */
long long lbrmt_steps_done(const lbrmt_sim *sim);
int lbrmt_num_solids(const lbrmt_sim *sim);
long long lbrmt_last_launch_count(const lbrmt_sim *sim);

/* Advance nsteps >= 1 steps with direct launches of the sequential schedule
 * (lbrmt_set_overlap) and a CUDA event around every kernel (on the
 * simulation's stream), then wait.  ms_out[k] receives
 * the mean duration in milliseconds of kernel k of a step: 0 = reference-map
 * kernel (advect, extrapolate, relabel), 1 = stress/force kernel, 2 = fused
 * lattice Boltzmann kernel (host array of 3 floats; 0 where not launched). */
lbrmt_status lbrmt_step_timed(lbrmt_sim *sim, int nsteps, float *ms_out);

/* Use (1) or bypass (0) CUDA graphs for lbrmt_step; default 1. */
lbrmt_status lbrmt_set_use_graphs(lbrmt_sim *sim, int enable);

/* Load the populations of the lattice Boltzmann kernel with tensor-memory
 * copies into shared memory (1, default) or directly (0).  The results are the
 * same bit for bit.  The tensor path needs nx times the storage size to be a
 * multiple of 16 bytes; lbrmt_uses_tma tells whether it is in use. */
lbrmt_status lbrmt_set_use_tma(lbrmt_sim *sim, int enable);
int lbrmt_uses_tma(const lbrmt_sim *sim);

/* Overlapped step (1, default) or sequential step (0).  Overlapped: each step
 * first classifies the lattice Boltzmann kernel's regions (64 nodes wide) from
 * the previous step's tile registry; the regions whose tiles and neighbour tiles
 * hold no solid (interfaces move less than one node per step, Appendix A) are
 * advanced on an internal lowest-priority stream concurrently with the
 * reference-map and stress kernels, which the simulation's stream runs at the
 * highest priority; the step ends when both are done (the caller's stream then
 * waits for the internal one).  The results are the same bit for bit.  A solid
 * found in a region that a step treated as free raises LBRMT_ERR_NUMERIC at the
 * next error check.  Not used with tensor-memory loads (lbrmt_set_use_tma) or
 * without solids; lbrmt_step_timed always takes the sequential schedule.
 * lbrmt_uses_overlap tells whether steps overlap (after initialisation). */
lbrmt_status lbrmt_set_overlap(lbrmt_sim *sim, int enable);
int lbrmt_uses_overlap(const lbrmt_sim *sim);

/* CTA width of the reference-map kernel (one CTA per solid, Sec. 3.1-3.2):
 * 0 (default) chooses 1024 threads when the solids number at most half the
 * SMs and FP32 arithmetic is used, else 256; 256 or 1024 fix it (1024 falls
 * back to 256 with FP64 arithmetic).  The solids' statistics are summed in an
 * order that depends on the width, so results agree to rounding, not bit for
 * bit.  Any other value gives LBRMT_ERR_ARG.  Takes effect at the next step;
 * lbrmt_rmt_threads tells the width in use (after initialisation, else 0). */
lbrmt_status lbrmt_set_rmt_threads(lbrmt_sim *sim, int threads);
int lbrmt_rmt_threads(const lbrmt_sim *sim);

/* Self-check of the failure path of the bounded device waits: one GPU
 * thread waits, with the bounded wait that guards the tensor-memory copies of
 * the lattice Boltzmann kernel, on a barrier that nothing completes, until the
 * wait gives up (about 2^31 clock cycles, ~1 s), and records the timeout in
 * the device error flags as that kernel does.  Returns LBRMT_ERR_TIMEOUT, as
 * it must, and clears the flags; LBRMT_OK would mean that the wait did not
 * give up.  A device error already pending is returned instead, without
 * running the check.  The simulation's state is not touched. */
lbrmt_status lbrmt_check_bounded_wait(lbrmt_sim *sim);

/* Text of the last error on this handle ("" if none). */
const char *lbrmt_last_error(const lbrmt_sim *sim);

/* Free the handle and all device memory it owns. */
void lbrmt_destroy(lbrmt_sim *sim);

/* ---------------------------------------------------------------------------
 * Adjoint.  The paper has no counterpart (it runs the method forward only).
 * The loss L is any function of the solids' centroids at the final step,
 * c_s = sum_x lambda_s(x) x / sum_x lambda_s(x), lambda_s = 1 - H_eps(phi_s)
 * over the domain nodes of the solid's tile (unwrapped coordinates).  The
 * reverse sweep applies the transposed Jacobian of every kernel of the step
 * (the branch decisions of the forward step held fixed) with checkpointing.
 * FP32 and FP64 arithmetic only.
 * ------------------------------------------------------------------------- */

/* Return to the initial state, run nsteps >= 1 steps keeping a copy of the
 * device state every checkpoint_every >= 1 steps and at the end, and write the
 * final centroids (S x 2 host doubles, may be NULL).  Synchronous.  Needs
 * about (nsteps / checkpoint_every + 1) times the simulation's state memory. */
lbrmt_status lbrmt_forward_checkpointed(lbrmt_sim *sim, int nsteps, int checkpoint_every, double *centroids_out);

/* Gradients of L through the last lbrmt_forward_checkpointed run, given
 * dL_dcentroid = dL/dc_s (S x 2 host doubles): dL_dG[s] = dL/dG_s and
 * dL_dratio[s] = dL/d(rho_s / rho_f) (S host doubles each, may be NULL), and
 * dL_dbody_dev = dL/df(x) for the body force field (2 nx ny device doubles,
 * x plane then y plane; needs force_kind LBRMT_FORCE_FIELD; may be NULL), and
 * dL_df0_dev = dL/df_q(x, t = 0) for the initial populations (9 nx ny device
 * doubles, plane q at offset q nx ny; may be NULL).
 * Recomputes each segment from its checkpoint (about one extra forward run);
 * leaves the simulation in the final state of the forward run.  Synchronous. */
lbrmt_status lbrmt_backward(lbrmt_sim *sim, const double *dL_dcentroid, double *dL_dG, double *dL_dratio,
                            double *dL_dbody_dev, double *dL_df0_dev);

/* ---------------------------------------------------------------------------
 * Batches: many independent simulations advanced together.  The paper has no
 * counterpart (it runs one instance of Algorithm 1 at a time); every member of
 * a batch computes exactly what it would compute alone (bit-identical fields),
 * but a batch step is one persistent launch per kernel of the step over the
 * work of all members, replayed through CUDA graphs.
 * ------------------------------------------------------------------------- */
typedef struct lbrmt_batch lbrmt_batch;

/* Create a batch of nsim (1..1024) simulations, one per config (all with the
 * same precision; tile_x 0 selects 32), on the given CUDA stream (NULL: the
 * legacy default stream, stepped without graphs).  Configs are validated as
 * by lbrmt_create; the allocator of cfgs[0] also holds the batch's own lists.
 * The batch owns its members. */
lbrmt_status lbrmt_create_batch(const lbrmt_config *cfgs, int nsim, void *cuda_stream, lbrmt_batch **out);

/* Add a solid to member sim_index (before lbrmt_batch_init); as
 * lbrmt_add_solid_shape / lbrmt_add_solid. */
lbrmt_status lbrmt_batch_add_solid_shape(lbrmt_batch *batch, int sim_index, int shape, double cx, double cy,
                                         double a, double b, double rho_s, double G, int *solid_id_out);
lbrmt_status lbrmt_batch_add_solid(lbrmt_batch *batch, int sim_index, int shape, double cx, double cy,
                                   double radius, double rho_s, double G, int *solid_id_out);

/* Initialise every member (Algorithm 1, initialisation).  With
 * autotune_steps > 0, first choose each grid size's tile shape among
 * tile_x = 16, 32, 64, 128 by timing whole batch steps (autotune_steps timed
 * steps per trial, greedy over grid sizes), then start every member again
 * from its initial state with the chosen shapes.  Synchronous. */
lbrmt_status lbrmt_batch_init(lbrmt_batch *batch, int autotune_steps);

/* Advance every member nsteps >= 0 steps (asynchronous). */
lbrmt_status lbrmt_batch_step(lbrmt_batch *batch, int nsteps);

/* As lbrmt_step_timed, for the batched kernels (ms_out: 3 floats, mean ms of
 * the reference-map, force and lattice Boltzmann launches of a batch step;
 * always the sequential schedule). */
lbrmt_status lbrmt_batch_step_timed(lbrmt_batch *batch, int nsteps, float *ms_out);

/* Overlapped batch step (1, default) or sequential (0), as lbrmt_set_overlap
 * for one simulation: every member's regions are classified from its previous
 * registry, and the lattice Boltzmann kernel of the solid-free regions of all
 * members runs on an internal lowest-priority stream concurrently with the
 * reference-map and force kernels, which run at the highest priority.  The
 * results are the same bit for bit.  Not used without solids.
 * lbrmt_batch_uses_overlap tells whether steps overlap (after initialisation). */
lbrmt_status lbrmt_batch_set_overlap(lbrmt_batch *batch, int enable);
int lbrmt_batch_uses_overlap(const lbrmt_batch *batch);

/* Wait for the stream and check every member's device error flags. */
lbrmt_status lbrmt_batch_sync(lbrmt_batch *batch);

/* Borrowed handle of member sim_index (after lbrmt_batch_init) for
 * lbrmt_read_fields*, lbrmt_solid_stats, lbrmt_total_mass and the other
 * queries; lbrmt_step on it returns LBRMT_ERR_STATE.  Do not destroy it. */
lbrmt_status lbrmt_batch_member(lbrmt_batch *batch, int sim_index, lbrmt_sim **out);

/* Number of members; tile_x in use by member sim_index. */
int lbrmt_batch_size(const lbrmt_batch *batch);
int lbrmt_batch_tile_x(const lbrmt_batch *batch, int sim_index);

/* Autotuner trials: fills up to cap entries of (nx, ny, tile_x, ms per batch
 * step) host arrays (any may be NULL) and returns the number of trials. */
int lbrmt_batch_tune_log(const lbrmt_batch *batch, int *nx, int *ny, int *tile_x, double *ms, int cap);

long long lbrmt_batch_steps_done(const lbrmt_batch *batch);
long long lbrmt_batch_last_launch_count(const lbrmt_batch *batch);
const char *lbrmt_batch_last_error(const lbrmt_batch *batch);

/* Free the batch, its members and all device memory they own. */
void lbrmt_destroy_batch(lbrmt_batch *batch);

#ifdef __cplusplus
}
#endif

#endif /* LBRMT_H */
