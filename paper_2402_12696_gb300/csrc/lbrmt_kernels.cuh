// lbrmt_kernels.cuh -- device code of the LBRMT time step for sm_103a.
//
// Three kernels make one step of Algorithm 1 (Sun & Rycroft, arXiv 2402.12696):
//   K2 rmt_solid_kernel   one CTA per solid: advect xi (Sec. 3.1), extrapolate
//                         it layer by layer (Sec. 3.2), relabel, register the
//                         32x8 tiles its blur zone touches, per-solid FP64 stats.
//   K3 force_kernel       one CTA per registered tile: half-edge Jacobians and
//                         neo-Hookean stresses (Sec. 3.3), multi-solid blend and
//                         contact (Sec. 3.6), divergence (Eq. 3_3_div_solid_stress),
//                         external accelerations and the SFC density difference.
//   K1 lb_step_kernel     one thread per node: moments with the half-force
//                         (Sec. 3.4), SFC equilibrium (Eq. 2_3_feq_sfc), Guo
//                         forcing (Eq. 2_2_Fi x rho), BGK collision, wall
//                         conditions (Sec. 3.5) and push streaming, FP64 mass.
// Populations are stored as deviations f_q - w_q rho_f in structure-of-arrays
// planes; the reference map of each solid lives in its own moving square tile
// in solid-local coordinates xi - X_c.
#pragma once

#include <cuda.h>  // CUtensorMap (the tensor maps are encoded through the runtime's driver entry point)
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

namespace lbrmt {

// Registry tiles are tile_x x tile_y nodes with tile_x * tile_y = TILE_N, one
// thread per node; tile_x in {16, 32, 64, 128} is chosen per simulation.
constexpr int TILE_N = 256;
constexpr int KMAX = 8;                     // registry slots per tile (upper bound)
constexpr int RMT_THREADS = 256;
#ifndef RMT_MIN_BLOCKS
#define RMT_MIN_BLOCKS 4
#endif
constexpr int LIST_CAP = 2048;              // per-layer target list in shared memory
constexpr int RMT_LIST_MIN_BYTES = 12288;   // least node-list space (bytes) for which K2 takes a smaller carveout
constexpr int TILE_SIDE_MAX = 448;          // largest solid tile side (byte labels + lists in shared memory)
constexpr int RMT_SMEM_MAX = ((TILE_SIDE_MAX * TILE_SIDE_MAX + 15) & ~15) + 8 * LIST_CAP;
// Force pool, per registered tile, TILE_N values per plane: F_x and F_y of the
// solid terms (without the body force), Delta rho as an unevaluated sum hi + lo
// (two planes' worth, the pair of node lt at POOL_DRHO + 2 lt, read as one
// 64-bit load in FP32; lo = 0 in FP64; in FP32 the pair carries Delta rho to
// ~1e-15, so the SFC equilibrium's rho - rho_t is not rounded against an O(1)
// number), with force_mode 1 only, the blended solid acceleration's y
// component (plane 1 then holds the stress divergence alone), and the
// half-force rho F / 2 of the collision that used the entry (planes 5 and 6,
// written by the LB kernel, read by the next step's moments).
constexpr int POOL_STRIDE = 7 * TILE_N;
constexpr int POOL_FX = 0, POOL_FY = TILE_N, POOL_DRHO = 2 * TILE_N, POOL_AY = 4 * TILE_N;
constexpr int POOL_CX = 5 * TILE_N, POOL_CY = 6 * TILE_N;
// Delta rho (hi, lo) of the pool entry p (p points at the tile's plane 0 + lt)
template <class R> __device__ __forceinline__ void pool_drho(const R *p, int lt, R &hi, R &lo) {
    if constexpr (sizeof(R) == 4) {
        const float2 v = *reinterpret_cast<const float2 *>(p - lt + POOL_DRHO + 2 * lt);
        hi = v.x;
        lo = v.y;
    } else {
        hi = p[POOL_DRHO + lt];
        lo = R(0);
    }
}
// Planes of a solid's tile: eta_x, eta_y and phi; FP32 adds the low parts of
// eta_x and eta_y on the advected nodes (eta = hi + lo), so the rounding of
// the stored reference map does not accumulate over the steps (zero on the
// extrapolated band, which is refitted every step from the advected nodes),
// and the low part of phi in and near the blur zone (phi = hi + lo to ~1e-13,
// for the density difference of Eq. 2_3_drho; zero elsewhere).
template <class R> __host__ __device__ constexpr int xi_planes() { return sizeof(R) == 4 ? 6 : 3; }
// Tie rules shared with the method's definition: a node with |phi| <= PHI_TIE
// is not solid; a directional extrapolation weight with cosine <= COS_TIE is zero.
constexpr double PHI_TIE = 1e-9;
constexpr double COS_TIE = 1e-9;

enum ErrBits : unsigned {
    ERR_NAN = 1u, ERR_TILE_OVERFLOW = 2u, ERR_SLOT_OVERFLOW = 4u, ERR_EXTRAP = 8u,
    ERR_SINGULAR = 16u, ERR_STENCIL = 32u, ERR_OVERFLOW16 = 64u, ERR_TIMEOUT = 128u, ERR_ALIGN = 256u,
    ERR_FREE_REGION = 512u
};

// Scalar parameters, passed by value.
struct SimParams {
    int nx, ny, wall_x, wall_y;
    int ntx, nty;
    int tx, ty, lx, ly;  // registry tile shape and log2 of each side
    int rk, lk, nrx;     // K1 region: rk = 2^lk registry tiles side by side, nrx regions per row
    long long P;  // plane size nx*ny
    double tau, rho_f, lid_u, eps, eta, gravity;
    int force_kind;
    int force_mode;  // 0: Guo term with rho F (Eq. 3_4_Fi as printed); 1: rho on the accelerations only
    double fa0, fa1;
    int n_layers, rmax, kmax, nsolids;
    // FP32 copies (GB300's FP64 pipe is narrow: no per-thread conversions)
    float omega_f, kf_f, rho_f_f, lid_u_f, eps_f, eta_f, fy_f;
    double omega, kf, fy;  // 1/tau, 1 - 1/(2 tau), constant y body force
    // grid of the solid-fraction table (LamEntry): phi_k = (k - lam_k0) lam_h, lam_h a power of two
    float lam_h, lam_inv_h, eps_lo;  // eps_lo = eps - (float)eps
    int lam_k0;
    // 16-bit storage: power-of-two scale (and inverse) per population plane and of the density plane
    float st_scale[9], st_inv[9], ct_scale, ct_inv;
};

// lambda(phi) = 1 - H_eps(phi) (Eq. 2_3_heaviside) and its first five Taylor
// coefficients at the table's grid points, for the FP32 path's Delta rho:
// lambda(phi_k + d) = l0 + l1 d + ... + l5 d^5 (|d| <= lam_h / 2, the next term
// below 1e-16), with l0 and l1 as float pairs.  Built in double on the host from
// the formula of Eq. 2_3_heaviside; it replaces FP64 sin, which this GPU's
// narrow FP64 pipe makes costly, and at 12 KB stays in L1.
struct LamEntry {
    float l0h, l0l, l1h, l1l, l2, l3, l4, l5;
};
constexpr int LAM_TAB_MAX = 513;  // entries (2 lam_k0 + 1)

// K1 walks regions LB_REGION_W nodes wide (rk registry tiles when tile_x is
// narrower): the push stores of a warp then cover long rows, which keeps the
// partial 32-byte sectors at the row ends a small share of the written bytes.
constexpr int LB_REGION_W = 64;
// K1 CTAs per SM the register allocation must allow: memory-latency bound, so
// occupancy buys bandwidth (FP32: 40 registers, 6 CTAs of 256; 16-bit storage
// needs 48 for its conversions, FP64 arithmetic 80)
template <class R, class S> constexpr int LB_MIN_BLOCKS = sizeof(R) == 8 ? 3 : (sizeof(S) == 2 ? 5 : 6);

__host__ __device__ inline void set_tile_params(SimParams &sp, int tx) {
    sp.tx = tx; sp.ty = TILE_N / tx;
    sp.lx = 0; while ((1 << sp.lx) < sp.tx) sp.lx++;
    sp.ly = 0; while ((1 << sp.ly) < sp.ty) sp.ly++;
    sp.ntx = (sp.nx + sp.tx - 1) / sp.tx;
    sp.nty = (sp.ny + sp.ty - 1) / sp.ty;
    sp.rk = tx < LB_REGION_W ? LB_REGION_W / tx : 1;
    sp.lk = 0; while ((1 << sp.lk) < sp.rk) sp.lk++;
    sp.nrx = (sp.ntx + sp.rk - 1) / sp.rk;
}


template <class R> __device__ __forceinline__ R pick(double d, float f);
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }

struct SolidDesc {
    double xc, yc, R, rho_s, G;  // R: disk radius (circumscribed radius of other shapes)
    int shape;                   // 0 disk, 1 axis-aligned ellipse, 2 axis-aligned rectangle
    double a, b;                 // semi-axes / half-sides along x and y
    double eps;                  // the blur-zone half-width (a threshold of the level set)
    double r2lo, drho, accel;   // R^2 - (double)(float)R^2, rho_s - rho_f, -(1 - rho_f/rho_s) g
    float R_f, G_f, r2hi_f, r2lo_f, drho_f, accel_f, Rlo_f, drho_lo_f;  // *_lo_f: the double minus its float
    int T;
    long long off;      // element offset of the tile (eta_x plane, then eta_y plane)
};

// Frame of one buffer of a solid's tile: origin o (global node of tile node
// (0,0), unwrapped) and off, a multiple of 2^-14.  A tile node at local l is the
// grid node x = o + l and stores eta = xi - x + d with d = o - X_c - off, so
// xi - X_c = eta + l + off: l + off is exact in FP32 and d follows the solid's
// mean motion, which keeps eta small.
struct Frame {
    int ox, oy;
    float offx, offy;
    // box (local, inclusive) holding every solid and band node of the tile;
    // values outside it are stale and never read
    short bx0, bx1, by0, by1;
};
__host__ __device__ __forceinline__ bool in_box(const Frame &f, int x, int y) {
    return x >= f.bx0 && x <= f.bx1 && y >= f.by0 && y <= f.by1;
}

// Device pointers of one simulation (type-erased; the kernels cast).
struct DevState {
    void *f[2];            // 9 planes each
    void *carry;           // 1 plane: rho^n - rho_f of the last collision where its
                           // registry did not hold the node's tile (NaN: no collision yet)
    void *xi[2];           // solid tiles
    Frame *frame[2];       // frame of xi[k] per solid
    int *reg_count[2];     // per tile: solids registered
    int *reg_solids[2];    // per tile: KMAX ids
    int *reg_active[2];    // list of tiles with count > 0
    int *reg_nactive[2];
    void *pool[2];         // per tile: POOL_STRIDE values (layout above)
    void *bfield;          // force_kind 3: body force field, x plane then y plane (nx*ny each)
    LamEntry *lamtab;      // solid-fraction table (FP32 arithmetic)
    int *order;            // solids by decreasing tile side (launch order of the solid kernel)
    unsigned char *busy[2]; // per K1 region, by step parity: 1 if it may hold solid forcing this step
    void *fbody;           // per row: body-force x component
    double *mass_partials; // per LB block
    double *stats_step;    // S x 8, stats of the state at the start of the last step
    SolidDesc *solids;
    unsigned *err;
};

// ---------------------------------------------------------------------------
// D2Q9 (Table d2q9): c_q and weights; opposite directions.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int cxq(int q) { return (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0); }
__host__ __device__ __forceinline__ int cyq(int q) { return (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0); }
__device__ __forceinline__ int oppq(int q) { return q == 0 ? 0 : (q <= 4 ? ((q + 1) & 3) + 1 : ((q - 3) & 3) + 5); }
template <class R> __device__ __forceinline__ R wq(int q) { return q == 0 ? R(4) / R(9) : (q <= 4 ? R(1) / R(9) : R(1) / R(36)); }

__device__ __forceinline__ int wrapi(int g, int n) { int r = g % n; return r < 0 ? r + n : r; }
__device__ __forceinline__ int floordiv(int a, int n) { return a >= 0 ? a / n : -((-a + n - 1) / n); }

template <class R> __device__ __forceinline__ R rsin(R x);
template <> __device__ __forceinline__ float rsin<float>(float x) { return sinf(x); }
template <> __device__ __forceinline__ double rsin<double>(double x) { return sin(x); }
template <class R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_<double>(double x) { return sqrt(x); }
template <class R> __device__ __forceinline__ R rcp_rn(R x);
template <> __device__ __forceinline__ float rcp_rn<float>(float x) { return __frcp_rn(x); }
template <> __device__ __forceinline__ double rcp_rn<double>(double x) { return __drcp_rn(x); }
template <class R> __device__ __forceinline__ R nanv();
template <> __device__ __forceinline__ float nanv<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double nanv<double>() { return __longlong_as_double(0x7ff8000000000000ll); }

// Smoothed Heaviside, Eq. 2_3_heaviside.
template <class R> __device__ __forceinline__ R heaviside(R phi, R eps) {
    if (phi <= -eps) return R(0);
    if (phi >= eps) return R(1);
    const R pi = R(3.14159265358979323846);
    return R(0.5) * (R(1) + phi / eps + rsin<R>(pi * phi / eps) / pi);
}

// Level set of a disk in solid-local reference coordinates, phi_0(X) = |X - c| - R.
template <class R> __device__ __forceinline__ R phi_disk(R X, R Y, R rad) { return rsqrt_<R>(X * X + Y * Y) - rad; }

// Storage of the populations and of the density plane (rho - rho_f of the last
// collision, from which the next step rebuilds its half-force term off the
// registered tiles).  FP32/FP64 store the values as they are.  The 16-bit
// variants store value x scale with a power-of-two scale (exact) per population
// plane q and one for the density plane,
// chosen at initialisation from bounds of the values (SimParams::st_scale,
// ct_scale): the largest value the bound admits fills about half of FP16's
// range, so small deviations stay normal numbers; a stored FP16 value beyond
// the range raises an error flag.  (Scaling cannot change the relative
// rounding of a normal number: it only moves the format's range.)
template <class S> __device__ __forceinline__ float to_f(S v) { return (float)v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <class S> __device__ __forceinline__ S from_f(float v) { return S(v); }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <class S> __host__ __device__ constexpr bool is16() { return sizeof(S) == 2; }

// population of plane q
template <class S, class R> __device__ __forceinline__ R ldS(const S *p, const SimParams &sp, int q) {
    if constexpr (is16<S>()) return R(to_f<S>(*p) * sp.st_inv[q]);
    else return R(*p);
}
template <class S, class R> __device__ __forceinline__ void stS(S *p, R v, const SimParams &sp, int q) {
    if constexpr (is16<S>()) *p = from_f<S>(float(v) * sp.st_scale[q]);
    else *p = S(v);
}
// density plane
template <class S, class R> __device__ __forceinline__ R ldC(const S *p, const SimParams &sp) {
    if constexpr (is16<S>()) return R(to_f<S>(*p) * sp.ct_inv);
    else return R(*p);
}
template <class S, class R> __device__ __forceinline__ void stC(S *p, R v, const SimParams &sp) {
    if constexpr (is16<S>()) *p = from_f<S>(float(v) * sp.ct_scale);
    else *p = S(v);
}
// read-only global load of a stored population
template <class S, class R> __device__ __forceinline__ R ldG(const S *p, const SimParams &sp, int q) {
    if constexpr (is16<S>()) return ldS<S, R>(p, sp, q);
    else return R(__ldg(p));
}
// a stored FP16 population of plane q would exceed the format's range
template <class S, class R> __device__ __forceinline__ bool store_overflow(R v, const SimParams &sp, int q) {
    if constexpr (std::is_same<S, __half>::value) return fabsf(float(v)) * sp.st_scale[q] > 60000.0f;
    else return false;
}
// the same for the density plane
template <class S, class R> __device__ __forceinline__ bool store_overflow_c(R v, const SimParams &sp) {
    if constexpr (std::is_same<S, __half>::value) return fabsf(float(v)) * sp.ct_scale > 60000.0f;
    else return false;
}

__device__ __forceinline__ bool allowed_cell(const SimParams &sp, int gx, int gy) {
    if (sp.wall_x && (gx < -2 || gx > sp.nx + 1)) return false;
    if (sp.wall_y && (gy < -2 || gy > sp.ny + 1)) return false;
    return true;
}
__device__ __forceinline__ bool domain_cell(const SimParams &sp, int gx, int gy) {
    if (sp.wall_x && (gx < 0 || gx >= sp.nx)) return false;
    if (sp.wall_y && (gy < 0 || gy >= sp.ny)) return false;
    return true;
}
__device__ __forceinline__ long long grid_index(const SimParams &sp, int gx, int gy) {
    return (long long)wrapi(gy, sp.ny) * sp.nx + wrapi(gx, sp.nx);
}

// Stored populations: g_q = f_q - w_q rho_f for q >= 1 and g_0 = f_0 - w_0 rho_f -
// Delta rho, where Delta rho is the SFC density difference (Eq. 2_3_drho) of the
// step that wrote them (zero off the registered tiles).  At the SFC rest state
// every g_q vanishes, so all nine stored numbers are small deviations.
template <class R>
__device__ __forceinline__ R rest_base(const SimParams &sp, const int *reg, const R *pool, int i, int j) {
    const int tile = (j >> sp.ly) * sp.ntx + (i >> sp.lx);
    return reg[tile] > 0 ? pool[(long long)tile * POOL_STRIDE + POOL_DRHO + 2 * (((j & (sp.ty - 1)) << sp.lx) + (i & (sp.tx - 1)))]
                         : R(0);
}
// The rest base with its low part, in double (readouts and uploads).
template <class R>
__device__ __forceinline__ double rest_base_d(const SimParams &sp, const int *reg, const R *pool, int i, int j) {
    const int tile = (j >> sp.ly) * sp.ntx + (i >> sp.lx);
    if (reg[tile] <= 0) return 0.0;
    const int lt = ((j & (sp.ty - 1)) << sp.lx) + (i & (sp.tx - 1));
    R hi, lo;
    pool_drho<R>(pool + (long long)tile * POOL_STRIDE + lt, lt, hi, lo);
    return (double)hi + (double)lo;
}

// a - b as an unevaluated sum: s = fl(a - b) and its exact error e, a - b = s + e
// (Knuth's two-sum, branch-free).
template <class R>
__device__ __forceinline__ R two_diff(R a, R b, R &e) {
    const R s = a - b;
    const R bb = s - a;
    e = (a - (s - bb)) - (b + bb);
    return s;
}

// Moments of node (i, j): rho and v = (sum c_q f_q + rho^{n-1} F^{n-1} / 2) / rho.
// reg/pool: registry and force pool of the step that wrote the populations.
// rho and v from the stored populations fq, the rest base dro and the half-force term (cx, cy).
template <class R>
__device__ __forceinline__ void moments_from(const SimParams &sp, const R (&fq)[9], R dro, R cx, R cy, R &rho, R &u,
                                             R &v) {
    R dr = dro + (((fq[0] + fq[1]) + (fq[2] + fq[3])) + ((fq[4] + fq[5]) + (fq[6] + fq[7])) + fq[8]);
    R jx = (fq[1] - fq[3]) + (fq[5] - fq[6]) + (fq[8] - fq[7]);
    R jy = (fq[2] - fq[4]) + (fq[5] - fq[7]) + (fq[6] - fq[8]);
    rho = pick<R>(sp.rho_f, sp.rho_f_f) + dr;
    R inv = rcp_rn<R>(rho);  // as the LB kernel
    u = (jx + cx) * inv;
    v = (jy + cy) * inv;
}

// Body force of node c in row j (Eq. 2_4_F_divs' f): the per-node field of
// force_kind 3, else the per-row x component and the constant y component.
template <class R>
__device__ __forceinline__ void body_force(const SimParams &sp, const R *fbody, const R *bfield, int j, long long c,
                                           R &Fx, R &Fy) {
    if (sp.force_kind == 3) {
        Fx = bfield[c];
        Fy = bfield[sp.P + c];
    } else {
        Fx = fbody[j];
        Fy = pick<R>(sp.fy, sp.fy_f);
    }
}

// Half-force term rho^{n-1} F^{n-1} / 2 of the moments (Sec. 3.4) at a node
// whose tile the previous step's registry did not hold: that step's force was
// the body force alone (Fx, Fy: the field is the same at every step) and its
// density rho_f + drp, so the product is the one the LB kernel formed then, to
// the bit.  (On registered tiles the pool holds the product itself, planes
// POOL_CX / POOL_CY.)  drp NaN: the populations have no previous collision
// (initialisation, an upload), and the term is zero.
template <class R>
__device__ __forceinline__ void free_carry(const SimParams &sp, R drp, R Fx, R Fy, R &cx, R &cy) {
    const R rho = pick<R>(sp.rho_f, sp.rho_f_f) + drp;
    const bool none = !(drp == drp);
    cx = none ? R(0) : R(0.5) * rho * Fx;
    cy = none ? R(0) : R(0.5) * rho * Fy;
}

// The half-force term of node (i, j), c = j nx + i: from the pool of the
// registry reg where it holds the node's tile, else from the density plane.
template <class R, class S>
__device__ __forceinline__ void node_carry(const SimParams &sp, const S *carry, const R *fbody, const R *bfield,
                                           const int *reg, const R *pool, int i, int j, long long c, R &cx, R &cy) {
    const int tile = (j >> sp.ly) * sp.ntx + (i >> sp.lx);
    if (reg[tile] > 0) {
        const R *po = pool + (long long)tile * POOL_STRIDE + (((j & (sp.ty - 1)) << sp.lx) + (i & (sp.tx - 1)));
        cx = po[POOL_CX];
        cy = po[POOL_CY];
    } else {
        R Fx, Fy;
        body_force<R>(sp, fbody, bfield, j, c, Fx, Fy);
        free_carry<R>(sp, ldC<S, R>(carry + c, sp), Fx, Fy, cx, cy);
    }
}

template <class R, class S>
__device__ __forceinline__ void node_moments(const SimParams &sp, const S *f, const S *carry, const R *fbody,
                                             const R *bfield, const int *reg, const R *pool, int i, int j, R &rho,
                                             R &u, R &v) {
    const long long c = (long long)j * sp.nx + i;
    R fq[9];
#pragma unroll
    for (int q = 0; q < 9; q++) fq[q] = ldS<S, R>(f + q * sp.P + c, sp, q);
    R cx, cy;
    node_carry<R, S>(sp, carry, fbody, bfield, reg, pool, i, j, c, cx, cy);
    moments_from<R>(sp, fq, rest_base<R>(sp, reg, pool, i, j), cx, cy, rho, u, v);
}

// Block-wide sum of NV values (blockDim.x multiple of 32, <= 1024).
template <class T, int NV>
__device__ void block_sum(T (&v)[NV], T *sh /* 32*NV */) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
        for (int k = 0; k < NV; k++) sh[warp * NV + k] = v[k];
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < NV; k++) {
            T t = lane < nw ? sh[lane * NV + k] : T(0);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            v[k] = t;
        }
    }
}

// ===========================================================================
// K2: reference-map advection, extrapolation and relabel, one CTA per solid.
// ===========================================================================
template <class R, class S>
struct RmtArgs {
    const S *f;          // populations f^n
    const S *carry;      // density plane of the step that wrote f^n
    const R *fbody, *bfield;  // body force (per row; per node with force_kind 3)
    const int *reg_prev; // registry and pool of the step that wrote f^n
    const R *pool_prev;
    const R *xi_in;      // xi^n tiles (unused at init)
    R *xi_out;           // xi^{n+1} tiles
    const Frame *frame_in;
    Frame *frame_out;    // origin read at entry; its box is written at exit
    Frame *frame_next;   // frame of the next step's output tile
    int *reg_count, *reg_solids, *reg_active, *reg_nactive;
    double *stats;       // S x 8 (state at time n), may be null at init
    const SolidDesc *solids;
    const int *order;    // CTA -> solid (largest tiles first), or null
    unsigned *err;
    int init;
};

// 2^{-k} exactly, k in [0, 60].
template <class R> __device__ __forceinline__ R pow2neg(int k);
template <> __device__ __forceinline__ float pow2neg<float>(int k) { return __int_as_float((127 - k) << 23); }
template <> __device__ __forceinline__ double pow2neg<double>(int k) {
    return __longlong_as_double((long long)(1023 - k) << 52);
}

// 1/|d| for |dx|, |dy| <= RMAX_TAB (filled by the host at configuration).
constexpr int RMAX_TAB = 20;
__constant__ float c_rinv_f[(RMAX_TAB + 1) * (RMAX_TAB + 1)];
__constant__ double c_rinv_d[(RMAX_TAB + 1) * (RMAX_TAB + 1)];
// The tables live in each translation unit that includes this header: every
// unit that launches a kernel reading them fills its own copy with this.
static inline cudaError_t upload_rinv_tables() {
    float tf[(RMAX_TAB + 1) * (RMAX_TAB + 1)];
    double td[(RMAX_TAB + 1) * (RMAX_TAB + 1)];
    for (int i = 0; i <= RMAX_TAB; i++)
        for (int j = 0; j <= RMAX_TAB; j++) {
            const double r2 = (double)(i * i + j * j);
            td[i * (RMAX_TAB + 1) + j] = r2 > 0 ? 1.0 / sqrt(r2) : 0.0;
            tf[i * (RMAX_TAB + 1) + j] = (float)td[i * (RMAX_TAB + 1) + j];
        }
    cudaError_t e = cudaMemcpyToSymbol(c_rinv_f, tf, sizeof(tf));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_rinv_d, td, sizeof(td));
}
template <class R> __device__ __forceinline__ R rinv_tab(int dx, int dy);
template <> __device__ __forceinline__ float rinv_tab<float>(int dx, int dy) { return c_rinv_f[abs(dx) * (RMAX_TAB + 1) + abs(dy)]; }
template <> __device__ __forceinline__ double rinv_tab<double>(int dx, int dy) { return c_rinv_d[abs(dx) * (RMAX_TAB + 1) + abs(dy)]; }

// Running sums of one weighted least-squares fit.  The positive-weight nodes
// are collinear iff the Gram determinant of their integer offsets vanishes,
// (n Sxx - Sx^2)(n Syy - Sy^2) - (n Sxy - Sx Sy)^2 = 0, an exact integer test.
template <class R>
struct Lsq {
    int nvalid, n, sx, sy, sxx, syy, sxy;
    bool haveref;
    R a, b, c, d, e, fw;            // M = [[a b c],[b d e],[c e fw]]
    R bx0, bx1, bx2, by0, by1, by2; // right-hand sides for eta_x - xref and eta_y - yref
    R xref, yref;                   // values of the first valid node (fit of differences)
};

template <class R>
__device__ __forceinline__ void lsq_cell(Lsq<R> &A, const signed char *lab, const R *X, const R *Y, int k, int l, int dx,
                                         int dy, bool use_n, R nhx, R nhy) {
    const int L = lab[k];
    if (!(L >= 0 && L < l)) return;
    A.nvalid++;
    R wt = pow2neg<R>(abs(dx) + abs(dy));  // 2^{-(r_i + r_j)}
    if (use_n) {
        const R dn = (R(-dx) * nhx + R(-dy) * nhy) * rinv_tab<R>(dx, dy);  // d = target - node
        wt = dn > R(COS_TIE) ? dn * wt : R(0);
    }
    if (!(wt > R(0))) return;
    A.n++; A.sx += dx; A.sy += dy; A.sxx += dx * dx; A.syy += dy * dy; A.sxy += dx * dy;
    R Xv = X[k], Yv = Y[k];
    if (!A.haveref) { A.xref = Xv; A.yref = Yv; A.haveref = true; }
    Xv -= A.xref; Yv -= A.yref;
    const R x = R(dx), y = R(dy);
    const R wx = wt * x, wy = wt * y;
    A.a += wx * x; A.b += wx * y; A.c += wx; A.d += wy * y; A.e += wy; A.fw += wt;
    A.bx0 += wx * Xv; A.bx1 += wy * Xv; A.bx2 += wt * Xv;
    A.by0 += wx * Yv; A.by1 += wy * Yv; A.by2 += wt * Yv;
}

// The 5x5 window of a target away from the tile edge, without branches on
// the node's validity (weights are zero for the nodes that do not count).
template <class R, bool USE_N>
__device__ __forceinline__ void lsq_window5(Lsq<R> &A, const signed char *lab, const R *X, const R *Y, int t, int T,
                                            int l, R nhx, R nhy) {
#pragma unroll
    for (int dy = -2; dy <= 2; dy++)
#pragma unroll
        for (int dx = -2; dx <= 2; dx++) {
            if (dx == 0 && dy == 0) continue;  // the target itself (layer l) never counts
            const int k = t + dy * T + dx;
            const int L = lab[k];
            const bool valid = (unsigned)L < (unsigned)l;  // 0 <= L < l
            R wt = valid ? pow2neg<R>(abs(dx) + abs(dy)) : R(0);
            if (USE_N) {
                const R dn = (R(-dx) * nhx + R(-dy) * nhy) * rinv_tab<R>(dx, dy);
                wt = dn > R(COS_TIE) ? dn * wt : R(0);
            }
            A.nvalid += valid ? 1 : 0;
            const bool pos = wt > R(0);
            A.n += pos ? 1 : 0;
            A.sx += pos ? dx : 0; A.sy += pos ? dy : 0;
            A.sxx += pos ? dx * dx : 0; A.syy += pos ? dy * dy : 0; A.sxy += pos ? dx * dy : 0;
            R Xv = R(0), Yv = R(0);
            if (pos) { Xv = X[k] - A.xref; Yv = Y[k] - A.yref; }
            const R wx = wt * R(dx), wy = wt * R(dy);
            A.a += wx * R(dx); A.b += wx * R(dy); A.c += wx; A.d += wy * R(dy); A.e += wy; A.fw += wt;
            A.bx0 += wx * Xv; A.bx1 += wy * Xv; A.bx2 += wt * Xv;
            A.by0 += wx * Yv; A.by1 += wy * Yv; A.by2 += wt * Yv;
        }
}

// The 5x5 window without directional weights (layers beyond the second): the
// weights 2^{-(|dx|+|dy|)} then depend only on which of the 24 nodes are valid,
// so the sums of M and of the collinearity test follow from each row's 5-bit
// validity mask by bit counts.  Every term is a multiple of 1/16, so these sums
// are exact, as the running sums of lsq_window5 are; only the right-hand sides
// read the nodes' values, accumulated in the same node order.
template <class R>
__device__ __forceinline__ void lsq_window5_mask(Lsq<R> &A, const signed char *lab, const R *X, const R *Y, int t,
                                                 int T, int l) {
    int n = 0, sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0;
    int a16 = 0, b16 = 0, c16 = 0, d16 = 0, e16 = 0, f16 = 0;  // 16 x the entries of M
    unsigned rows = 0;                                         // 5 bits per row, dx = -2..2
#pragma unroll
    for (int dy = -2; dy <= 2; dy++) {
        unsigned r = 0;
#pragma unroll
        for (int dx = -2; dx <= 2; dx++) {
            if (dx == 0 && dy == 0) continue;  // the target itself (layer l) never counts
            const int L = lab[t + dy * T + dx];
            r |= ((unsigned)L < (unsigned)l ? 1u : 0u) << (dx + 2);
        }
        rows |= r << (5 * (dy + 2));
        const int c0 = (r >> 2) & 1, p1 = __popc(r & 0x0au), p2 = __popc(r & 0x11u);
        const int d1 = (int)((r >> 3) & 1) - (int)((r >> 1) & 1), d2 = (int)((r >> 4) & 1) - (int)(r & 1);
        const int nr = c0 + p1 + p2, sxr = d1 + 2 * d2;
        // row sums of 4 2^{-|dx|} dx^k (k = 0, 1, 2), row weight 4 2^{-|dy|}
        const int s0 = 4 * c0 + 2 * p1 + p2, s1 = 2 * d1 + 2 * d2, s2 = 2 * p1 + 4 * p2;
        const int g = dy == 0 ? 4 : (dy == 1 || dy == -1 ? 2 : 1);
        n += nr; sx += sxr; sxx += p1 + 4 * p2; sy += dy * nr; syy += dy * dy * nr; sxy += dy * sxr;
        f16 += g * s0; c16 += g * s1; a16 += g * s2; e16 += g * dy * s0; d16 += g * dy * dy * s0; b16 += g * dy * s1;
    }
    A.nvalid += n; A.n += n; A.sx += sx; A.sy += sy; A.sxx += sxx; A.syy += syy; A.sxy += sxy;
    const R q = R(0.0625);
    A.a += R(a16) * q; A.b += R(b16) * q; A.c += R(c16) * q; A.d += R(d16) * q; A.e += R(e16) * q; A.fw += R(f16) * q;
#pragma unroll
    for (int dy = -2; dy <= 2; dy++)
#pragma unroll
        for (int dx = -2; dx <= 2; dx++) {
            if (dx == 0 && dy == 0) continue;
            if (!((rows >> (5 * (dy + 2) + dx + 2)) & 1u)) continue;
            const int k = t + dy * T + dx;
            const R Xv = X[k] - A.xref, Yv = Y[k] - A.yref;
            const R w = pow2neg<R>((dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy));
            const R wx = w * R(dx), wy = w * R(dy);
            A.bx0 += wx * Xv; A.bx1 += wy * Xv; A.bx2 += w * Xv;
            A.by0 += wx * Yv; A.by1 += wy * Yv; A.by2 += w * Yv;
        }
}

// Weighted least-squares fit of one target (Sec. 3.2, steps (i)-(iii)).  The
// weights do not depend on the window size, so growing r from r-1 only adds
// the ring |dx| = r or |dy| = r to the sums of the smaller window.  The fit is
// of differences from the value at the target's 4-neighbour in layer l - 1
// (a valid node by construction), which keeps the sums small.
template <class R>
__device__ void extrapolate_target(const SimParams &sp, const signed char *lab, R *X, R *Y, int T, int tx, int ty,
                                   int l, bool use_n, R nhx, R nhy, unsigned *err) {
    const int t = ty * T + tx;
    Lsq<R> A;
    A.nvalid = A.n = A.sx = A.sy = A.sxx = A.syy = A.sxy = 0;
    A.a = A.b = A.c = A.d = A.e = A.fw = R(0);
    A.bx0 = A.bx1 = A.bx2 = A.by0 = A.by1 = A.by2 = R(0);
    {
        int kref = t + T;
        if (tx > 0 && lab[t - 1] == l - 1) kref = t - 1;
        else if (tx < T - 1 && lab[t + 1] == l - 1) kref = t + 1;
        else if (ty > 0 && lab[t - T] == l - 1) kref = t - T;
        A.xref = X[kref];
        A.yref = Y[kref];
        A.haveref = true;
    }
    if (tx >= 2 && ty >= 2 && tx < T - 2 && ty < T - 2) {
        if (use_n) lsq_window5<R, true>(A, lab, X, Y, t, T, l, nhx, nhy);
        else lsq_window5_mask<R>(A, lab, X, Y, t, T, l);
    } else {
        for (int dy = -2; dy <= 2; dy++)
            for (int dx = -2; dx <= 2; dx++)
                if (tx + dx >= 0 && ty + dy >= 0 && tx + dx < T && ty + dy < T)
                    lsq_cell<R>(A, lab, X, Y, t + dy * T + dx, l, dx, dy, use_n, nhx, nhy);
    }
    for (int r = 2; r <= sp.rmax; r++) {
        if (r > 2) {
            for (int q = -r; q <= r; q++) {
                const int ring[4][2] = {{q, -r}, {q, r}, {-r, q}, {r, q}};
                for (int m = 0; m < 4; m++) {
                    if (m >= 2 && (q == -r || q == r)) continue;  // corners counted once
                    const int dx = ring[m][0], dy = ring[m][1];
                    if (tx + dx >= 0 && ty + dy >= 0 && tx + dx < T && ty + dy < T)
                        lsq_cell<R>(A, lab, X, Y, t + dy * T + dx, l, dx, dy, use_n, nhx, nhy);
                }
            }
        }
        if (A.nvalid < 3 || A.n < 3) continue;
        const long long g1 = (long long)A.n * A.sxx - (long long)A.sx * A.sx;
        const long long g2 = (long long)A.n * A.syy - (long long)A.sy * A.sy;
        const long long g3 = (long long)A.n * A.sxy - (long long)A.sx * A.sy;
        if (g1 * g2 - g3 * g3 == 0) continue;  // positive-weight nodes on one line
        // third row of M^{-1} from the cofactors of the symmetric M
        const R c13 = A.b * A.e - A.c * A.d, c23 = A.b * A.c - A.a * A.e, c33 = A.a * A.d - A.b * A.b;
        const R det = A.a * (A.d * A.fw - A.e * A.e) - A.b * (A.b * A.fw - A.c * A.e) + A.c * (A.b * A.e - A.c * A.d);
        if (!(det != R(0))) continue;
        X[t] = A.xref + (c13 * A.bx0 + c23 * A.bx1 + c33 * A.bx2) / det;
        Y[t] = A.yref + (c13 * A.by0 + c23 * A.by1 + c33 * A.by2) / det;
        return;
    }
    atomicOr(err, ERR_EXTRAP);
    X[t] = nanv<R>();
    Y[t] = nanv<R>();
}

template <class R> __device__ __forceinline__ R mul_rn(R a, R b);
template <> __device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <class R> __device__ __forceinline__ R add_rn(R a, R b);
template <> __device__ __forceinline__ float add_rn<float>(float a, float b) { return __fadd_rn(a, b); }
template <> __device__ __forceinline__ double add_rn<double>(double a, double b) { return __dadd_rn(a, b); }
template <class R> __device__ __forceinline__ R fma_rn(R a, R b, R c);
template <> __device__ __forceinline__ float fma_rn<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double fma_rn<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// R^2 as an unevaluated sum hi + lo in precision R (from the host-side split).
template <class R>
struct Rsq {
    R hi, lo, rad;
    int shape;
    double a, b, eps;
    __device__ __forceinline__ Rsq() {}
    __device__ __forceinline__ explicit Rsq(const SolidDesc &sd) {
        hi = pick<R>(sd.R * sd.R, sd.r2hi_f);
        lo = pick<R>(0.0, sd.r2lo_f);
        rad = pick<R>(sd.R, sd.R_f);
        shape = sd.shape;
        a = sd.a;
        b = sd.b;
        eps = sd.eps;
    }
};

// Distance from (y0, y1) >= 0 to the ellipse (x/e0)^2 + (y/e1)^2 = 1, e0 >= e1:
// the closest point is e_i^2 y_i / (t + e_i^2) for the root t of
// sum (e_i y_i / (t + e_i^2))^2 = 1 (Eberly's characterisation).  In s = t / e1^2
// the function is decreasing and convex on the bracket [z1 - 1, s1], so Newton
// steps from the bracket's left end (where it is >= 0) rise monotonically to the
// root; they stop when they no longer move or leave the bracket.
__device__ inline double ellipse_distance_q1(double e0, double e1, double y0, double y1) {
    if (y1 > 0.0) {
        if (y0 > 0.0) {
            const double z0 = y0 / e0, z1 = y1 / e1, g = z0 * z0 + z1 * z1 - 1.0;
            if (g == 0.0) return 0.0;
            const double r0 = (e0 / e1) * (e0 / e1), n0 = r0 * z0;
            const double hi = g < 0.0 ? 0.0 : hypot(n0, z1) - 1.0;
            double s = z1 - 1.0;
            for (int it = 0; it < 100; it++) {
                const double ia = 1.0 / (s + r0), ib = 1.0 / (s + 1.0);
                const double ra = n0 * ia, rb = z1 * ib, f = ra * ra + rb * rb - 1.0;
                if (!(f > 0.0)) break;
                const double df = -2.0 * (ra * ra * ia + rb * rb * ib);
                const double sn = s - f / df;
                if (!(sn > s) || sn > hi) break;
                s = sn;
            }
            return hypot(r0 * y0 / (s + r0) - y0, y1 / (s + 1.0) - y1);
        }
        return fabs(y1 - e1);
    }
    const double num = e0 * y0, den = e0 * e0 - e1 * e1;
    if (num < den) {
        const double x = num / den;
        return hypot(e0 * x - y0, e1 * sqrt(1.0 - x * x));
    }
    return fabs(y0 - e0);
}

// The same distance with the root found in FP32 (the same monotone Newton
// steps), for FP32 simulations (their stored level set is FP32; GB300's FP64
// pipe is narrow).  The FP32 distance is within ~1e-6 of the exact one; where
// that could move a node across a threshold of the method (phi = 0, the solid
// set; phi = eps, the blur zone) -- within `shell` of either -- the root is
// polished by two Newton steps in double and the distance formed in double.
__device__ inline double ellipse_distance_q1_mixed(double e0, double e1, double y0, double y1, double eps,
                                                   double shell) {
    if (!(y1 > 0.0 && y0 > 0.0)) return ellipse_distance_q1(e0, e1, y0, y1);  // no iteration on the axes
    const double z0 = y0 / e0, z1 = y1 / e1, g = z0 * z0 + z1 * z1 - 1.0;
    if (g == 0.0) return 0.0;
    const double r0 = (e0 / e1) * (e0 / e1), n0 = r0 * z0;
    const double hi = g < 0.0 ? 0.0 : hypot(n0, z1) - 1.0;
    const float r0f = (float)r0, n0f = (float)n0, z1f = (float)z1, hif = (float)hi;
    // FP32 steps with CUDA's fast division (the iteration corrects its own rounding)
    float s = z1f - 1.0f;
    for (int it = 0; it < 100; it++) {
        const float ia = __fdividef(1.0f, s + r0f), ib = __fdividef(1.0f, s + 1.0f);
        const float ra = n0f * ia, rb = z1f * ib, f = ra * ra + rb * rb - 1.0f;
        if (!(f > 0.0f)) break;
        const float df = -2.0f * (ra * ra * ia + rb * rb * ib);
        const float sn = s - __fdividef(f, df);
        if (!(sn > s) || sn > hif) break;
        s = sn;
    }
    const float y0f = (float)y0, y1f = (float)y1;
    const float df32 = hypotf(__fdividef(r0f * y0f, s + r0f) - y0f, __fdividef(y1f, s + 1.0f) - y1f);
    if (fabsf(df32) >= (float)shell && fabsf(df32 - (float)eps) >= (float)shell) return (double)df32;
    double sd = (double)s;
    for (int it = 0; it < 2; it++) {
        const double ia = 1.0 / (sd + r0), ib = 1.0 / (sd + 1.0);
        const double ra = n0 * ia, rb = z1 * ib, f = ra * ra + rb * rb - 1.0;
        const double dfd = -2.0 * (ra * ra * ia + rb * rb * ib);
        const double sn = sd - f / dfd;
        if (sn == sn && sn >= z1 - 1.0 && sn <= (hi > 0.0 ? hi : 0.0)) sd = sn;
    }
    return hypot(r0 * y0 / (sd + r0) - y0, y1 / (sd + 1.0) - y1);
}

// Signed distance (negative inside) of q (relative to the centre) to the
// axis-aligned ellipse (shape 1, semi-axes a, b) or rectangle (shape 2,
// half-sides a, b), in double precision.
__device__ inline double shape_sdf(int shape, double a, double b, double qx, double qy) {
    if (shape == 2) {
        const double dx = fabs(qx) - a, dy = fabs(qy) - b;
        return hypot(fmax(dx, 0.0), fmax(dy, 0.0)) + fmin(fmax(dx, dy), 0.0);
    }
    double y0 = fabs(qx), y1 = fabs(qy), e0 = a, e1 = b;
    if (e0 < e1) {
        double t = e0; e0 = e1; e1 = t;
        t = y0; y0 = y1; y1 = t;
    }
    const double d = ellipse_distance_q1(e0, e1, y0, y1);
    return (y0 / e0) * (y0 / e0) + (y1 / e1) * (y1 / e1) < 1.0 ? -d : d;
}

// shape_sdf with the ellipse distance of ellipse_distance_q1_mixed (FP32 simulations).
__device__ inline double shape_sdf_mixed(int shape, double a, double b, double qx, double qy, double eps) {
    if (shape == 2) return shape_sdf(shape, a, b, qx, qy);
    double y0 = fabs(qx), y1 = fabs(qy), e0 = a, e1 = b;
    if (e0 < e1) {
        double t = e0; e0 = e1; e1 = t;
        t = y0; y0 = y1; y1 = t;
    }
    const double d = ellipse_distance_q1_mixed(e0, e1, y0, y1, eps, 1e-3);
    return (y0 / e0) * (y0 / e0) + (y1 / e1) * (y1 / e1) < 1.0 ? -d : d;
}

// The same with the root polished in double wherever the distance is below
// eps + shell (the blur zone and a shell around it): there the result is
// exact to ~1e-13, for the level set's low part.
__device__ inline double shape_sdf_polished(int shape, double a, double b, double qx, double qy, double eps,
                                            double shell) {
    if (shape == 2) return shape_sdf(shape, a, b, qx, qy);
    double y0 = fabs(qx), y1 = fabs(qy), e0 = a, e1 = b;
    if (e0 < e1) {
        double t = e0; e0 = e1; e1 = t;
        t = y0; y0 = y1; y1 = t;
    }
    // polish below eps + shell: the shell argument covers [0, eps + shell] around zero
    const double d = ellipse_distance_q1_mixed(e0, e1, y0, y1, 0.0, eps + shell);
    return (y0 / e0) * (y0 / e0) + (y1 / e1) * (y1 / e1) < 1.0 ? -d : d;
}

// Level set phi_0 of a disk at a tile node: with p = l + off (exact) and eta,
// phi = |p + eta| - R = (|p|^2 - R^2 + 2 p.eta + |eta|^2) / (|p + eta| + R),
// where |p|^2 - R^2 is formed with error-free products and a two-sum, so
// phi keeps its relative precision near the interface.
template <class R>
__device__ __forceinline__ R phi_eta(R ex, R ey, int lx, int ly, const Frame &fr, const Rsq<R> &q) {
    if (q.shape != 0) {  // ellipses and rectangles: q = eta + l + off, exact in double
        const double X = ((double)lx + (double)fr.offx) + (double)ex, Y = ((double)ly + (double)fr.offy) + (double)ey;
        return R(sizeof(R) == 4 ? shape_sdf_mixed(q.shape, q.a, q.b, X, Y, q.eps) : shape_sdf(q.shape, q.a, q.b, X, Y));
    }
    const R px = add_rn<R>(R(lx), R(fr.offx)), py = add_rn<R>(R(ly), R(fr.offy));  // exact
    const R a = mul_rn<R>(px, px), ea = fma_rn<R>(px, px, -a);
    const R b = mul_rn<R>(py, py), eb = fma_rn<R>(py, py, -b);
    const R s2 = add_rn<R>(a, b);
    const R bv = add_rn<R>(s2, -a);
    const R es = add_rn<R>(add_rn<R>(a, -add_rn<R>(s2, -bv)), add_rn<R>(b, -bv));
    const R pq = add_rn<R>(s2, -q.hi) + (((ea + eb) + es) - q.lo);
    const R num = pq + (R(2) * (px * ex + py * ey) + (ex * ex + ey * ey));
    const R X = px + ex, Y = py + ey;
    return num / (rsqrt_<R>(X * X + Y * Y) + q.rad);
}

// s = fl(a + b) and its exact error e (Knuth's two-sum).
__device__ __forceinline__ float two_sum_f(float a, float b, float &e) {
    const float s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}

// phi_0 of a tile node as a float pair ph + pl (error ~1e-14): for a disk,
// phi = (|p|^2 - R^2) / (|p| + R) with p = (l + off) + eta (hi + lo), in
// float-float arithmetic; other shapes take the signed distance in double.
__device__ __forceinline__ void phi_node_ff(float ex, float ey, float exl, float eyl, int lx, int ly, const Frame &fr,
                                            const Rsq<float> &q, float Rlo, float &ph, float &pl) {
    if (q.shape != 0) {
        const double X = ((double)lx + (double)fr.offx) + ((double)ex + (double)exl);
        const double Y = ((double)ly + (double)fr.offy) + ((double)ey + (double)eyl);
        const double d = shape_sdf(q.shape, q.a, q.b, X, Y);
        ph = (float)d;
        pl = (float)(d - (double)ph);
        return;
    }
    float e;
    const float pxh = two_sum_f(__fadd_rn((float)lx, fr.offx), ex, e), pxl = e + exl;
    const float pyh = two_sum_f(__fadd_rn((float)ly, fr.offy), ey, e), pyl = e + eyl;
    const float a = __fmul_rn(pxh, pxh), ea = __fmaf_rn(pxh, pxh, -a);
    const float b = __fmul_rn(pyh, pyh), eb = __fmaf_rn(pyh, pyh, -b);
    float es;
    const float sh = two_sum_f(a, b, es);
    const float sl = ((es + ea) + eb) + 2.0f * (pxh * pxl + pyh * pyl);  // |p|^2 = sh + sl
    float en;
    const float nh = two_sum_f(sh, -q.hi, en);
    const float nl = en + (sl - q.lo);                                   // |p|^2 - R^2 = nh + nl
    const float r = __fsqrt_rn(sh);
    const float rl = (__fmaf_rn(-r, r, sh) + sl) / (2.0f * r);           // |p| = r + rl
    float ed;
    const float dh = two_sum_f(r, q.rad, ed), dl = ed + (rl + Rlo);      // |p| + R = dh + dl
    const float q1 = __fdiv_rn(nh, dh);
    const float p1 = __fmul_rn(q1, dh), ep1 = __fmaf_rn(q1, dh, -p1);
    const float res = (((nh - p1) - ep1) + nl) - q1 * dl;                // num - q1 den
    const float q2 = res / dh;
    ph = q1 + q2;
    pl = q2 - (ph - q1);
}

// lambda = 1 - H_eps(phi) for phi = ph + pl as a float pair lh + ll, from the
// table (FP32 path).
__device__ __forceinline__ void lambda_ff(const SimParams &sp, const LamEntry *tab, float ph, float pl, float &lh,
                                          float &ll) {
    // the thresholds of Eq. 2_3_heaviside, exactly: phi + eps and phi - eps as
    // float sums (ph -/+ eps_hi is exact near the threshold, Sterbenz)
    if ((ph + sp.eps_f) + (pl + sp.eps_lo) <= 0.0f) { lh = 1.0f; ll = 0.0f; return; }
    if ((ph - sp.eps_f) + (pl - sp.eps_lo) >= 0.0f) { lh = 0.0f; ll = 0.0f; return; }
    const int k = (int)rintf(ph * sp.lam_inv_h);
    const LamEntry t = tab[k + sp.lam_k0];
    const float dh = ph - (float)k * sp.lam_h;  // exact: phi_k is a multiple of lam_h within lam_h / 2 of ph
    const float d = dh + pl;
    const float p = __fmul_rn(dh, t.l1h), ep = __fmaf_rn(dh, t.l1h, -p);
    const float rest = (((ep + dh * t.l1l) + pl * t.l1h) + t.l0l) + d * d * (t.l2 + d * (t.l3 + d * (t.l4 + d * t.l5)));
    float e;
    const float s = two_sum_f(t.l0h, p, e);
    const float lo = e + rest;
    lh = s + lo;
    ll = lo - (lh - s);
}

// Float-float accumulation: (h, l) += (a, b); (h, l) += (a, b) (c, d); (h, l) /= (a, b).
__device__ __forceinline__ void ff_add(float &h, float &l, float a, float b) {
    float e;
    const float s = two_sum_f(h, a, e);
    const float t = e + (l + b);
    h = s + t;
    l = t - (h - s);
}
__device__ __forceinline__ void ff_add_prod(float &h, float &l, float a, float b, float c, float d) {
    const float p = __fmul_rn(a, c), ep = __fmaf_rn(a, c, -p);
    ff_add(h, l, p, ep + (a * d + b * c));
}
__device__ __forceinline__ void ff_div(float &h, float &l, float a, float b) {
    const float q1 = __fdiv_rn(h, a);
    const float p = __fmul_rn(q1, a), ep = __fmaf_rn(q1, a, -p);
    const float r = (((h - p) - ep) + l) - q1 * b;
    const float q2 = r / a;
    h = q1 + q2;
    l = q2 - (h - q1);
}

// Half-width of the shell around the blur zone where K3 takes lambda to ~1e-13.
constexpr float PHI_D_SHELL = 1e-3f;

// d = o - X_c - off of a frame, in double.
__device__ __forceinline__ double frame_d(const Frame &fr, double c, bool xdir) {
    return xdir ? (double)fr.ox - c - (double)fr.offx : (double)fr.oy - c - (double)fr.offy;
}

// off for origin o and displacement estimate d: o - X_c - d on the 2^-14 grid.
__device__ __forceinline__ float frame_off(int o, double c, double d) {
    return (float)(rint(((double)o - c - d) * 16384.0) / 16384.0);
}

__device__ __forceinline__ void warp_minmax(int &v, bool is_min) {
    const unsigned u = (unsigned)(v + (1 << 30));  // shift to non-negative for the unsigned reduction
    const unsigned r = is_min ? __reduce_min_sync(0xffffffffu, u) : __reduce_max_sync(0xffffffffu, u);
    v = (int)r - (1 << 30);
}

// Disjoint ranges of tile indices (side 2^shift, ntiles per row or column) that
// cover the node interval [lo, hi] of one axis of extent n: clipped at walls,
// wrapped (and merged where the two wrapped pieces share tiles) when periodic.
__device__ __forceinline__ int tile_ranges(int lo, int hi, int n, int wall, int shift, int ntiles, int r0[2],
                                           int r1[2]) {
    if (wall) {
        lo = max(lo, 0);
        hi = min(hi, n - 1);
        if (lo > hi) return 0;
        r0[0] = lo >> shift; r1[0] = hi >> shift;
        return 1;
    }
    if (hi - lo + 1 >= n) { r0[0] = 0; r1[0] = ntiles - 1; return 1; }
    const int k0 = floordiv(lo, n), k1 = floordiv(hi, n);
    const int a = (lo - k0 * n) >> shift, b = (hi - k1 * n) >> shift;
    if (k0 == k1) { r0[0] = a; r1[0] = b; return 1; }
    if (b + 1 >= a) { r0[0] = 0; r1[0] = ntiles - 1; return 1; }
    r0[0] = 0; r1[0] = b; r0[1] = a; r1[1] = ntiles - 1;
    return 2;
}

// Row-major walk of a w-wide box by a CTA: (c, r) of item k, advanced by blockDim.x items at a time.
struct BoxWalk {
    int c, r, dc, dr, w;
    __device__ __forceinline__ BoxWalk(int w_) : w(w_ > 0 ? w_ : 1) {
        c = threadIdx.x % w; r = threadIdx.x / w; dc = blockDim.x % w; dr = blockDim.x / w;
    }
    __device__ __forceinline__ void next() { c += dc; r += dr; if (c >= w) { c -= w; r++; } }
};

// Layers 1..NL around the solid set S (label 0) in a tile's label bytes (-1
// free): layer l = the allowed nodes l 4-neighbour dilation steps from S (Sec.
// 3.2; nodes beyond the pad of a no-slip side never count).  The allowed cells
// of a tile form a rectangle, where that number of steps is the L1 distance to
// S, so the labels come from a separable L1 distance transform in place on the
// label bytes, over the box of S grown by NL: a sweep per row, then one per
// column (distances capped at NL + 1), then the nodes beyond NL or outside the
// allowed cells are freed again.  cnt (shared, may be null): per-layer counts
// are added to cnt[1..NL].  The caller synchronises before reading the labels.
__device__ __forceinline__ void label_layers_l1(const SimParams &sp, signed char *lab, int T, int sx0, int sx1,
                                                int sy0, int sy1, int2 oo, int NL, int *cnt) {
    const int x0 = max(sx0 - NL, 0), x1 = min(sx1 + NL, T - 1), y0 = max(sy0 - NL, 0), y1 = min(sy1 + NL, T - 1);
    const int cap = NL + 1;
    for (int y = y0 + (int)threadIdx.x; y <= y1; y += blockDim.x) {
        signed char *row = lab + y * T;
        int last = -(1 << 20);
        for (int x = x0; x <= x1; x++) {
            if (row[x] == 0) last = x;
            else row[x] = (signed char)min(x - last, cap);
        }
        last = 1 << 20;
        for (int x = x1; x >= x0; x--) {
            if (row[x] == 0) last = x;
            else row[x] = (signed char)min((int)row[x], min(last - x, cap));
        }
    }
    __syncthreads();
    for (int x = x0 + (int)threadIdx.x; x <= x1; x += blockDim.x) {
        int d = cap;
        for (int y = y0; y <= y1; y++) {
            signed char *q = lab + y * T + x;
            d = min((int)*q, d + 1);
            *q = (signed char)d;
        }
        d = cap;
        for (int y = y1; y >= y0; y--) {
            signed char *q = lab + y * T + x;
            d = min((int)*q, d + 1);
            *q = (signed char)d;
        }
    }
    __syncthreads();
    const int w = x1 - x0 + 1, n = w * (y1 - y0 + 1);
    BoxWalk wk(w);
    for (int k = threadIdx.x; k < n; k += blockDim.x, wk.next()) {
        const int lx = x0 + wk.c, ly = y0 + wk.r, t = ly * T + lx;
        const int d = lab[t];
        if (d < 1) continue;
        if (d <= NL && allowed_cell(sp, oo.x + lx, oo.y + ly)) {
            if (cnt) atomicAdd(&cnt[d], 1);
        } else {
            lab[t] = -1;
        }
    }
}

// The nodes of layers 1..NL (labelled, in the box [x0, x1] x [y0, y1]) in one
// list, layer l at lists[loff[l] .. loff[l + 1]) (packed lx | ly << 16), so
// that a layer's targets fill whole warps.  cnt holds the per-layer counts of
// label_layers_l1 and is used up.  False (and no list) when more than cap
// nodes; the caller then scans the tile for each layer.  Synchronises.
__device__ __forceinline__ bool list_layers(const signed char *lab, int T, int x0, int x1, int y0, int y1, int NL,
                                            int *cnt, int *loff, int *lists, int cap) {
    if (threadIdx.x == 0) {
        loff[1] = 0;
        for (int l = 1; l <= NL; l++) {
            loff[l + 1] = loff[l] + cnt[l];
            cnt[l] = loff[l];
        }
    }
    __syncthreads();
    const bool listed = loff[NL + 1] <= cap;
    if (listed) {
        const int w = x1 - x0 + 1, n = w * (y1 - y0 + 1);
        BoxWalk wk(w);
        for (int k = threadIdx.x; k < n; k += blockDim.x, wk.next()) {
            const int lx = x0 + wk.c, ly = y0 + wk.r;
            const int d = lab[ly * T + lx];
            if (d >= 1) lists[atomicAdd(&cnt[d], 1)] = lx | (ly << 16);
        }
    }
    __syncthreads();
    return listed;
}

// One node of pass 0 (advection): its stored state and the LB state at it,
// gathered with independent loads (the rest base is loaded whatever the
// registry count and selected after).
template <class R>
struct P0Node {
    int ix, iy, cnt;
    R ex, ey, phi, cx, cy, pv;
    R f[9];
};

template <class R, class S>
__device__ __forceinline__ void p0_gather(const SimParams &sp, const RmtArgs<R, S> &a, const R *Xi, const R *Yi,
                                          const R *Pi, int T, int2 oo, int shx, int shy, int entry, P0Node<R> &nd) {
    nd.ix = entry & 0xffff;
    nd.iy = entry >> 16;
    const int k = nd.iy * T + nd.ix;
    const int i = wrapi(oo.x + nd.ix - shx, sp.nx), j = wrapi(oo.y + nd.iy - shy, sp.ny);
    const long long c = (long long)j * sp.nx + i;
    const int tile = (j >> sp.ly) * sp.ntx + (i >> sp.lx);
    nd.ex = Xi[k];
    nd.ey = Yi[k];
    nd.phi = Pi[k];
#pragma unroll
    for (int q = 0; q < 9; q++) nd.f[q] = ldS<S, R>(a.f + q * sp.P + c, sp, q);
    nd.cnt = a.reg_prev[tile];
    // rest base and half-force term from the pool (its address is valid whether
    // or not the tile is registered; every node listed here is: see p0_finish)
    const int lt = ((j & (sp.ty - 1)) << sp.lx) + (i & (sp.tx - 1));
    const R *po = a.pool_prev + (long long)tile * POOL_STRIDE + lt;
    nd.pv = po[POOL_DRHO + lt];  // hi part of the (hi, lo) pair of node lt
    nd.cx = po[POOL_CX];
    nd.cy = po[POOL_CY];
}

// The rest of pass 0 for a gathered node of the blur zone or the solid:
// statistics, and for a solid node the upwind advection (Eqs. 3_1_refmap_adv,
// 3_1_eno) into the output tile.
template <class R, class S>
__device__ __forceinline__ void p0_finish(const SimParams &sp, const RmtArgs<R, S> &a, const P0Node<R> &nd,
                                          const R *Xi, const R *Yi, R *Xo, R *Yo, signed char *lab, int T,
                                          const Frame &fi, int2 oo, int shx, int shy, R ddx, R ddy, R eps, R (&stl)[6],
                                          int (&sb)[4]) {
    const int ix = nd.ix, iy = nd.iy, lx = ix - shx, ly = iy - shy;
    R rho, u, v, cx = nd.cx, cy = nd.cy;
    if (nd.cnt <= 0) {
        // Not expected: the previous registry covers the blur zone of phi^n grown
        // by one node, which holds every node listed here.  Then the half-force
        // term comes from the density plane and the body force.
        const int i = wrapi(oo.x + ix - shx, sp.nx), j = wrapi(oo.y + iy - shy, sp.ny);
        const long long c = (long long)j * sp.nx + i;
        R Fx, Fy;
        body_force<R>(sp, a.fbody, a.bfield, j, c, Fx, Fy);
        free_carry<R>(sp, ldC<S, R>(a.carry + c, sp), Fx, Fy, cx, cy);
    }
    moments_from<R>(sp, nd.f, nd.cnt > 0 ? nd.pv : R(0), cx, cy, rho, u, v);
    const R lam = R(1) - heaviside<R>(nd.phi, eps);
    stl[0] += lam; stl[1] += lam * R(lx); stl[2] += lam * R(ly);
    stl[3] += lam * rho; stl[4] += lam * rho * u; stl[5] += lam * rho * v;
    if (!(nd.phi < -R(PHI_TIE))) return;
    const int sx = (u >= R(0)) ? -1 : 1, sy = (v >= R(0)) ? -1 : 1;
    const int x2 = ix + 2 * sx, y2 = iy + 2 * sy;
    if (x2 < fi.bx0 || x2 > fi.bx1 || y2 < fi.by0 || y2 > fi.by1) {
        atomicOr(a.err, ERR_STENCIL);
        return;
    }
    const int k = iy * T + ix;
    const int k1 = k + sx, k2 = k + 2 * sx, k3 = k + sy * T, k4 = k + 2 * sy * T;
    const R X1 = Xi[k1], X2 = Xi[k2], X3 = Xi[k3], X4 = Xi[k4];
    const R Y1 = Yi[k1], Y2 = Yi[k2], Y3 = Yi[k3], Y4 = Yi[k4];
    // the low parts of eta (FP32) follow the phi plane; loaded with the stencil
    const R exl = xi_planes<R>() == 6 ? Xi[3 * T * T + k] : R(0);
    const R eyl = xi_planes<R>() == 6 ? Xi[4 * T * T + k] : R(0);
    if (!(X1 == X1 && X2 == X2 && X3 == X3 && X4 == X4)) atomicOr(a.err, ERR_STENCIL);
    // one-sided second-order differences of eta; xi = eta + position adds (1,0)/(0,1)
    const R ex = nd.ex, ey = nd.ey;
    const R hx = R(-sx) * R(0.5), hy = R(-sy) * R(0.5);
    const R dXdx = hx * (R(3) * ex - R(4) * X1 + X2), dYdx = hx * (R(3) * ey - R(4) * Y1 + Y2);
    const R dXdy = hy * (R(3) * ex - R(4) * X3 + X4), dYdy = hy * (R(3) * ey - R(4) * Y3 + Y4);
    // xi = eta + x - d: the node's own motion enters as -(u - dd)
    const int t = ly * T + lx;
    if constexpr (xi_planes<R>() == 6) {
        // eta^{n+1} = (hi + lo) + dd - (u + u.grad eta) in float-float: the frame
        // shift dd and the update enter with their exact rounding errors, so
        // hi + lo carries eta to ~u_32^2 and only the small update rounds
        const R dX = u + (u * dXdx + v * dXdy), dY = v + (u * dYdx + v * dYdy);
        R e1, e2;
        R s1 = two_diff<R>(ex, -ddx, e1);
        R s2 = two_diff<R>(s1, dX, e2);
        R tl = (e1 + e2) + exl;
        R hi = s2 + tl;
        Xo[t] = hi;
        Xo[3 * T * T + t] = tl - (hi - s2);
        s1 = two_diff<R>(ey, -ddy, e1);
        s2 = two_diff<R>(s1, dY, e2);
        tl = (e1 + e2) + eyl;
        hi = s2 + tl;
        Yo[t] = hi;
        Xo[4 * T * T + t] = tl - (hi - s2);
    } else {
        Xo[t] = ex - (u - ddx) - (u * dXdx + v * dXdy);
        Yo[t] = ey - (v - ddy) - (u * dYdx + v * dYdy);
    }
    lab[t] = 0;
    sb[0] = min(sb[0], lx); sb[1] = max(sb[1], lx); sb[2] = min(sb[2], ly); sb[3] = max(sb[3], ly);
}

template <class R, class S>
__device__ void rmt_solid(const SimParams &sp, const RmtArgs<R, S> &a, const int s) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int lcnt[24];  // per layer: node count, then the next free list slot
    __shared__ int loff[24];  // per layer: first list slot (layer l at loff[l] .. loff[l + 1])
    __shared__ int bb[12];    // S bbox (0-3), band bbox (4-7), blur-zone bbox (8-11)
    __shared__ double red[32 * 6];
    __syncthreads();  // the shared state of a previous solid is no longer read
    const SolidDesc sd = a.solids[s];
    const int T = sd.T, TT = T * T;
    const int lane = threadIdx.x & 31;
    signed char *lab = reinterpret_cast<signed char *>(smem);        // -1 free, 0 solid, l layer
    // after the labels, the rest of the launch's dynamic shared memory holds
    // ints: pass 0's per-warp node lists, then the layer lists
    int *lists = reinterpret_cast<int *>(smem + ((TT + 15) & ~15));
    unsigned dsm;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsm));
    const int list_cap = ((int)dsm - ((TT + 15) & ~15)) >> 2;
    const Frame fo = a.frame_out[s];
    const Frame fi = a.init ? fo : a.frame_in[s];
    const int2 oo = make_int2(fo.ox, fo.oy);
    const int shx = fo.ox - fi.ox, shy = fo.oy - fi.oy;  // same node: local index shifts by this
    // eta_out = eta_in + (d_out - d_in); exact (integer part plus multiples of 2^-14)
    const R ddx = R((double)shx - ((double)fo.offx - (double)fi.offx));
    const R ddy = R((double)shy - ((double)fo.offy - (double)fi.offy));
    const Rsq<R> rq(sd);
    R *Xo = a.xi_out + sd.off;
    R *Yo = Xo + TT;
    R *Po = Yo + TT;  // phi^{n+1} of the tile nodes (third plane), written by the relabel
    const R *Xi = a.init ? nullptr : a.xi_in + sd.off;
    const R *Yi = a.init ? nullptr : Xi + TT;
    const R *Pi = a.init ? nullptr : Yi + TT;  // phi^n, stored by the previous step's relabel
    const R eps = pick<R>(sp.eps, sp.eps_f);
    if (threadIdx.x < 12) bb[threadIdx.x] = (threadIdx.x & 1) ? -(1 << 29) : (1 << 29);
    if (threadIdx.x < 24) lcnt[threadIdx.x] = 0;
    for (int k = threadIdx.x; k < (TT + 15) >> 4; k += blockDim.x)
        reinterpret_cast<int4 *>(lab)[k] = make_int4(-1, -1, -1, -1);
    R stl[6] = {0, 0, 0, 0, 0, 0};  // sum lambda, lambda lx, lambda ly, lambda rho, lambda rho u, lambda rho v
    int sb[4] = {1 << 29, -(1 << 29), 1 << 29, -(1 << 29)};
    __syncthreads();

    // Pass 0: the advected set S = {domain nodes with phi^n < 0}, Eqs. 3_1_refmap_adv / 3_1_eno,
    // over the input tile's box (the whole tile at initialisation).
    const int ib0 = a.init ? 0 : fi.bx0, ib1 = a.init ? T - 1 : fi.bx1;
    const int jb0 = a.init ? 0 : fi.by0, jb1 = a.init ? T - 1 : fi.by1;
    const int bw = ib1 - ib0 + 1, bn = (ib1 >= ib0 && jb1 >= jb0) ? bw * (jb1 - jb0 + 1) : 0;
    if (a.init) {
        BoxWalk wk(bw);
        for (int kk = threadIdx.x; kk < bn; kk += blockDim.x, wk.next()) {
            const int ix = ib0 + wk.c, iy = jb0 + wk.r;  // input-tile coordinates
            const int lx = ix - shx, ly = iy - shy;      // output-tile coordinates
            const int gx = oo.x + lx, gy = oo.y + ly;
            // xi = x: eta = d of the initial frame
            const R e0x = R(frame_d(fo, sd.xc, true)), e0y = R(frame_d(fo, sd.yc, false));
            if (domain_cell(sp, gx, gy) && phi_eta(e0x, e0y, lx, ly, fo, rq) < -R(PHI_TIE)) {
                const int t = ly * T + lx;
                Xo[t] = e0x; Yo[t] = e0y; lab[t] = 0;
                sb[0] = min(sb[0], lx); sb[1] = max(sb[1], lx); sb[2] = min(sb[2], ly); sb[3] = max(sb[3], ly);
            }
        }
    } else {
        // (a) each warp lists, in box order, the nodes of its share of the box
        // (items threadIdx.x + m blockDim.x) that lie in the blur zone or the
        // solid, in its own segment of the (not yet used) layer lists; (b) it
        // advances them two per lane at a time, every load of both nodes issued
        // before the arithmetic -- at the end of its share, or earlier whenever
        // the segment could overflow, after which the listing goes on.
        const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5;
        const int seg_cap = list_cap / nw;
        int *seg = lists + warp * seg_cap;
        if (seg_cap >= 128) {
            // (four of a thread's items at a time: their phi loads first, then the
            // ballots in item order, which add at most 128 entries)
            int base = 0;
            do {
                int nseg = 0;
                for (; base < bn && nseg <= seg_cap - 128; base += 4 * blockDim.x) {
                    R ph[4];
                    int ent[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int kk = base + q * (int)blockDim.x + (int)threadIdx.x;
                        const int ix = ib0 + kk % bw, iy = jb0 + kk / bw;
                        ent[q] = ix | (iy << 16);
                        ph[q] = kk < bn ? Pi[iy * T + ix] : eps;
                    }
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        bool hit = false;
                        if (ph[q] < eps) {
                            const int lx = (ent[q] & 0xffff) - shx, ly = (ent[q] >> 16) - shy;
                            if (domain_cell(sp, oo.x + lx, oo.y + ly)) {
                                if (lx < 0 || ly < 0 || lx >= T || ly >= T) atomicOr(a.err, ERR_TILE_OVERFLOW);
                                else hit = true;
                            }
                        }
                        const unsigned m = __ballot_sync(0xffffffffu, hit);
                        if (hit) seg[nseg + __popc(m & ((1u << lane) - 1u))] = ent[q];
                        nseg += __popc(m);
                    }
                }
                __syncwarp();
                for (int e = lane; e < nseg; e += 64) {
                    const bool two = e + 32 < nseg;
                    P0Node<R> n1, n2;
                    p0_gather<R, S>(sp, a, Xi, Yi, Pi, T, oo, shx, shy, seg[e], n1);
                    p0_gather<R, S>(sp, a, Xi, Yi, Pi, T, oo, shx, shy, seg[two ? e + 32 : e], n2);
                    p0_finish<R, S>(sp, a, n1, Xi, Yi, Xo, Yo, lab, T, fi, oo, shx, shy, ddx, ddy, eps, stl, sb);
                    if (two)
                        p0_finish<R, S>(sp, a, n2, Xi, Yi, Xo, Yo, lab, T, fi, oo, shx, shy, ddx, ddy, eps, stl, sb);
                }
                __syncwarp();
            } while (base < bn);
        } else {
            // segments too small to list four ballots: each thread walks its share
            BoxWalk wk2(bw);
            for (int kk = threadIdx.x; kk < bn; kk += blockDim.x, wk2.next()) {
                const int ix = ib0 + wk2.c, iy = jb0 + wk2.r;
                const int lx = ix - shx, ly = iy - shy;
                if (!(Pi[iy * T + ix] < eps) || !domain_cell(sp, oo.x + lx, oo.y + ly)) continue;
                if (lx < 0 || ly < 0 || lx >= T || ly >= T) {
                    atomicOr(a.err, ERR_TILE_OVERFLOW);
                    continue;
                }
                P0Node<R> nd;
                p0_gather<R, S>(sp, a, Xi, Yi, Pi, T, oo, shx, shy, ix | (iy << 16), nd);
                p0_finish<R, S>(sp, a, nd, Xi, Yi, Xo, Yo, lab, T, fi, oo, shx, shy, ddx, ddy, eps, stl, sb);
            }
        }
    }
    for (int k = 0; k < 4; k++) warp_minmax(sb[k], (k & 1) == 0);
    if (lane == 0) {
        atomicMin(&bb[0], sb[0]); atomicMax(&bb[1], sb[1]); atomicMin(&bb[2], sb[2]); atomicMax(&bb[3], sb[3]);
    }
    __syncthreads();

    // Layers 1..n_layers around S (Sec. 3.2; 11 layers, Sec. 4), labelled at once
    // (label_layers_l1), then listed by a counting pass and fitted one after
    // another, each from S and the layers before it.
    const int sx0 = bb[0], sx1 = bb[1], sy0 = bb[2], sy1 = bb[3];
    if (sx0 > sx1) {
        if (threadIdx.x == 0) atomicOr(a.err, ERR_TILE_OVERFLOW);  // the solid vanished
    }
    const int NL = sp.n_layers;
    bool listed = false;  // every layer's nodes are in the lists (else each layer scans the tile)
    if (sx0 <= sx1) {
        const int x0 = max(sx0 - NL, 0), x1 = min(sx1 + NL, T - 1), y0 = max(sy0 - NL, 0), y1 = min(sy1 + NL, T - 1);
        label_layers_l1(sp, lab, T, sx0, sx1, sy0, sy1, oo, NL, lcnt);
        __syncthreads();
        listed = list_layers(lab, T, x0, x1, y0, y1, NL, lcnt, loff, lists, list_cap);
    }
    for (int l = 1; l <= NL && sx0 <= sx1; l++) {
        const int nitems = listed ? loff[l + 1] - loff[l] : TT;
        for (int k = threadIdx.x; k < nitems; k += blockDim.x) {
            int lx, ly;
            if (listed) {
                const int e = lists[loff[l] + k];
                lx = e & 0xffff; ly = e >> 16;
            } else {  // too many band nodes for the lists: scan the tile
                lx = k % T; ly = k / T;
                if (lab[k] != l) continue;
            }
            const int t = ly * T + lx;
            if (a.init) {  // xi = x on the band at initialisation
                Xo[t] = R(frame_d(fo, sd.xc, true));
                Yo[t] = R(frame_d(fo, sd.yc, false));
                continue;
            }
            bool use_n = false;
            R nhx = 0, nhy = 0;
            if (l <= 2) {
                // surface normal: central difference of phi^n at the target (input frame)
                const int ix = lx + shx, iy = ly + shy;
                if (ix > fi.bx0 && iy > fi.by0 && ix < fi.bx1 && iy < fi.by1) {
                    const int k0 = iy * T + ix;
                    const R Xe = Xi[k0 + 1], Xw = Xi[k0 - 1], Xn = Xi[k0 + T], Xs = Xi[k0 - T];
                    if (Xe == Xe && Xw == Xw && Xn == Xn && Xs == Xs) {
                        const R pe = Pi[k0 + 1], pw = Pi[k0 - 1], pn = Pi[k0 + T], ps = Pi[k0 - T];
                        const R gxp = (pe - pw) / R(2), gyp = (pn - ps) / R(2);
                        const R nn = rsqrt_<R>(gxp * gxp + gyp * gyp);
                        if (nn > R(0)) { use_n = true; nhx = gxp / nn; nhy = gyp / nn; }
                    }
                }
            }
            extrapolate_target<R>(sp, lab, Xo, Yo, T, lx, ly, l, use_n, nhx, nhy, a.err);
        }
        __syncthreads();
    }

    // Relabel phi^{n+1} = phi_0(xi^{n+1}) over the box that can hold band nodes
    // (layer l lies within l of the solid bbox); band and blur-zone bboxes;
    // invalidate the free nodes of the box.
    int bx[8] = {1 << 29, -(1 << 29), 1 << 29, -(1 << 29), 1 << 29, -(1 << 29), 1 << 29, -(1 << 29)};
    if (sx0 <= sx1) {
        const int x0 = max(sx0 - sp.n_layers, 0), x1 = min(sx1 + sp.n_layers, T - 1);
        const int y0 = max(sy0 - sp.n_layers, 0), y1 = min(sy1 + sp.n_layers, T - 1);
        const int w = x1 - x0 + 1, n = w * (y1 - y0 + 1);
        BoxWalk wk(w);
        for (int k = threadIdx.x; k < n; k += blockDim.x, wk.next()) {
            const int lx = x0 + wk.c, ly = y0 + wk.r, t = ly * T + lx;
            if (lab[t] >= 0) {
                bx[0] = min(bx[0], lx); bx[1] = max(bx[1], lx); bx[2] = min(bx[2], ly); bx[3] = max(bx[3], ly);
                R phi = phi_eta(Xo[t], Yo[t], lx, ly, fo, rq);
                if constexpr (xi_planes<R>() == 6) {
                    // FP32: the level set as a float pair hi + lo in and near the blur
                    // zone (the stresses and sets read hi; the density difference both)
                    R exl = R(0), eyl = R(0);
                    if (a.init || lab[t] > 0) {
                        // the next step advects only nodes within a layer of this
                        // step's solid (interfaces move less than one node per step):
                        // their extrapolated eta has no low part
                        if (a.init || lab[t] <= 2) {
                            Xo[3 * TT + t] = R(0);
                            Xo[4 * TT + t] = R(0);
                        }
                    } else {
                        exl = Xo[3 * TT + t];  // the advection's low parts
                        eyl = Xo[4 * TT + t];
                    }
                    if (phi > -eps - R(PHI_D_SHELL) && phi < eps + R(PHI_D_SHELL)) {
                        R pl;
                        if (rq.shape == 0) {
                            phi_node_ff(Xo[t], Yo[t], exl, eyl, lx, ly, fo, rq, sd.Rlo_f, phi, pl);
                        } else {
                            const double X = ((double)lx + (double)fo.offx) + ((double)Xo[t] + (double)exl);
                            const double Y = ((double)ly + (double)fo.offy) + ((double)Yo[t] + (double)eyl);
                            const double dd = shape_sdf_polished(rq.shape, rq.a, rq.b, X, Y, sp.eps, PHI_D_SHELL);
                            phi = R(dd);
                            pl = R(dd - (double)phi);
                        }
                        Xo[5 * TT + t] = pl;  // read only where |phi| < eps + PHI_D_SHELL
                    }
                }
                Po[t] = phi;
                if (phi < eps) {
                    bx[4] = min(bx[4], lx); bx[5] = max(bx[5], lx); bx[6] = min(bx[6], ly); bx[7] = max(bx[7], ly);
                }
            } else {
                Xo[t] = nanv<R>();
                Yo[t] = nanv<R>();
                Po[t] = nanv<R>();
            }
        }
    }
    for (int k = 0; k < 8; k++) warp_minmax(bx[k], (k & 1) == 0);
    if (lane == 0)
        for (int k = 0; k < 8; k += 2) { atomicMin(&bb[4 + k], bx[k]); atomicMax(&bb[5 + k], bx[k + 1]); }
    // the solid's sums (its mean velocity sets the next frame's offset): in the
    // arithmetic precision (the terms are; FP64 is a narrow pipe on this GPU)
    double st[6];
    if (a.stats) block_sum<R, 6>(stl, reinterpret_cast<R *>(red));
    for (int k = 0; k < 6; k++) st[k] = (double)stl[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        if (a.stats) {
            double *o = a.stats + 8 * s;
            const double L = st[0];
            o[0] = L; o[1] = oo.x + st[1] / L; o[2] = oo.y + st[2] / L; o[3] = st[3]; o[4] = st[4]; o[5] = st[5];
            o[6] = 0; o[7] = 0;
        }
        int2 nx = oo;
        // mean velocity of the solid at time n (zero at initialisation) moves d
        double ux = 0.0, uy = 0.0;
        if (a.stats && st[3] > 0.0) { ux = st[4] / st[3]; uy = st[5] / st[3]; }
        Frame fb = fo;
        if (bb[4] > bb[5]) {
            atomicOr(a.err, ERR_TILE_OVERFLOW);
            fb.bx0 = fb.by0 = 1; fb.bx1 = fb.by1 = 0;
        } else {
            if (bb[4] < 1 || bb[6] < 1 || bb[5] > T - 2 || bb[7] > T - 2) atomicOr(a.err, ERR_TILE_OVERFLOW);
            fb.bx0 = (short)bb[4]; fb.bx1 = (short)bb[5]; fb.by0 = (short)bb[6]; fb.by1 = (short)bb[7];
            // centre the next frame on the solid (not on its band, which walls clip): the
            // frame then follows the solid's translation and eta stays small
            if (bb[0] <= bb[1]) {
                nx.x = oo.x + (bb[0] + bb[1]) / 2 - T / 2;
                nx.y = oo.y + (bb[2] + bb[3]) / 2 - T / 2;
            }
        }
        a.frame_out[s] = fb;
        Frame fn;
        fn.ox = nx.x;
        fn.oy = nx.y;
        fn.offx = frame_off(nx.x, sd.xc, frame_d(fo, sd.xc, true) + ux);
        fn.offy = frame_off(nx.y, sd.yc, frame_d(fo, sd.yc, false) + uy);
        fn.bx0 = fn.by0 = 1; fn.bx1 = fn.by1 = 0;  // filled by the step that writes that tile
        a.frame_next[s] = fn;
    }
    // Register the tiles that the blur zone (grown by one node) touches, each once.
    if (bb[8] <= bb[9]) {
        int rx0[2], rx1[2], ry0[2], ry1[2];
        const int nrx = tile_ranges(oo.x + bb[8] - 1, oo.x + bb[9] + 1, sp.nx, sp.wall_x, sp.lx, sp.ntx, rx0, rx1);
        const int nry = tile_ranges(oo.y + bb[10] - 1, oo.y + bb[11] + 1, sp.ny, sp.wall_y, sp.ly, sp.nty, ry0, ry1);
        for (int ay = 0; ay < nry; ay++)
            for (int ax = 0; ax < nrx; ax++) {
                const int tx0 = rx0[ax], ty0 = ry0[ay];
                const int ntxr = rx1[ax] - tx0 + 1, nall = ntxr * (ry1[ay] - ty0 + 1);
                for (int k = threadIdx.x; k < nall; k += blockDim.x) {
                    const int tile = (ty0 + k / ntxr) * sp.ntx + tx0 + k % ntxr;
                    const int slot = atomicAdd(&a.reg_count[tile], 1);
                    if (slot < sp.kmax) a.reg_solids[tile * KMAX + slot] = s;
                    else atomicOr(a.err, ERR_SLOT_OVERFLOW);
                    if (slot == 0) a.reg_active[atomicAdd(a.reg_nactive, 1)] = tile;
                }
            }
    }
}

template <class R, class S>
__global__ void __launch_bounds__(RMT_THREADS, sizeof(R) == 4 ? RMT_MIN_BLOCKS : 2) rmt_solid_kernel(SimParams sp, RmtArgs<R, S> a) {
    rmt_solid<R, S>(sp, a, a.order ? a.order[blockIdx.x] : (int)blockIdx.x);
}

// The same with 1024-thread CTAs, for simulations with fewer solids than SMs:
// each solid's layer chain then runs on four times the threads.  Same register
// budget as the 256-thread kernel (64), hence the same instructions per node.
constexpr int RMT_THREADS_BIG = 1024;
template <class R, class S>
__global__ void __launch_bounds__(RMT_THREADS_BIG, 1) rmt_solid_kernel_big(SimParams sp, RmtArgs<R, S> a) {
    rmt_solid<R, S>(sp, a, a.order ? a.order[blockIdx.x] : (int)blockIdx.x);
}

// ===========================================================================
// K3: stress divergence, contact and node terms per registered tile.
// ===========================================================================
template <class R>
struct ForceArgs {
    const R *xi;          // xi^{n+1} tiles
    const Frame *frame;   // their frames
    const int *reg_count, *reg_solids, *reg_active, *reg_nactive;
    R *pool;
    const SolidDesc *solids;
    const LamEntry *lamtab;
    unsigned *err;
};

// Half-edge Jacobian of Eq. 3_3_refmap_jacobian from a 2x3 stencil: a = the
// node on the low side of the edge, b = the high side, k = 0,1,2 across.
template <class R>
__device__ __forceinline__ void edge_grad(const R a0, const R a1, const R a2, const R b0, const R b1, const R b2,
                                          R &dn, R &dt) {
    dn = b1 - a1;
    dt = (b2 + a2 - b0 - a0) / R(4);
}

// Neo-Hookean plane-strain deviatoric stress, Eq. 3_3_solid_stress, for the
// Jacobian J = d xi / dx = I + A.  Evaluated in the algebraically identical
// small-strain form: with delta = det J - 1 = tr A + det A,
//   F - I = (adj J - det J I) / det J = D,   E = F F^T - I = D + D^T + D D^T,
//   tau = G (E - tr(E)/3 I),
// so no O(1) terms cancel when the strain is small.
template <class R>
__device__ __forceinline__ bool stress_from_grad(R Axx, R Axy, R Ayx, R Ayy, R G, R &txx, R &txy, R &tyy) {
    const R dl = (Axx + Ayy) + (Axx * Ayy - Axy * Ayx);
    const R det = R(1) + dl;
    if (det == R(0)) return false;
    const R inv = R(1) / det;
    const R Dxx = (Ayy - dl) * inv, Dxy = -Axy * inv, Dyx = -Ayx * inv, Dyy = (Axx - dl) * inv;
    const R Exx = R(2) * Dxx + (Dxx * Dxx + Dxy * Dxy);
    const R Exy = (Dxy + Dyx) + (Dxx * Dyx + Dxy * Dyy);
    const R Eyy = R(2) * Dyy + (Dyx * Dyx + Dyy * Dyy);
    txx = G * (R(2) * Exx - Eyy) / R(3);
    txy = G * Exy;
    tyy = G * (R(2) * Eyy - Exx) / R(3);
    return true;
}

// Per-tile constants of the registered solids (static shared memory of K3).
// Threads per CTA of K3: the 2 tx ty + tx + ty half-edges of a 16x16 tile
// (544) take two rounds of 288 threads where 256 threads need three.  Four
// such CTAs fit an SM (48 registers); the overlapped step launches three per
// SM so that the free regions' K1 runs beside them.  The node phase uses the
// first TILE_N threads.
constexpr int K3_THREADS = TILE_N + 32;

template <class R>
struct ForceShared {
    int ids[KMAX];
    int nk;
    Frame sfr[KMAX];
    R sG[KMAX], sD[KMAX], sA[KMAX];
    float sDh[KMAX], sDl[KMAX];  // rho_s - rho_f as a float pair (the FP32 node terms' Delta rho)
    Rsq<R> srq[KMAX];
    int sT[KMAX];
    long long soff[KMAX];
};

// Dynamic shared memory of K3 for a tile shape: xi_x, xi_y, phi per slot on the
// tile plus a one-node halo, and three stress components per half-edge.
__host__ __device__ __forceinline__ int force_patch_n(int tx, int ty) { return (tx + 2) * (ty + 2); }
__host__ __device__ __forceinline__ int force_smem_elems(int tx, int ty) {
    return 3 * KMAX * force_patch_n(tx, ty) + 3 * ((tx + 1) * ty + tx * (ty + 1));
}
__host__ __device__ __forceinline__ int force_smem_max() {
    int m = 0;
    for (int tx = 16; tx <= 128; tx *= 2) m = force_smem_elems(tx, TILE_N / tx) > m ? force_smem_elems(tx, TILE_N / tx) : m;
    return m;
}

// The registered solids of a tile and their descriptors into fs, read by one
// whole warp (lane k: registry slot k) in parallel; slot = rank of the id (ids
// are distinct): a fixed summation order.
template <class R>
__device__ __forceinline__ void force_solids(const SimParams &sp, const ForceArgs<R> &a, const int tile,
                                             ForceShared<R> &fs, const int k) {
    const int n = min(a.reg_count[tile], sp.kmax);
    const int id = k < n ? a.reg_solids[tile * KMAX + k] : 0x7fffffff;
    int rank = 0;
#pragma unroll
    for (int m = 0; m < KMAX; m++) rank += __shfl_sync(0xffffffffu, id, m) < id ? 1 : 0;
    if (k < n) {
        const SolidDesc &sd = a.solids[id];
        fs.ids[rank] = id;
        fs.sfr[rank] = a.frame[id];
        fs.sG[rank] = pick<R>(sd.G, sd.G_f);
        fs.sD[rank] = pick<R>(sd.drho, sd.drho_f);
        fs.sA[rank] = pick<R>(sd.accel, sd.accel_f);
        fs.sDh[rank] = sd.drho_f;
        fs.sDl[rank] = sd.drho_lo_f;
        fs.srq[rank] = Rsq<R>(sd);
        fs.sT[rank] = sd.T;
        fs.soff[rank] = sd.off;
    }
    if (k == 0) fs.nk = n;
}

// One registered tile of K3.  LOADED: fs already holds the tile's solids (read
// during the previous tile); else the first warp reads them.  next >= 0: the
// warp beyond the tile's TILE_N node threads reads the solids of tile `next`
// into fs_next during the node phase, where it has no node (blockDim.x >=
// TILE_N + 32).
template <class R, bool LOADED = false>
__device__ void force_tile(const SimParams &sp, const ForceArgs<R> &a, const int tile, ForceShared<R> &fs, R *dyn,
                           const int next = -1, ForceShared<R> *fs_next = nullptr) {
    const int TX = sp.tx, PX = TX + 2, PN = force_patch_n(TX, sp.ty);
    const int NXE = (TX + 1) * sp.ty, NYE = TX * (sp.ty + 1);
    R *sX = dyn;                       // [KMAX][PN]
    R *sY = sX + KMAX * PN;
    R *sP = sY + KMAX * PN;
    R *eT = sP + KMAX * PN;            // [(NXE + NYE) * 3] edge stresses
    int *ids = fs.ids;
    Frame *sfr = fs.sfr;
    R *sG = fs.sG, *sD = fs.sD, *sA = fs.sA;
    Rsq<R> *srq = fs.srq;
    int *sT = fs.sT;
    long long *soff = fs.soff;
    const R eps = pick<R>(sp.eps, sp.eps_f), eta = pick<R>(sp.eta, sp.eta_f);
    {
        const int tx = tile % sp.ntx, ty = tile / sp.ntx;
        const int i0 = tx * TX, j0 = ty * sp.ty;
        if (!LOADED) {
            if (threadIdx.x < 32) force_solids<R>(sp, a, tile, fs, threadIdx.x);
            __syncthreads();
        }
        const int n = fs.nk;
        // Stage each solid's xi (and phi) on the tile plus a one-node halo.
        for (int ks = 0; ks < n; ks++) {
            const Frame fr = sfr[ks];
            const int T = sT[ks];
            const R *Xs = a.xi + soff[ks];
            // local coordinates of patch node (0, 0) in the solid's frame (periodic: wrapped once here)
            const int bx0 = sp.wall_x ? i0 - 1 - fr.ox : wrapi(i0 - 1 - fr.ox, sp.nx);
            const int by0 = sp.wall_y ? j0 - 1 - fr.oy : wrapi(j0 - 1 - fr.oy, sp.ny);
            BoxWalk wk(PX);
            for (int p = threadIdx.x; p < PN; p += blockDim.x, wk.next()) {
                int lx = bx0 + wk.c, ly = by0 + wk.r;
                if (!sp.wall_x) while (lx >= sp.nx) lx -= sp.nx;
                if (!sp.wall_y) while (ly >= sp.ny) ly -= sp.ny;
                R X = nanv<R>(), Y = nanv<R>(), P = nanv<R>();
                if (in_box(fr, lx, ly)) {
                    // the three loads at once (the phi plane's address is valid in
                    // the box); phi counts only where eta does
                    X = Xs[ly * T + lx];
                    Y = Xs[T * T + ly * T + lx];
                    P = Xs[2 * T * T + ly * T + lx];
                }
                if (!(X == X)) P = nanv<R>();
                sX[ks * PN + p] = X; sY[ks * PN + p] = Y; sP[ks * PN + p] = P;
            }
        }
        __syncthreads();
        // Half-edge stresses: blended solid stress (Eq. 3_6_global_stress) plus contact.
        for (int e = threadIdx.x; e < NXE + NYE; e += blockDim.x) {
            int pa[3], pb[3];  // patch indices of the 2x3 stencil (a low side, b high side)
            const bool xedge = e < NXE;
            if (xedge) {
                const int ex = e % (TX + 1), ey = e / (TX + 1);  // edge between col ex-1 and ex (tile coords)
                for (int k = 0; k < 3; k++) { pa[k] = (ey + k) * PX + ex; pb[k] = (ey + k) * PX + ex + 1; }
            } else {
                const int f = e - NXE;
                const int ex = f % TX, ey = f / TX;               // edge between row ey-1 and ey
                for (int k = 0; k < 3; k++) { pa[k] = ey * PX + ex + k; pb[k] = (ey + 1) * PX + ex + k; }
            }
            R Sxx = 0, Sxy = 0, Syy = 0, L = 0, Cxx = 0, Cxy = 0, Cyy = 0;
            bool okv[KMAX];
            R phh[KMAX];
            for (int ks = 0; ks < n; ks++) {
                const R *X = sX + ks * PN, *Y = sY + ks * PN, *P = sP + ks * PN;
                bool ok = true;
                for (int k = 0; k < 3; k++) ok = ok && (P[pa[k]] == P[pa[k]]) && (P[pb[k]] == P[pb[k]]);
                okv[ks] = ok;
                if (!ok) continue;
                const R ph = R(0.5) * (P[pa[1]] + P[pb[1]]);
                phh[ks] = ph;
                // beyond the blur zone the solid's stress has weight lambda = 0 in
                // Eq. 3_6_global_stress: it is not formed (nor its Jacobian checked)
                if (!(ph < eps)) continue;
                const R lam = R(1) - heaviside<R>(ph, eps);
                R dXn, dXt, dYn, dYt, txx, txy, tyy;
                edge_grad<R>(X[pa[0]], X[pa[1]], X[pa[2]], X[pb[0]], X[pb[1]], X[pb[2]], dXn, dXt);
                edge_grad<R>(Y[pa[0]], Y[pa[1]], Y[pa[2]], Y[pb[0]], Y[pb[1]], Y[pb[2]], dYn, dYt);
                const R G = sG[ks];
                // J = d xi / dx = I + d eta / dx (the stored eta excludes the node position)
                const bool good = xedge ? stress_from_grad<R>(dXn, dXt, dYn, dYt, G, txx, txy, tyy)
                                        : stress_from_grad<R>(dXt, dXn, dYt, dYn, G, txx, txy, tyy);
                if (!good) { atomicOr(a.err, ERR_SINGULAR); continue; }
                Sxx += lam * txx; Sxy += lam * txy; Syy += lam * tyy; L += lam;
            }
            for (int ks = 0; ks < n; ks++) {
                if (!okv[ks] || !(phh[ks] < eps)) continue;
                for (int kt = ks + 1; kt < n; kt++) {
                    if (!okv[kt] || !(phh[kt] < eps)) continue;
                    const R fs = R(0.5) * (R(1) - phh[ks] / eps), ft = R(0.5) * (R(1) - phh[kt] / eps);
                    const R fm = fs < ft ? fs : ft;
                    const R *Ps = sP + ks * PN, *Pt = sP + kt * PN;
                    R gn, gt;
                    edge_grad<R>(Ps[pa[0]] - Pt[pa[0]], Ps[pa[1]] - Pt[pa[1]], Ps[pa[2]] - Pt[pa[2]],
                                 Ps[pb[0]] - Pt[pb[0]], Ps[pb[1]] - Pt[pb[1]], Ps[pb[2]] - Pt[pb[2]], gn, gt);
                    const R gxx = xedge ? gn : gt, gyy = xedge ? gt : gn;
                    const R nrm = rsqrt_<R>(gxx * gxx + gyy * gyy);
                    if (nrm == R(0)) continue;
                    const R nx_ = gxx / nrm, ny_ = gyy / nrm;
                    const R kk = -eta * fm * (sG[ks] + sG[kt]);
                    Cxx += kk * (nx_ * nx_ - R(0.5)); Cxy += kk * (nx_ * ny_); Cyy += kk * (ny_ * ny_ - R(0.5));
                }
            }
            if (L > R(1)) { Sxx /= L; Sxy /= L; Syy /= L; }
            eT[3 * e + 0] = Sxx + Cxx; eT[3 * e + 1] = Sxy + Cxy; eT[3 * e + 2] = Syy + Cyy;
        }
        __syncthreads();
        // Node: divergence (Eq. 3_3_div_solid_stress), solid fraction, drho, solid acceleration.
        // Meanwhile the warp past the node threads reads the next tile's solids.
        if (next >= 0 && threadIdx.x >= TILE_N && threadIdx.x < TILE_N + 32)
            force_solids<R>(sp, a, next, *fs_next, threadIdx.x - TILE_N);
        {
            const int cx = threadIdx.x & (TX - 1), cy = threadIdx.x >> sp.lx;
            const int i = i0 + cx, j = j0 + cy;
            if (threadIdx.x < TILE_N && i < sp.nx && j < sp.ny) {
                const R *tl = eT + 3 * (cy * (TX + 1) + cx), *tr = eT + 3 * (cy * (TX + 1) + cx + 1);
                const R *tb = eT + 3 * (NXE + cy * TX + cx), *tt = eT + 3 * (NXE + (cy + 1) * TX + cx);
                const R fsx = (tr[0] - tl[0]) + (tt[1] - tb[1]);
                const R fsy = (tr[1] - tl[1]) + (tt[2] - tb[2]);
                const int p = (cy + 1) * PX + cx + 1;
                R L = 0, Ay = 0, Dh = 0, Dl = 0;
                if constexpr (sizeof(R) == 4) {
                    // Delta rho = sum lambda (rho_s - rho_f) is an O(1) number whose
                    // rounding would drive the pressure: lambda comes as a float pair
                    // from the level set's pair (the relabel's low part) in and near
                    // the blur zone, exactly 0 or 1 elsewhere; float-float sums
                    float Lh = 0.0f, Ll = 0.0f;
                    for (int ks = 0; ks < n; ks++) {
                        const R ph = sP[ks * PN + p];
                        if (!(ph == ph)) continue;
                        float lh = 0.0f, ll = 0.0f;
                        // phi's low part exists where |phi| < eps + PHI_D_SHELL (the relabel's
                        // test, on its FP32 phi); within half that shell it is read
                        if (ph <= -eps - R(0.5f * PHI_D_SHELL)) lh = 1.0f;
                        else if (ph < eps + R(0.5f * PHI_D_SHELL)) {
                            const Frame &fr = sfr[ks];
                            const int lx = sp.wall_x ? i - fr.ox : wrapi(i - fr.ox, sp.nx);
                            const int ly = sp.wall_y ? j - fr.oy : wrapi(j - fr.oy, sp.ny);
                            const int T = sT[ks];
                            lambda_ff(sp, a.lamtab, ph, a.xi[soff[ks] + 5 * T * T + ly * T + lx], lh, ll);
                        }
                        if (lh == 0.0f) continue;
                        L += lh;
                        Ay += lh * sA[ks];
                        ff_add(Lh, Ll, lh, ll);
                        ff_add_prod(Dh, Dl, lh, ll, fs.sDh[ks], fs.sDl[ks]);
                    }
                    if (Lh + Ll > 1.0f) ff_div(Dh, Dl, Lh, Ll);
                } else {
                    double Ld = 0.0, Dd = 0.0;
                    for (int ks = 0; ks < n; ks++) {
                        const R ph = sP[ks * PN + p];
                        if (!(ph == ph)) continue;
                        const R lam = R(1) - heaviside<R>(ph, eps);
                        L += lam;
                        Ay += lam * sA[ks];
                        Ld += lam;
                        Dd += lam * sD[ks];
                    }
                    if (Ld > 1.0) Dd /= Ld;
                    Dh = R(Dd);
                }
                if (L > R(1)) Ay /= L;
                R *po = a.pool + (long long)tile * POOL_STRIDE + threadIdx.x;
                po[POOL_FX] = fsx;
                if (sp.force_mode == 1) {
                    po[POOL_FY] = fsy;
                    po[POOL_AY] = Ay;
                } else {
                    po[POOL_FY] = fsy + Ay;
                }
                R *pd = a.pool + (long long)tile * POOL_STRIDE + POOL_DRHO + 2 * threadIdx.x;
                pd[0] = Dh;
                pd[1] = Dl;
            }
        }
        __syncthreads();
    }
}

template <class R>
__global__ void __launch_bounds__(K3_THREADS) __maxnreg__(sizeof(R) == 4 ? 48 : 224) force_kernel(SimParams sp, ForceArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ForceShared<R> fs[2];  // this tile's solids, and the next tile's (read during this one)
    const int nact = *a.reg_nactive;
    int it = blockIdx.x;
    if (it >= nact) return;  // uniform over the CTA
    int tile = a.reg_active[it];
    if (threadIdx.x < 32) force_solids<R>(sp, a, tile, fs[0], threadIdx.x);
    __syncthreads();
    for (int b = 0; it < nact; it += gridDim.x, b ^= 1) {
        const int next = it + (int)gridDim.x < nact ? a.reg_active[it + gridDim.x] : -1;
        force_tile<R, true>(sp, a, tile, fs[b], reinterpret_cast<R *>(smem), next, &fs[b ^ 1]);
        tile = next;
    }
}

// ===========================================================================
// K1: fused moments + SFC equilibrium + Guo forcing + BGK + walls + push stream.
// ===========================================================================
template <class R, class S>
struct LbArgs {
    const S *f_in;
    S *f_out;
    // plane q of f_in, and of f_out shifted by the push of direction q
    // (f_out + q P + c_q,y nx + c_q,x): one address operation per interior access
    const S *fin_q[9];
    S *fout_push[9];
    S *carry;                  // density plane: read (previous step), then written
    const R *fbody;            // per row x body force
    const R *bfield;           // force_kind 3: per-node body force (x plane, y plane)
    R *tape;                   // optional: rho, ux, uy, Fx, Fy of every node (5 planes)
    const int *reg_count;      // registry of this step
    R *pool;                   // its pool: solid terms read, half-force written
    int *clr_count;            // registry of the previous step: read, then cleared for the next step
    int *clr_nactive;
    const R *pool_prev;        // force pool of the previous step (its Delta rho is the rest base)
    unsigned *err;
};

// The arithmetic of one node of K1 once its inputs are loaded: moments, SFC
// equilibrium, Guo forcing and BGK collision.  f: the stored populations (f[0]
// becomes relative to this step's Delta rho); fh: the post-collision values in
// stored form.  dro, dro_lo: the rest base (Delta rho of the step that wrote
// f); cx0, cy0: rho^{n-1} F^{n-1} / 2; Fx, Fy: the body force in, the whole
// force out; po: this step's pool entry of the node (lt) if the registry holds
// its tile, else null.  Returns rho - rho_f; rho, ux, uy for the tape.
template <class R>
__device__ __forceinline__ R lb_collide(const SimParams &sp, R (&f)[9], R (&fh)[9], const R dro, const R dro_lo,
                                        const R cx0, const R cy0, R &Fx, R &Fy, const R *po, const int lt, R &rho,
                                        R &ux, R &uy, unsigned *err) {
    const R ds = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
    const R dr = dro + ds;  // rho - rho_f
    const R jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    const R jy = (f[2] - f[4]) + (f[5] - f[7]) + (f[6] - f[8]);
    rho = pick<R>(sp.rho_f, sp.rho_f_f) + dr;
    const R inv = rcp_rn<R>(rho);
    ux = (jx + cx0) * inv;
    uy = (jy + cy0) * inv;
    R drt = R(0), drt_lo = R(0);
    if (po) {
        pool_drho<R>(po, lt, drt, drt_lo);
        if (sp.force_mode == 1) {
            // conservative form: the stress divergence enters the Guo term without rho
            Fx += po[POOL_FX] * inv;
            Fy += po[POOL_FY] * inv + po[POOL_AY];
        } else {
            Fx += po[POOL_FX];
            Fy += po[POOL_FY];
        }
    }
    if (!(ux + uy == ux + uy)) atomicOr(err, ERR_NAN);  // a NaN rho makes both velocities NaN
    const R omega = pick<R>(sp.omega, sp.omega_f), kf = pick<R>(sp.kf, sp.kf_f);
    const R u2 = ux * ux + uy * uy;
    const R uF = ux * Fx + uy * Fy;
    R dde;
    const R dds = two_diff<R>(dro, drt, dde);
    const R dd = dds + (dde + (dro_lo - drt_lo));  // change of the rest base over the step (small)
    const R ddr = dd + ds;       // rho - rho_t, without rounding against Delta rho
    f[0] += dd;                  // rest population relative to this step's Delta rho
    // Collision f^ = f - omega (f - f^eq) + (1 - omega/2) F_i (Eq. 2_2_bgk_force) with
    // f^eq of Eq. 2_3_feq_sfc in the stored form (minus w rho_f, minus Delta rho for
    // q = 0) and the Guo term of Eq. 2_2_Fi times rho.  Opposite directions share the
    // even parts (in c) of f^eq and F_i and differ in the sign of the odd parts.
    const R om1 = R(1) - omega;
    const R r15u2 = R(1.5) * u2, r3uF = R(3) * uF;
    {
        const R w = R(4) / R(9), rw = rho * w;
        fh[0] = om1 * f[0] + omega * (w * ddr - rw * r15u2) - kf * rw * r3uF;
    }
#pragma unroll
    for (int pr = 0; pr < 4; pr++) {
        const int q = pr + 1 + (pr >= 2 ? 2 : 0);  // 1, 2, 5, 6; partners 3, 4, 7, 8
        const int qo = oppq(q);
        const R w = wq<R>(q), rw = rho * w;
        const R cu = R(cxq(q)) * ux + R(cyq(q)) * uy;
        const R cF = R(cxq(q)) * Fx + R(cyq(q)) * Fy;
        const R even = omega * (w * ddr + rw * (R(4.5) * cu * cu - r15u2)) + kf * rw * (R(9) * cu * cF - r3uF);
        const R odd = R(3) * rw * (omega * cu + kf * cF);
        fh[q] = om1 * f[q] + even + odd;
        fh[qo] = om1 * f[qo] + even - odd;
    }
    return dr;
}

// One node (i, j) of K1: moments, SFC equilibrium, Guo forcing, BGK collision,
// walls and push streaming.  tile / lt: the node's registry tile and its index
// there (the pool's layout); interior: every push target of the caller's block
// lies inside the domain.  STAGED: the node's populations and density plane
// were staged in shared memory (9 + 1 planes of TILE_N values, node lt at
// offset lt).  Returns rho - rho_f.
// The half-force term rho F / 2 that the next step's moments need is kept
// where its force came from: on a tile this step's registry holds, in the
// pool (planes POOL_CX / POOL_CY); elsewhere the force is the body force
// alone and only rho - rho_f is stored (the density plane, one value instead
// of two), the next step multiplying it out again (free_carry).
// REG false: the node's tile is registered in neither this step's nor the
// previous step's registry (a free region), so neither is read.
template <class R, class S, bool STAGED, bool REG = true>
__device__ __forceinline__ R lb_node(const SimParams &sp, const LbArgs<R, S> &a, const int i, const int j,
                                     const int tile, const int lt, const bool interior, const S *stage) {
    const int nx = sp.nx, ny = sp.ny, P = (int)sp.P;  // 9 P < 2^31 is checked at creation
    const int c = j * nx + i;
    const int prev_count = REG ? a.clr_count[tile] : 0;  // cleared by the caller after every node read it
    R f[9];
#pragma unroll
    for (int q = 0; q < 9; q++)  // shared-memory stage: plain loads (the read-only path is global only)
        f[q] = STAGED ? ldS<S, R>(stage + q * TILE_N + lt, sp, q) : ldG<S, R>(a.fin_q[q] + c, sp, q);
    const R drp = STAGED ? ldC<S, R>(stage + 9 * TILE_N + lt, sp) : ldC<S, R>(a.carry + c, sp);
    R Fx, Fy;  // the body force (this step's and the previous step's)
    body_force<R>(sp, a.fbody, a.bfield, j, c, Fx, Fy);
    R dro = R(0), dro_lo = R(0);  // rest base: Delta rho of the step that wrote f (hi + lo)
    R cx0, cy0;                   // rho^{n-1} F^{n-1} / 2
    if (prev_count > 0) {
        const R *pp = a.pool_prev + (long long)tile * POOL_STRIDE + lt;
        pool_drho<R>(pp, lt, dro, dro_lo);
        cx0 = pp[POOL_CX];
        cy0 = pp[POOL_CY];
    } else {
        free_carry<R>(sp, drp, Fx, Fy, cx0, cy0);
    }
    R *po = (REG && a.reg_count[tile] > 0) ? a.pool + (long long)tile * POOL_STRIDE + lt : nullptr;
    R fh[9], rho, ux, uy;
    const R dr = lb_collide<R>(sp, f, fh, dro, dro_lo, cx0, cy0, Fx, Fy, po, lt, rho, ux, uy, a.err);
    if (a.tape) {
        a.tape[c] = rho; a.tape[P + c] = ux; a.tape[2 * P + c] = uy;
        a.tape[3 * P + c] = Fx; a.tape[4 * P + c] = Fy;
    }
    if (REG && po) {
        po[POOL_CX] = R(0.5) * rho * Fx;
        po[POOL_CY] = R(0.5) * rho * Fy;
    } else {
        stC<S, R>(a.carry + c, dr, sp);
    }
    if constexpr (is16<S>()) {
        bool ov = store_overflow_c<S, R>(dr, sp);
#pragma unroll
        for (int q = 0; q < 9; q++) ov = ov || store_overflow<S, R>(fh[q], sp, q);
        if (ov) atomicOr(a.err, ERR_OVERFLOW16);
    }
    stS<S, R>(a.fout_push[0] + c, fh[0], sp, 0);
    if (interior) {
#pragma unroll
        for (int q = 1; q < 9; q++) stS<S, R>(a.fout_push[q] + c, fh[q], sp, q);
    } else {
#pragma unroll
        for (int q = 1; q < 9; q++) {
            int di = i + cxq(q), dj = j + cyq(q);
            const bool ox = di < 0 || di >= nx, oy = dj < 0 || dj >= ny;
            if ((ox && sp.wall_x) || (oy && sp.wall_y)) {
                // halfway bounce-back; the top wall moves with lid_u (Sec. 3.5)
                const R uw = (oy && sp.wall_y && dj >= ny) ? pick<R>(sp.lid_u, sp.lid_u_f) : R(0);
                const R val = fh[q] - R(6) * wq<R>(q) * rho * (R(cxq(q)) * uw);
                stS<S, R>(a.f_out + oppq(q) * P + c, val, sp, oppq(q));
            } else {
                if (ox) di = di < 0 ? di + nx : di - nx;
                if (oy) dj = dj < 0 ? dj + ny : dj - ny;
                stS<S, R>(a.f_out + q * P + dj * nx + di, fh[q], sp, q);
            }
        }
    }
    return dr;
}

// One registry tile (bx, by) of K1, one thread per node (the staged form: the
// tile's planes are in shared memory).
template <class R, class S, bool STAGED>
__device__ __forceinline__ void lb_tile(const SimParams &sp, const LbArgs<R, S> &a, const int bx, const int by,
                                        const S *stage) {
    const int lt = threadIdx.x;
    const int i = bx * sp.tx + (lt & (sp.tx - 1)), j = by * sp.ty + (lt >> sp.lx);
    const int tile = by * sp.ntx + bx;
    const bool interior = bx > 0 && (bx + 1) * sp.tx < sp.nx && by > 0 && (by + 1) * sp.ty < sp.ny;
    if (i < sp.nx && j < sp.ny) lb_node<R, S, STAGED>(sp, a, i, j, tile, lt, interior, stage);
    __syncthreads();
    if (lt == 0) {
        a.clr_count[tile] = 0;
        if (tile == 0) *a.clr_nactive = 0;
    }
}

// One region (rx, ry) of K1: rk registry tiles side by side (LB_REGION_W x ty
// nodes, or one tile when tile_x >= LB_REGION_W), walked in rk passes of TILE_N
// nodes, each pass a band of whole rows.
// REG false: a free region (no registry reads; its registry tiles are empty,
// so there is nothing to clear).
template <class R, class S, bool REG = true, bool CLR_ACTIVE = true>
__device__ __forceinline__ void lb_region(const SimParams &sp, const LbArgs<R, S> &a, const int rx, const int ry) {
    const int lt = threadIdx.x;
    const int lw = sp.lx + sp.lk, W = 1 << lw;
    const int x0 = rx << lw, y0 = ry * sp.ty;
    const bool interior = x0 > 0 && x0 + W < sp.nx && y0 > 0 && y0 + sp.ty < sp.ny;
    for (int p = 0; p < sp.rk; p++) {
        const int n = p * TILE_N + lt;
        const int xl = n & (W - 1), yl = n >> lw;
        const int i = x0 + xl, j = y0 + yl;
        if (i < sp.nx && j < sp.ny) {
            const int tile = ry * sp.ntx + (rx << sp.lk) + (xl >> sp.lx);
            lb_node<R, S, false, REG>(sp, a, i, j, tile, (yl << sp.lx) + (xl & (sp.tx - 1)), interior, nullptr);
        }
    }
    if (REG) {
        __syncthreads();  // every node of the region's tiles has read the previous registry
        if (lt < sp.rk) {
            const int bx = (rx << sp.lk) + lt;
            if (bx < sp.ntx) a.clr_count[ry * sp.ntx + bx] = 0;
        }
    }
    if (CLR_ACTIVE && lt == 0 && rx == 0 && ry == 0) *a.clr_nactive = 0;
}

// K1 over the regions of one kind.  MODE 0: every region; 1: the busy regions
// (busy[r] != 0); 2: the free regions, without registry reads.  The split lets
// the free regions run concurrently with K2 and K3 (overlapped step).
template <class R, class S, int MODE>
__global__ void __launch_bounds__(TILE_N, LB_MIN_BLOCKS<R, S>) lb_step_kernel(SimParams sp, LbArgs<R, S> a,
                                                                           const unsigned char *busy) {
    if (MODE != 0) {
        const bool b = busy[blockIdx.y * sp.nrx + blockIdx.x] != 0;
        if (b != (MODE == 1)) return;  // uniform over the CTA, before any barrier
    }
    lb_region<R, S, MODE != 2, MODE == 0>(sp, a, blockIdx.x, blockIdx.y);
}

// Classification of the K1 regions of the overlapped step n, after K2 of step
// n: a region is busy when one of its registry tiles is registered in registry
// n (the step's solid forcing and Delta rho) or in registry n - 1 (the rest base
// of the populations the step reads); a free region needs neither.  Every node
// that the reference-map kernel of step n + 1 reads (solid and blur-zone nodes
// of phi^{n+1} and their 4-neighbours) lies in registry n's tiles, so the next
// step's solid kernels need only the busy regions of this one.  Also clears the
// active-tile count of registry n - 1 (its counts are cleared by the busy K1).
static __global__ void lb_classify_kernel(SimParams sp, const int *reg_now, const int *reg_prev, unsigned char *busy,
                                          int *nactive_prev) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r == 0) *nactive_prev = 0;
    if (r >= sp.nrx * sp.nty) return;
    const int rx = r % sp.nrx, ry = r / sp.nrx;
    const int b0 = rx << sp.lk, b1 = min(b0 + sp.rk, sp.ntx);
    bool any = false;
    for (int bx = b0; bx < b1; bx++) {
        const int t = ry * sp.ntx + bx;
        any = any || reg_now[t] > 0 || reg_prev[t] > 0;
    }
    busy[r] = any ? 1 : 0;
}

// Classification of the K1 regions for the overlapped step n: a region is busy
// when one of its registry tiles or of their 8 neighbour tiles is registered in
// registry n - 1.  A registry covers the tiles that the box of the blur zone,
// grown by one node, touches; interfaces move less than one node per step, so
// registry n lies inside the busy regions and a free region needs neither
// registry.  The previous classification is checked on the fly: a tile of a
// region that step n - 1 treated as free must not be in registry n - 1.
__device__ __forceinline__ void classify_region(const SimParams &sp, int r, const int *reg_prev,
                                                const unsigned char *busy_prev, unsigned char *busy, unsigned *err) {
    const int rx = r % sp.nrx, ry = r / sp.nrx;
    const int b0 = rx << sp.lk, b1 = min(b0 + sp.rk, sp.ntx) - 1;  // the region's tile columns
    bool any = false, own = false;
    for (int dy = -1; dy <= 1; dy++) {
        int by = ry + dy;
        if (by < 0 || by >= sp.nty) {
            if (sp.wall_y) continue;
            by = by < 0 ? by + sp.nty : by - sp.nty;
        }
        for (int bx = b0 - 1; bx <= b1 + 1; bx++) {
            int tx = bx;
            if (tx < 0 || tx >= sp.ntx) {
                if (sp.wall_x) continue;
                tx = tx < 0 ? tx + sp.ntx : tx - sp.ntx;
            }
            if (reg_prev[by * sp.ntx + tx] > 0) {
                any = true;
                if (dy == 0 && bx >= b0 && bx <= b1) own = true;
            }
        }
    }
    if (own && !busy_prev[r]) atomicOr(err, ERR_FREE_REGION);
    busy[r] = any ? 1 : 0;
}

// ---------------------------------------------------------------------------
// K1 with TMA staging: persistent CTAs walk the tiles with a grid stride; one
// thread loads each tile's 9 population planes and its density plane with
// two 3-D bulk tensor copies (boxes tile_x x tile_y x 9 and x 1) into one of
// two shared-memory stages, completing on an mbarrier, so the copies of the
// next tile overlap the collision of the current one.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap *map, int x, int y, int z, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Wait for the phase with the given parity to complete; false after ~2^31 cycles.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
    const long long t0 = clock64();
    while (true) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1ll << 31)) return false;
    }
}

template <class R, class S>
__global__ void __launch_bounds__(TILE_N, LB_MIN_BLOCKS<R, S>) lb_tma_kernel(SimParams sp, LbArgs<R, S> a,
                                                        const __grid_constant__ CUtensorMap tm_f,
                                                        const __grid_constant__ CUtensorMap tm_c, int ntiles) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long bar[2];
    __shared__ int ok;
    // the stages start on a 128-byte boundary of the shared window (the launch
    // reserves 128 bytes for this): tensor copies write to 128-byte aligned addresses
    const unsigned pad = (128u - (smem_u32(smem) & 127u)) & 127u;
    S *stage0 = reinterpret_cast<S *>(smem + pad);
    const unsigned stage_elems = 10u * TILE_N, stage_bytes = stage_elems * (unsigned)sizeof(S);
    const int lt = threadIdx.x;
    if (lt == 0) {
        ok = ((smem_u32(stage0) & 127u) == 0u && ((stage_bytes & 127u) == 0u)) ? 1 : 0;
        if (!ok) atomicOr(a.err, ERR_ALIGN);
        mbar_init(smem_u32(&bar[0]), 1);
        mbar_init(smem_u32(&bar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (!ok) return;  // nothing issued yet
    auto issue = [&](int tile, int st) {
        const int bx = tile % sp.ntx, by = tile / sp.ntx;
        const unsigned b = smem_u32(&bar[st]);
        const unsigned dst = smem_u32(stage0 + st * stage_elems);
        mbar_expect_tx(b, stage_bytes);
        tma_load_3d(dst, &tm_f, bx * sp.tx, by * sp.ty, 0, b);
        tma_load_3d(dst + 9u * TILE_N * (unsigned)sizeof(S), &tm_c, bx * sp.tx, by * sp.ty, 0, b);
    };
    int tile = blockIdx.x;
    if (lt == 0) {
        if (tile < ntiles) issue(tile, 0);
        if (tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x, 1);
    }
    for (int it = 0; tile < ntiles; tile += gridDim.x, it++) {
        const int st = it & 1;
        if (lt == 0) ok = mbar_wait_bounded(smem_u32(&bar[st]), (it >> 1) & 1) ? 1 : 0;
        __syncthreads();
        if (!ok) {
            if (lt == 0) {
                atomicOr(a.err, ERR_TIMEOUT);
                // let the other stage's copy (if one was issued) land before leaving
                if (tile + (int)gridDim.x < ntiles) mbar_wait_bounded(smem_u32(&bar[st ^ 1]), ((it + 1) >> 1) & 1);
            }
            return;
        }
        lb_tile<R, S, true>(sp, a, tile % sp.ntx, tile / sp.ntx, stage0 + st * stage_elems);
        // every thread has read stage st (lb_tile ends with a barrier): refill it
        if (lt == 0 && tile + 2 * (int)gridDim.x < ntiles) issue(tile + 2 * gridDim.x, st);
    }
}

// Initial populations f = f^eq,SFC(rho_t, 0): in the stored form (relative to
// w_q rho_f and, for q = 0, to the initial Delta rho) every value is zero.
template <class R, class S>
__global__ void init_f_kernel(SimParams sp, S *f, S *carry) {
    const int i = blockIdx.x * sp.tx + (threadIdx.x & (sp.tx - 1)), j = blockIdx.y * sp.ty + (threadIdx.x >> sp.lx);
    if (i >= sp.nx || j >= sp.ny) return;
    const long long c = (long long)j * sp.nx + i;
    for (int q = 0; q < 9; q++) stS<S, R>(f + q * sp.P + c, R(0), sp, q);
    stC<S, R>(carry + c, R(NAN), sp);  // no previous collision (the pools start at zero)
}

// Self-check of the failure path of the tensor-copy pipeline: one thread
// waits, with the pipeline's bounded wait, on an mbarrier that nothing
// completes (no copy is issued, no thread arrives) and records the timeout as
// lb_tma_kernel does.  Nothing is in flight when it gives up.
static __global__ void bounded_wait_check_kernel(unsigned *err) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (!mbar_wait_bounded(smem_u32(&bar), 0)) atomicOr(err, ERR_TIMEOUT);
    }
}

// Total mass, one registry tile per CTA: each node's rho - rho_f (its nine
// stored values and its rest base, Delta rho of the step that wrote them, hi +
// lo) is formed in FP64 and the CTA's sum written to partials[tile]; the
// partials are then added in a fixed order (mass_reduce_kernel).
template <class R, class S>
__global__ void __launch_bounds__(TILE_N) mass_tile_kernel(SimParams sp, const S *f, const int *reg_count, const R *pool,
                                                           double *partials) {
    __shared__ double red[32];
    const int i = blockIdx.x * sp.tx + (threadIdx.x & (sp.tx - 1)), j = blockIdx.y * sp.ty + (threadIdx.x >> sp.lx);
    double v[1] = {0.0};
    if (i < sp.nx && j < sp.ny) {
        const long long c = (long long)j * sp.nx + i;
        double dr = rest_base_d<R>(sp, reg_count, pool, i, j);
        for (int q = 0; q < 9; q++) dr += (double)ldS<S, R>(f + q * sp.P + c, sp, q);
        v[0] = dr;
    }
    block_sum<double, 1>(v, red);
    if (threadIdx.x == 0) partials[blockIdx.y * sp.ntx + blockIdx.x] = v[0];
}

// Fields to a double grid.  kind: 0 rho, 1 ux, 2 uy, 3 Fx, 4 Fy, 5 drho, 20+q f_q.
template <class R, class S>
__global__ void field_kernel(SimParams sp, const S *f, const S *carry, const R *fbody, const R *bfield, const int *reg_count,
                             const R *pool, int kind, double *out) {
    const int i = blockIdx.x * sp.tx + (threadIdx.x & (sp.tx - 1)), j = blockIdx.y * sp.ty + (threadIdx.x >> sp.lx);
    if (i >= sp.nx || j >= sp.ny) return;
    const int tile = blockIdx.y * sp.ntx + blockIdx.x;
    const long long c = (long long)j * sp.nx + i;
    double v = 0;
    if (kind == 0) {
        // rho = rho_f + rest base + stored values, summed in FP64 so the readout adds no rounding
        double dr = rest_base_d<R>(sp, reg_count, pool, i, j);
        for (int q = 0; q < 9; q++) dr += (double)ldS<S, R>(f + q * sp.P + c, sp, q);
        v = sp.rho_f + dr;
    } else if (kind <= 2) {
        R rho, u, w;
        node_moments<R, S>(sp, f, carry, fbody, bfield, reg_count, pool, i, j, rho, u, w);
        v = kind == 1 ? (double)u : (double)w;
    } else if (kind <= 5) {
        const R *po = pool + (long long)tile * POOL_STRIDE + threadIdx.x;
        const bool reg = reg_count[tile] > 0;
        const R bx = sp.force_kind == 3 ? bfield[c] : fbody[j];
        const R by = sp.force_kind == 3 ? bfield[sp.P + c] : pick<R>(sp.fy, sp.fy_f);
        if (kind == 3) v = (double)(bx + (reg ? po[POOL_FX] : R(0)));
        else if (kind == 4) v = (double)(by + (reg ? po[POOL_FY] + (sp.force_mode == 1 ? po[POOL_AY] : R(0)) : R(0)));
        else v = rest_base_d<R>(sp, reg_count, pool, i, j);
    } else {
        const int q = kind - 20;
        v = (double)ldS<S, R>(f + q * sp.P + c, sp, q) + wq<double>(q) * sp.rho_f;  // the exact weight, as the upload
        if (q == 0) v += rest_base_d<R>(sp, reg_count, pool, i, j);
    }
    out[c] = v;
}

// Deformation measures of solid node (lx, ly) from central differences of xi
// over its 4-neighbours, J = d xi / dx = I + A: det F - 1 with F = J^-1 (the
// volumetric deviation of Sec. 4.1), and the von Mises stress of the
// neo-Hookean stress of Eq. 3_3_solid_stress in plane strain (the out-of-plane
// deviatoric component is -(tau_xx + tau_yy)).  False where a neighbour is
// missing or J is singular.
// det F - 1 (F = J^-1) from the 4-neighbour values of eta = xi - position
// (d xi / dx = I + d eta / dx by central differences); false where a neighbour
// is invalid or J is singular.  A = d eta / dx is returned for the stress.
template <class R>
__device__ __forceinline__ bool det_dev_from_stencil(R Xe, R Xw, R Xn, R Xs, R Ye, R Yw, R Yn, R Ys, R &Axx, R &Axy,
                                                     R &Ayx, R &Ayy, R &ddet) {
    if (!(Xe == Xe && Xw == Xw && Xn == Xn && Xs == Xs)) return false;
    Axx = R(0.5) * (Xe - Xw); Axy = R(0.5) * (Xn - Xs); Ayx = R(0.5) * (Ye - Yw); Ayy = R(0.5) * (Yn - Ys);
    const R dl = (Axx + Ayy) + (Axx * Ayy - Axy * Ayx);  // det J - 1
    if (R(1) + dl == R(0)) return false;
    ddet = -dl / (R(1) + dl);
    return true;
}

template <class R>
__device__ __forceinline__ bool node_deformation(const R *X, const R *Y, int T, int lx, int ly, const Frame &fr, R G,
                                                 R &ddet, R &vm) {
    if (!(lx > fr.bx0 && lx < fr.bx1 && ly > fr.by0 && ly < fr.by1)) return false;
    const int k = ly * T + lx;
    const R Xe = X[k + 1], Xw = X[k - 1], Xn = X[k + T], Xs = X[k - T];
    const R Ye = Y[k + 1], Yw = Y[k - 1], Yn = Y[k + T], Ys = Y[k - T];
    R Axx, Axy, Ayx, Ayy;
    if (!det_dev_from_stencil<R>(Xe, Xw, Xn, Xs, Ye, Yw, Yn, Ys, Axx, Axy, Ayx, Ayy, ddet)) return false;
    R txx, txy, tyy;
    stress_from_grad<R>(Axx, Axy, Ayx, Ayy, G, txx, txy, tyy);
    const R tzz = -(txx + tyy);
    vm = rsqrt_<R>(R(1.5) * (txx * txx + tyy * tyy + tzz * tzz + R(2) * txy * txy));
    return true;
}

// One solid's field onto the grid: kind 0, 1 the reference map, 2 the level
// set (on the solid and its band), 4 det F - 1 and 5 the von Mises stress (on
// the solid nodes, phi < 0); NaN elsewhere.
template <class R>
__global__ void solid_field_kernel(SimParams sp, const R *xi, const Frame *frames, const SolidDesc *solids, int s,
                                   int kind, double *out) {
    const SolidDesc sd = solids[s];
    const Frame fr = frames[s];
    const int2 o = make_int2(fr.ox, fr.oy);
    const Rsq<R> rq(sd);
    const int T = sd.T;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T * T; t += gridDim.x * blockDim.x) {
        const int lx = t % T, ly = t / T;
        const int gx = o.x + lx, gy = o.y + ly;
        if (!in_box(fr, lx, ly) || !domain_cell(sp, gx, gy)) continue;
        const R X = xi[sd.off + t], Y = xi[sd.off + T * T + t];
        if (!(X == X)) continue;
        const long long c = grid_index(sp, gx, gy);
        double v;
        // xi = eta + l + off + X_c
        // the low parts of eta are kept on the solid's nodes (phi < 0; the band's are
        // refitted every step and carry none)
        const bool low = xi_planes<R>() == 6 && xi[sd.off + 2 * T * T + t] < R(0);
        if (kind == 0) {
            v = (double)X + ((double)lx + (double)fr.offx + sd.xc);
            if (low) v += (double)xi[sd.off + 3 * T * T + t];
        } else if (kind == 1) {
            v = (double)Y + ((double)ly + (double)fr.offy + sd.yc);
            if (low) v += (double)xi[sd.off + 4 * T * T + t];
        } else if (kind == 2) v = (double)xi[sd.off + 2 * T * T + t];
        else {
            if (!(xi[sd.off + 2 * T * T + t] < -R(PHI_TIE))) continue;
            R ddet, vm;
            if (!node_deformation<R>(xi + sd.off, xi + sd.off + T * T, T, lx, ly, fr, pick<R>(sd.G, sd.G_f), ddet, vm))
                continue;
            v = kind == 4 ? (double)ddet : (double)vm;
        }
        out[c] = v;
    }
}

// Per-solid FP64 statistics of the current state (one CTA per solid).
// Per-solid statistics of the current state (FP64 sums; Sec. 4 outputs):
// mass-like sum L = sum lambda, centroid, sum lambda rho, momentum, and over the
// solid's nodes max |det F - 1| and its lambda-weighted mean.  One CTA per solid.
// Each warp walks its share of the band box (outside it xi is invalid) and
// queues, in shared memory, the nodes of the solid and blur zone (phi < eps);
// every 32 queued nodes it takes one per lane with all its loads issued first.
constexpr int STATS_THREADS = 256;
constexpr int STATS_COLS = 10;  // per solid: area, centroid (2), mass, momentum (2), det F (2), contact force (2)
template <class R, class S>
struct StatsNode {
    int lx, ly, reg;
    bool inner;  // strictly inside the band box: the deformation stencil is on the tile
    R phi, f[9], pool, cx, cy, st[8];
};
// Every load of one queued node, issued before any is used: the populations,
// the half-force term's sources (the pool's half-force and the density plane
// and body force, one of them used) and the rest base (the pool entries are
// read alongside the registry count and used only if the tile is registered;
// their addresses are valid either way), phi, and the 4-neighbour stencil of
// eta for det F.
template <class R, class S>
__device__ __forceinline__ void stats_gather(const SimParams &sp, const S *f, const S *carry, const R *fbody,
                                             const R *bfield, const int *reg, const R *pool, const R *xi, int T,
                                             int2 ow, const Frame &fr, int e, StatsNode<R, S> &nd) {
    nd.lx = e & 0xffff;
    nd.ly = e >> 16;
    const int t = nd.ly * T + nd.lx;
    nd.phi = xi[2 * T * T + t];
    // ow: the tile origin wrapped into the grid, so one subtraction wraps a node
    int i = ow.x + nd.lx, j = ow.y + nd.ly;
    while (i >= sp.nx) i -= sp.nx;
    while (j >= sp.ny) j -= sp.ny;
    const long long c = (long long)j * sp.nx + i;
#pragma unroll
    for (int q = 0; q < 9; q++) nd.f[q] = ldS<S, R>(f + q * sp.P + c, sp, q);
    const int tile = (j >> sp.ly) * sp.ntx + (i >> sp.lx);
    const int lt = ((j & (sp.ty - 1)) << sp.lx) + (i & (sp.tx - 1));
    const R *po = pool + (long long)tile * POOL_STRIDE + lt;
    nd.reg = reg[tile];
    nd.pool = po[POOL_DRHO + lt];
    const R pcx = po[POOL_CX], pcy = po[POOL_CY], drp = ldC<S, R>(carry + c, sp);
    R Fx, Fy;
    body_force<R>(sp, fbody, bfield, j, c, Fx, Fy);
    nd.inner = nd.lx > fr.bx0 && nd.lx < fr.bx1 && nd.ly > fr.by0 && nd.ly < fr.by1;
    if (nd.inner) {
        const R *Y = xi + T * T;
        nd.st[0] = xi[t + 1]; nd.st[1] = xi[t - 1]; nd.st[2] = xi[t + T]; nd.st[3] = xi[t - T];
        nd.st[4] = Y[t + 1]; nd.st[5] = Y[t - 1]; nd.st[6] = Y[t + T]; nd.st[7] = Y[t - T];
    }
    // the half-force term: from the pool on a registered tile, else rebuilt
    if (nd.reg > 0) {
        nd.cx = pcx;
        nd.cy = pcy;
    } else {
        free_carry<R>(sp, drp, Fx, Fy, nd.cx, nd.cy);
    }
}
// One node's terms, added to the thread's partial sums in the arithmetic
// precision (FP64 is a narrow pipe on this GPU; the FP32 path's inputs are FP32
// anyway); positions relative to the tile origin.  Each warp then sums its
// threads' terms in that precision and the warps' sums are added in FP64.
// Compensated accumulation (Neumaier): acc + cmp carries the sum of the added
// terms to ~2 u |sum| whatever their count (cmp stays zero in FP64).
template <class R>
__device__ __forceinline__ void comp_add(R &acc, R &cmp, R v) {
    if constexpr (sizeof(R) == 4) {
        const R t = acc + v;
        cmp += fabsf(acc) >= fabsf(v) ? (acc - t) + v : (v - t) + acc;
        acc = t;
    } else {
        acc += v;
    }
}

template <class R, class S>
__device__ __forceinline__ void stats_finish(const SimParams &sp, const StatsNode<R, S> &nd, R eps, R (&acc)[8],
                                             R (&cmp)[8], R &mx) {
    R rho, u, v;
    moments_from<R>(sp, nd.f, nd.reg > 0 ? nd.pool : R(0), nd.cx, nd.cy, rho, u, v);
    const R lam = R(1) - heaviside<R>(nd.phi, eps), lr = lam * rho;
    comp_add(acc[0], cmp[0], lam); comp_add(acc[1], cmp[1], lam * R(nd.lx)); comp_add(acc[2], cmp[2], lam * R(nd.ly));
    comp_add(acc[3], cmp[3], lr); comp_add(acc[4], cmp[4], lr * u); comp_add(acc[5], cmp[5], lr * v);
    R Axx, Axy, Ayx, Ayy, ddet;
    if (nd.phi < -R(PHI_TIE) && nd.inner &&
        det_dev_from_stencil<R>(nd.st[0], nd.st[1], nd.st[2], nd.st[3], nd.st[4], nd.st[5], nd.st[6], nd.st[7], Axx,
                                Axy, Ayx, Ayy, ddet)) {
        const R a = ddet < R(0) ? -ddet : ddet;
        comp_add(acc[6], cmp[6], lam * a);
        comp_add(acc[7], cmp[7], lam);
        mx = a > mx ? a : mx;
    }
}

// Level set of solid `sol` at grid node (i, j) from its tile (frame fr), or
// NaN where the node is outside the tile's box or not a valid band node.
template <class R>
__device__ __forceinline__ R tile_phi(const SimParams &sp, const R *xi, const SolidDesc &sd, const Frame &fr, int i, int j) {
    int lx = i - fr.ox, ly = j - fr.oy;
    if (!sp.wall_x) {  // periodic: the node and the frame origin are within a period or two
        while (lx < 0) lx += sp.nx;
        while (lx >= sp.nx) lx -= sp.nx;
    }
    if (!sp.wall_y) {
        while (ly < 0) ly += sp.ny;
        while (ly >= sp.ny) ly -= sp.ny;
    }
    if (!in_box(fr, lx, ly)) return nanv<R>();
    const R *X = xi + sd.off;
    const int T = sd.T, t = ly * T + lx;
    const R x = X[t], p = X[2 * T * T + t];  // both loads at once (phi's address is valid in the box)
    return x == x ? p : nanv<R>();
}

// Contact stress of a pair (Eqs. 3_6_collision_stress .. 3_6_normal) on the
// half-edge of direction dir (0: between (i-1, j) and (i, j); 1: between
// (i, j-1) and (i, j)), from the level sets ps, pt of the two solids on the
// 3 x 4 (or 4 x 3) nodes around it, as the force kernel forms it; false where
// a stencil node is missing or the pair is not in contact there.
template <class R>
__device__ __forceinline__ bool pair_edge_tau(const R (&ps)[4][4], const R (&pt)[4][4], int dir, int ex, int ey, R eps,
                                              R eta, R Gsum, R (&tau)[3]) {
    R as[3], bs[3], at[3], bt[3];
    for (int k = 0; k < 3; k++) {
        // node indices in the 4x4 block: a on the low side of the edge, b on the high side
        const int ax = dir == 0 ? ex - 1 : ex - 1 + k, ay = dir == 0 ? ey - 1 + k : ey - 1;
        const int bx = dir == 0 ? ex : ex - 1 + k, by = dir == 0 ? ey - 1 + k : ey;
        as[k] = ps[ay][ax]; bs[k] = ps[by][bx]; at[k] = pt[ay][ax]; bt[k] = pt[by][bx];
        if (!(as[k] == as[k] && bs[k] == bs[k] && at[k] == at[k] && bt[k] == bt[k])) return false;
    }
    const R phs = R(0.5) * (as[1] + bs[1]), pht = R(0.5) * (at[1] + bt[1]);
    if (!(phs < eps) || !(pht < eps)) return false;
    const R fs = R(0.5) * (R(1) - phs / eps), ft = R(0.5) * (R(1) - pht / eps);
    const R fm = fs < ft ? fs : ft;
    R gn, gt;
    edge_grad<R>(as[0] - at[0], as[1] - at[1], as[2] - at[2], bs[0] - bt[0], bs[1] - bt[1], bs[2] - bt[2], gn, gt);
    const R gxx = dir == 0 ? gn : gt, gyy = dir == 0 ? gt : gn;
    const R nrm = rsqrt_<R>(gxx * gxx + gyy * gyy);
    if (nrm == R(0)) return false;
    const R nx_ = gxx / nrm, ny_ = gyy / nrm;
    const R kk = -eta * fm * Gsum;
    tau[0] = kk * (nx_ * nx_ - R(0.5)); tau[1] = kk * (nx_ * ny_); tau[2] = kk * (ny_ * ny_ - R(0.5));
    return true;
}

// The pair contact divergences of one tile that solid s shares with another
// (the nodes nearer to s), added to fc; used by contact_force_sum below.
template <class R>
__device__ __forceinline__ void contact_tile_sum(const SimParams &sp, const R *xi, const Frame *frames,
                                                 const SolidDesc *solids, const int *reg, const int *reg_solids, int s,
                                                 const SolidDesc &sd, const Frame &fr, R eps, R eta, int tile,
                                                 double (&fc)[2]) {
                    const int bx = tile % sp.ntx, by = tile / sp.ntx;
                    const int n = min(reg[tile], sp.kmax);
                    for (int lt = threadIdx.x; lt < TILE_N; lt += blockDim.x) {  // the tile's nodes
                    const int i = bx * sp.tx + (lt & (sp.tx - 1)), j = by * sp.ty + (lt >> sp.lx);
                    if (i >= sp.nx || j >= sp.ny) continue;
                    // 4x4 block of level sets: nodes (i-1..i+2, j-1..j+2), block index (x - i + 1, y - j + 1).
                    // The node's four half-edges need the cross (1,1), (0,1), (2,1), (1,0), (1,2)
                    // for their contact test (both solids' edge-averaged phi below eps): it is
                    // read first, the rest of the blocks only where an edge passes the test.
                    R ps[4][4];
                    ps[1][1] = tile_phi<R>(sp, xi, sd, fr, i, j);
                    if (!(ps[1][1] == ps[1][1])) continue;
                    ps[1][0] = tile_phi<R>(sp, xi, sd, fr, i - 1, j);
                    ps[1][2] = tile_phi<R>(sp, xi, sd, fr, i + 1, j);
                    ps[0][1] = tile_phi<R>(sp, xi, sd, fr, i, j - 1);
                    ps[2][1] = tile_phi<R>(sp, xi, sd, fr, i, j + 1);
                    bool have_s = false;  // the rest of ps read
                    for (int k = 0; k < n; k++) {
                        const int t = reg_solids[tile * KMAX + k];
                        if (t == s) continue;
                        const SolidDesc td = solids[t];
                        const Frame tf = frames[t];
                        R pt[4][4];
                        pt[1][1] = tile_phi<R>(sp, xi, td, tf, i, j);
                        pt[1][0] = tile_phi<R>(sp, xi, td, tf, i - 1, j);
                        pt[1][2] = tile_phi<R>(sp, xi, td, tf, i + 1, j);
                        pt[0][1] = tile_phi<R>(sp, xi, td, tf, i, j - 1);
                        pt[2][1] = tile_phi<R>(sp, xi, td, tf, i, j + 1);
                        {
                            // an edge whose two nodes are not both valid, or whose averaged phi of
                            // either solid is not below eps, carries no contact stress
                            const R e2 = R(2) * eps;
                            const bool cl = ps[1][0] + ps[1][1] < e2 && pt[1][0] + pt[1][1] < e2;
                            const bool cr = ps[1][2] + ps[1][1] < e2 && pt[1][2] + pt[1][1] < e2;
                            const bool cb = ps[0][1] + ps[1][1] < e2 && pt[0][1] + pt[1][1] < e2;
                            const bool ct = ps[2][1] + ps[1][1] < e2 && pt[2][1] + pt[1][1] < e2;
                            if (!(cl || cr || cb || ct)) continue;
                        }
                        if (!have_s) {
                            for (int yy = 0; yy < 4; yy++)
                                for (int xx = 0; xx < 4; xx++)
                                    if (!((xx == 1 || yy == 1) && xx < 3 && yy < 3))
                                        ps[yy][xx] = tile_phi<R>(sp, xi, sd, fr, i - 1 + xx, j - 1 + yy);
                            have_s = true;
                        }
                        for (int yy = 0; yy < 4; yy++)
                            for (int xx = 0; xx < 4; xx++)
                                if (!((xx == 1 || yy == 1) && xx < 3 && yy < 3))
                                    pt[yy][xx] = tile_phi<R>(sp, xi, td, tf, i - 1 + xx, j - 1 + yy);
                        const R p0 = pt[1][1];
                        const double w = !(p0 == p0) || ps[1][1] < p0 ? 1.0 : (ps[1][1] == p0 ? 0.5 : 0.0);
                        if (w == 0.0) continue;
                        const R Gsum = pick<R>(sd.G + td.G, sd.G_f + td.G_f);
                        R tl[3] = {0, 0, 0}, tr[3] = {0, 0, 0}, tb[3] = {0, 0, 0}, tt[3] = {0, 0, 0};
                        bool any = pair_edge_tau<R>(ps, pt, 0, 1, 1, eps, eta, Gsum, tl);
                        any = pair_edge_tau<R>(ps, pt, 0, 2, 1, eps, eta, Gsum, tr) || any;
                        any = pair_edge_tau<R>(ps, pt, 1, 1, 1, eps, eta, Gsum, tb) || any;
                        any = pair_edge_tau<R>(ps, pt, 1, 1, 2, eps, eta, Gsum, tt) || any;
                        if (!any) continue;
                        fc[0] += w * (double)((tr[0] - tl[0]) + (tt[1] - tb[1]));
                        fc[1] += w * (double)((tr[1] - tl[1]) + (tt[2] - tb[2]));
                    }
                    }
}

// Net contact force on solid s: over the registry tiles around it that also
// hold another solid t, the divergence (Eq. 3_3_div_solid_stress) of the pair's
// contact stress at every domain node nearer to s than to t (phi_s < phi_t,
// half where equal; a node outside t's band is nearer to s), summed over the
// pairs in FP64 by the CTA's threads.
constexpr int CONTACT_CAP = 128;  // tiles a solid shares with another, listed in shared memory

template <class R>
__device__ __noinline__ void contact_force_sum(const SimParams &sp, const int *reg, const int *reg_solids, const R *xi,
                                  const Frame *frames, const SolidDesc *solids, int s, const Frame &fr, double (&fc)[2],
                                  int *ctile /* shared, CONTACT_CAP */, int *nct /* shared */) {
    const SolidDesc sd = solids[s];
    const R eps = pick<R>(sp.eps, sp.eps_f), eta = pick<R>(sp.eta, sp.eta_f);
    if (fr.bx0 > fr.bx1) return;  // uniform over the CTA
    int rx0[2], rx1[2], ry0[2], ry1[2];
    const int nrx = tile_ranges(fr.ox + fr.bx0, fr.ox + fr.bx1, sp.nx, sp.wall_x, sp.lx, sp.ntx, rx0, rx1);
    const int nry = tile_ranges(fr.oy + fr.by0, fr.oy + fr.by1, sp.ny, sp.wall_y, sp.ly, sp.nty, ry0, ry1);
    // The box's tiles that the solid shares with another, found by the CTA's
    // threads at once and listed in increasing tile index: the order of the
    // ranges walked row by row, which the per-thread FP64 sums follow.
    const int lx0 = nrx > 0 ? rx1[0] - rx0[0] + 1 : 0, lx1 = nrx > 1 ? rx1[1] - rx0[1] + 1 : 0;
    const int ly0 = nry > 0 ? ry1[0] - ry0[0] + 1 : 0, ly1 = nry > 1 ? ry1[1] - ry0[1] + 1 : 0;
    const int TXn = lx0 + lx1, ntot = TXn * (ly0 + ly1);
    if (threadIdx.x == 0) *nct = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < ntot; k += blockDim.x) {
        const int kx = k % TXn, ky = k / TXn;
        const int bx = kx < lx0 ? rx0[0] + kx : rx0[1] + (kx - lx0);
        const int by = ky < ly0 ? ry0[0] + ky : ry0[1] + (ky - ly0);
        const int tile = by * sp.ntx + bx;
        const int n = min(reg[tile], sp.kmax);
        if (n < 2) continue;
        bool mine = false;
        for (int m = 0; m < n; m++) mine = mine || reg_solids[tile * KMAX + m] == s;
        if (mine) {
            const int pos = atomicAdd(nct, 1);
            if (pos < CONTACT_CAP) ctile[pos] = tile;
        }
    }
    __syncthreads();
    const int ncand = *nct;
    if (ncand > CONTACT_CAP) {  // more than the list holds: every tile of the box in turn, in the same order
        for (int ay = 0; ay < nry; ay++)
            for (int by = ry0[ay]; by <= ry1[ay]; by++)
                for (int ax = 0; ax < nrx; ax++)
                    for (int bx = rx0[ax]; bx <= rx1[ax]; bx++) {
                        const int tile = by * sp.ntx + bx;
                        const int n = min(reg[tile], sp.kmax);
                        if (n < 2) continue;
                        bool mine = false;
                        for (int m = 0; m < n; m++) mine = mine || reg_solids[tile * KMAX + m] == s;
                        if (mine) contact_tile_sum<R>(sp, xi, frames, solids, reg, reg_solids, s, sd, fr, eps, eta,
                                                      tile, fc);
                    }
        return;
    }
    if (threadIdx.x == 0)  // insertion sort of the (short) list
        for (int a = 1; a < ncand; a++) {
            const int v = ctile[a];
            int b = a - 1;
            while (b >= 0 && ctile[b] > v) { ctile[b + 1] = ctile[b]; b--; }
            ctile[b + 1] = v;
        }
    __syncthreads();
    for (int c = 0; c < ncand; c++) contact_tile_sum<R>(sp, xi, frames, solids, reg, reg_solids, s, sd, fr, eps, eta,
                                                        ctile[c], fc);
}

template <class R, class S>
__global__ void __launch_bounds__(STATS_THREADS, sizeof(R) == 4 ? 3 : 2) solid_stats_kernel(SimParams sp, const S *f, const S *carry,
                                                                    const R *fbody, const R *bfield, const int *reg, const int *reg_solids, const R *pool,
                                                                    const R *xi, const Frame *frames,
                                                                    const SolidDesc *solids, const int *order,
                                                                    double *out) {
    __shared__ double red[32 * STATS_COLS];
    __shared__ unsigned long long dmax;
    __shared__ int queue[STATS_THREADS / 32][64];  // per warp: < 32 waiting + one round of 32
    __shared__ int ctile[CONTACT_CAP], nct;         // tiles shared with another solid (contact sum)
    const int s = order ? order[blockIdx.x] : (int)blockIdx.x;  // largest tiles first, as K2
    const SolidDesc sd = solids[s];
    const Frame fr = frames[s];
    const int2 o = make_int2(fr.ox, fr.oy), ow = make_int2(wrapi(fr.ox, sp.nx), wrapi(fr.oy, sp.ny));
    const int T = sd.T;
    const R *X = xi + sd.off;
    const R eps = pick<R>(sp.eps, sp.eps_f);
    R acc[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    R cmp[8] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    R mx = R(0);
    if (threadIdx.x == 0) dmax = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int *qu = queue[warp];
    int qn = 0;  // warp-uniform
    auto drain = [&](int cnt) {  // the last cnt (<= 32) queued nodes, one per lane
        StatsNode<R, S> nd;
        if (lane < cnt) {
            stats_gather<R, S>(sp, f, carry, fbody, bfield, reg, pool, X, T, ow, fr, qu[qn - cnt + lane], nd);
            stats_finish<R, S>(sp, nd, eps, acc, cmp, mx);
        }
        __syncwarp();
        qn -= cnt;
    };
    const int w = fr.bx1 - fr.bx0 + 1, h = fr.by1 - fr.by0 + 1;
    const int n = w > 0 && h > 0 ? w * h : 0;
    // four rounds of the walk per pass: their loads are issued together.  Each
    // lane steps its box position (c, r) by the warps' stride, without divisions.
    constexpr int WU = 4;
    const int step = nw * 32;
    int c = 0, r = 0, dc = 0, dr = 0;
    if (w > 0) { c = (warp * 32 + lane) % w; r = (warp * 32 + lane) / w; dc = step % w; dr = step / w; }
    for (int base = warp * 32; base < n; base += WU * step) {
        int ee[WU];
        bool keep[WU];
        R xv[WU], pv[WU];
#pragma unroll
        for (int u = 0; u < WU; u++) {
            const int lx = fr.bx0 + c, ly = fr.by0 + r;
            keep[u] = base + u * step + lane < n && domain_cell(sp, o.x + lx, o.y + ly);
            ee[u] = (ly << 16) | lx;
            xv[u] = pv[u] = R(0);
            if (keep[u]) {
                const int t = ly * T + lx;
                xv[u] = X[t];
                pv[u] = X[2 * T * T + t];
            }
            c += dc; r += dr;
            if (c >= w) { c -= w; r++; }
        }
#pragma unroll
        for (int u = 0; u < WU; u++) {
            const bool kp = keep[u] && xv[u] == xv[u] && pv[u] < eps;
            const unsigned m = __ballot_sync(0xffffffffu, kp);
            if (kp) qu[qn + __popc(m & ((1u << lane) - 1u))] = ee[u];
            qn += __popc(m);
            __syncwarp();
            if (qn >= 32) drain(32);
        }
    }
    if (qn > 0) drain(qn);
    // each thread's compensated sums in FP64, then warp and CTA sums in FP64
    double v[STATS_COLS];
#pragma unroll
    for (int k = 0; k < 8; k++) v[k] = (double)acc[k] + (double)cmp[k];
    for (int d = 16; d > 0; d >>= 1) {
        const R m2 = __shfl_down_sync(0xffffffffu, mx, d);
        mx = m2 > mx ? m2 : mx;
    }
    if (lane == 0) atomicMax(&dmax, (unsigned long long)__double_as_longlong((double)mx));  // non-negative: bits order as values
    // the net contact force (FP64, accumulated at the contact nodes only)
    v[8] = v[9] = 0.0;
    {
        double fc[2] = {0.0, 0.0};
        contact_force_sum<R>(sp, reg, reg_solids, xi, frames, solids, s, fr, fc, ctile, &nct);
        v[8] = fc[0];
        v[9] = fc[1];
    }
#pragma unroll
    for (int k = 0; k < STATS_COLS; k++)
        for (int d = 16; d > 0; d >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], d);
    if (lane == 0)
        for (int k = 0; k < STATS_COLS; k++) red[warp * STATS_COLS + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double st[STATS_COLS];
        for (int k = 0; k < STATS_COLS; k++) {
            st[k] = 0.0;
            for (int ww = 0; ww < nw; ww++) st[k] += red[ww * STATS_COLS + k];
        }
        double *q = out + STATS_COLS * s;
        q[0] = st[0]; q[1] = o.x + st[1] / st[0]; q[2] = o.y + st[2] / st[0]; q[3] = st[3]; q[4] = st[4]; q[5] = st[5];
        q[6] = __longlong_as_double((long long)dmax);
        q[7] = st[7] > 0.0 ? st[6] / st[7] : 0.0;
        q[8] = st[8]; q[9] = st[9];
    }
}

// Fixed-order FP64 sum of the per-block mass partials (single CTA).
__global__ void mass_reduce_kernel(const double *partials, int n, double base, double *out);

}  // namespace lbrmt
