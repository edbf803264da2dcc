// lbrmt_adjoint.cuh -- reverse (adjoint) kernels of one LBRMT step and the
// centroid loss, for FP32 or FP64 arithmetic with full-precision storage.
//
// The forward step n -> n+1 (Algorithm 1) maps
//   K2: xi^{n+1} = advect(xi^n, u^n) on S^n = {phi(xi^n) < 0} (Eqs. 3_1_refmap_adv,
//       3_1_eno), then the layered weighted least-squares extrapolation of the band
//       (Sec. 3.2) whose weights for layers 1-2 use the normal of phi(xi^n);
//   K3: F^(n) = div tau(xi^{n+1}) + blended solid acceleration + body force
//       (Eqs. 3_3_refmap_jacobian, 3_3_solid_stress, 3_6_global_stress,
//       3_6_collision_stress, 3_3_div_solid_stress), Delta rho^(n) (Eq. 2_3_drho);
//   K1: f^{n+1}(x + c_q) = BGK collision of f^n with f^eq,SFC(rho^n, u^n, Delta rho)
//       and the Guo term (Eqs. 2_2_bgk_force, 2_3_feq_sfc, 3_4_Fi), with halfway
//       bounce-back (Sec. 3.5); u^n = (sum c f^n + rho^{n-1} F^(n-1) / 2) / rho^n.
// The kernels below apply the transposed Jacobians in the reverse order
// (K1, K3, K2), with the branch decisions of the forward step (solid set,
// layers, windows, upwind directions, contact pairs) recomputed from the
// recorded state; the adjoint of the populations is that of the absolute f_q.
#pragma once

#include "lbrmt_kernels.cuh"

namespace lbrmt {

template <class R> __device__ __forceinline__ R rcos(R x);
template <> __device__ __forceinline__ float rcos<float>(float x) { return cosf(x); }
template <> __device__ __forceinline__ double rcos<double>(double x) { return cos(x); }

// dH/dphi of the smoothed Heaviside.
template <class R> __device__ __forceinline__ R dheaviside(R phi, R eps) {
    if (phi <= -eps || phi >= eps) return R(0);
    const R pi = R(3.14159265358979323846);
    return R(0.5) * (R(1) + rcos<R>(pi * phi / eps)) / eps;
}

// d phi / d eta at a tile node: phi = |p + eta| - R with p = l + off.
template <class R>
__device__ __forceinline__ void dphi_deta(R ex, R ey, int lx, int ly, const Frame &fr, R &gx, R &gy) {
    const R X = (R(lx) + R(fr.offx)) + ex, Y = (R(ly) + R(fr.offy)) + ey;
    const R r = rsqrt_<R>(X * X + Y * Y);
    if (r > R(0)) { gx = X / r; gy = Y / r; }
    else { gx = R(0); gy = R(0); }
}

// ---------------------------------------------------------------------------
// K1 reverse: one node per thread.
// ---------------------------------------------------------------------------
template <class R>
struct LbAdjArgs {
    const R *tape;     // rho^n, ux^n, uy^n, Fx^(n), Fy^(n) (5 planes)
    const R *fb_next;  // adjoint of f^{n+1} (9 planes)
    const R *cb_next;  // adjoint of the stored half-force rho^n F^(n) / 2 (2 planes)
    R *fb, *cb;        // adjoint of f^n, of the half-force read at step n
    R *Fb, *Db;        // adjoint of F^(n) (2 planes) and Delta rho^(n)
    double *bodyb;     // adjoint of the body force field, accumulated (2 planes) or null
};

template <class R>
__global__ void __launch_bounds__(256) lb_adjoint_kernel(SimParams sp, LbAdjArgs<R> a) {
    const long long P = sp.P;
    const int nx = sp.nx, ny = sp.ny;
    const R omega = pick<R>(sp.omega, sp.omega_f), kf = pick<R>(sp.kf, sp.kf_f);
    const R lid = pick<R>(sp.lid_u, sp.lid_u_f);
    for (long long c = blockIdx.x * 256ll + threadIdx.x; c < P; c += (long long)gridDim.x * 256) {
        const int i = (int)(c % nx), j = (int)(c / nx);
        const R rho = a.tape[c], ux = a.tape[P + c], uy = a.tape[2 * P + c];
        const R Fx = a.tape[3 * P + c], Fy = a.tape[4 * P + c];
        // adjoint of the post-collision populations: pull of the push, bounce-back at walls
        R am[9];
        R rhob = R(0);
        am[0] = a.fb_next[c];
#pragma unroll
        for (int q = 1; q < 9; q++) {
            int di = i + cxq(q), dj = j + cyq(q);
            const bool ox = di < 0 || di >= nx, oy = dj < 0 || dj >= ny;
            if ((ox && sp.wall_x) || (oy && sp.wall_y)) {
                const R g = a.fb_next[oppq(q) * P + c];
                am[q] = g;
                const R uw = (oy && sp.wall_y && dj >= ny) ? lid : R(0);
                rhob -= R(6) * wq<R>(q) * R(cxq(q)) * uw * g;
            } else {
                if (ox) di = di < 0 ? di + nx : di - nx;
                if (oy) dj = dj < 0 ? dj + ny : dj - ny;
                am[q] = a.fb_next[q * P + (long long)dj * nx + di];
            }
        }
        const R cbx = a.cb_next[c], cby = a.cb_next[P + c];
        const R u2 = ux * ux + uy * uy, uF = ux * Fx + uy * Fy;
        R ubx = R(0), uby = R(0), sw = R(0);
        R Fbx = R(0.5) * rho * cbx, Fby = R(0.5) * rho * cby;
        rhob += R(0.5) * (Fx * cbx + Fy * cby);
#pragma unroll
        for (int q = 0; q < 9; q++) {
            const R w = wq<R>(q), cx = R(cxq(q)), cy = R(cyq(q));
            const R cu = cx * ux + cy * uy, cF = cx * Fx + cy * Fy;
            const R A = R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * u2;  // f^eq_q = w rho A + Delta rho (delta_q0 - w)
            const R B = R(3) * (cF - uF) + R(9) * cu * cF;                  // Guo term = rho w B
            const R aq = am[q];
            rhob += aq * w * (omega * A + kf * B);
            const R rw = aq * rho * w;
            ubx += rw * (omega * (R(3) * cx + R(9) * cu * cx - R(3) * ux) + kf * (R(9) * cF * cx - R(3) * Fx));
            uby += rw * (omega * (R(3) * cy + R(9) * cu * cy - R(3) * uy) + kf * (R(9) * cF * cy - R(3) * Fy));
            Fbx += rw * kf * (R(3) * (cx - ux) + R(9) * cu * cx);
            Fby += rw * kf * (R(3) * (cy - uy) + R(9) * cu * cy);
            sw += w * aq;
        }
        const R Dbv = omega * (am[0] - sw);
        // u = (sum c f + half-force) / rho
        const R inv = R(1) / rho;
        const R jbx = ubx * inv, jby = uby * inv;
        rhob -= (ubx * ux + uby * uy) * inv;
        a.cb[c] = jbx;
        a.cb[P + c] = jby;
#pragma unroll
        for (int q = 0; q < 9; q++) a.fb[q * P + c] = (R(1) - omega) * am[q] + rhob + R(cxq(q)) * jbx + R(cyq(q)) * jby;
        a.Fb[c] = Fbx;
        a.Fb[P + c] = Fby;
        a.Db[c] = Dbv;
        if (a.bodyb) {
            a.bodyb[c] += (double)Fbx;
            a.bodyb[P + c] += (double)Fby;
        }
    }
}

// ---------------------------------------------------------------------------
// K3 reverse: one registered tile per CTA iteration.
// ---------------------------------------------------------------------------
template <class R>
struct ForceAdjArgs {
    const R *xi;            // xi^{n+1} tiles
    const Frame *frame;     // their frames
    const int *reg_count, *reg_solids, *reg_active, *reg_nactive;  // registry of step n
    const SolidDesc *solids;
    const R *Fb;            // adjoint of F^(n) (2 planes); null: zero (node terms only)
    const R *Db;            // adjoint of Delta rho^(n) (1 plane)
    R *xib;                 // adjoint of xi^{n+1}, accumulated (same tiles and frames)
    double *Gb, *Rb;        // per-solid adjoints of G and of rho_s / rho_f, accumulated
};

__host__ __device__ __forceinline__ int force_adj_smem_elems(int tx, int ty) {
    return 6 * KMAX * force_patch_n(tx, ty) + 3 * ((tx + 1) * ty + tx * (ty + 1)) + 3 * TILE_N;
}
__host__ __device__ __forceinline__ int force_adj_smem_max() {
    int m = 0;
    for (int tx = 16; tx <= 128; tx *= 2) m = force_adj_smem_elems(tx, TILE_N / tx) > m ? force_adj_smem_elems(tx, TILE_N / tx) : m;
    return m;
}

// Reverse of stress_from_grad: given the adjoint of (txx, txy, tyy), add the
// adjoint of (Axx, Axy, Ayx, Ayy).
template <class R>
__device__ __forceinline__ void stress_adjoint(R Axx, R Axy, R Ayx, R Ayy, R G, R tbxx, R tbxy, R tbyy, R &Abxx,
                                               R &Abxy, R &Abyx, R &Abyy) {
    const R dl = (Axx + Ayy) + (Axx * Ayy - Axy * Ayx);
    const R inv = R(1) / (R(1) + dl);
    const R Dxx = (Ayy - dl) * inv, Dxy = -Axy * inv, Dyx = -Ayx * inv, Dyy = (Axx - dl) * inv;
    const R Ebxx = G * (R(2) * tbxx - tbyy) / R(3), Ebyy = G * (R(2) * tbyy - tbxx) / R(3), Ebxy = G * tbxy;
    const R Dbxx = Ebxx * (R(2) + R(2) * Dxx) + Ebxy * Dyx;
    const R Dbxy = Ebxx * R(2) * Dxy + Ebxy * (R(1) + Dyy);
    const R Dbyx = Ebxy * (R(1) + Dxx) + Ebyy * R(2) * Dyx;
    const R Dbyy = Ebxy * Dxy + Ebyy * (R(2) + R(2) * Dyy);
    R dlb = -(Dbxx + Dbyy) * inv;
    const R invb = Dbxx * (Ayy - dl) - Dbxy * Axy - Dbyx * Ayx + Dbyy * (Axx - dl);
    dlb += -invb * inv * inv;
    Abyy += Dbxx * inv + dlb * (R(1) + Axx);
    Abxx += Dbyy * inv + dlb * (R(1) + Ayy);
    Abxy += -Dbxy * inv - dlb * Ayx;
    Abyx += -Dbyx * inv - dlb * Axy;
}

template <class R>
__device__ void force_adjoint_tile(const SimParams &sp, const ForceAdjArgs<R> &a, const int tile, ForceShared<R> &fs,
                                   double *sGb, double *sRb, R *dyn, bool node_only) {
    const int TX = sp.tx, PX = TX + 2, PN = force_patch_n(TX, sp.ty);
    const int NXE = (TX + 1) * sp.ty, NYE = TX * (sp.ty + 1);
    R *sX = dyn, *sY = sX + KMAX * PN, *sP = sY + KMAX * PN;
    R *bX = sP + KMAX * PN, *bY = bX + KMAX * PN, *bP = bY + KMAX * PN;
    R *eTb = bP + KMAX * PN;          // [(NXE + NYE) * 3]
    R *nF = eTb + 3 * (NXE + NYE);    // [3 * TILE_N]: F_x, F_y, Delta rho adjoints of the tile nodes
    const R eps = pick<R>(sp.eps, sp.eps_f), eta = pick<R>(sp.eta, sp.eta_f);
    const R rho_f = pick<R>(sp.rho_f, sp.rho_f_f);
    const int tx = tile % sp.ntx, ty = tile / sp.ntx;
    const int i0 = tx * TX, j0 = ty * sp.ty;
    if (threadIdx.x == 0) {
        int n = min(a.reg_count[tile], sp.kmax);
        for (int k = 0; k < n; k++) fs.ids[k] = a.reg_solids[tile * KMAX + k];
        for (int k = 1; k < n; k++) {
            int v = fs.ids[k], m = k - 1;
            while (m >= 0 && fs.ids[m] > v) { fs.ids[m + 1] = fs.ids[m]; m--; }
            fs.ids[m + 1] = v;
        }
        fs.nk = n;
    }
    __syncthreads();
    const int n = fs.nk;
    if (threadIdx.x < n) {
        const SolidDesc &sd = a.solids[fs.ids[threadIdx.x]];
        fs.sfr[threadIdx.x] = a.frame[fs.ids[threadIdx.x]];
        fs.sG[threadIdx.x] = pick<R>(sd.G, sd.G_f);
        fs.sD[threadIdx.x] = pick<R>(sd.drho, sd.drho_f);
        fs.sA[threadIdx.x] = pick<R>(sd.accel, sd.accel_f);
        fs.srq[threadIdx.x] = Rsq<R>(sd);
        fs.sT[threadIdx.x] = sd.T;
        fs.soff[threadIdx.x] = sd.off;
        sGb[threadIdx.x] = 0.0;
        sRb[threadIdx.x] = 0.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * PN; idx += blockDim.x) {
        const int ks = idx / PN, p = idx % PN;
        const int px = p % PX, py = p / PX;
        const int gx = i0 - 1 + px, gy = j0 - 1 + py;
        const Frame fr = fs.sfr[ks];
        const int T = fs.sT[ks];
        const int lx = sp.wall_x ? gx - fr.ox : wrapi(gx - fr.ox, sp.nx);
        const int ly = sp.wall_y ? gy - fr.oy : wrapi(gy - fr.oy, sp.ny);
        R X = nanv<R>(), Y = nanv<R>(), Pv = nanv<R>();
        if (in_box(fr, lx, ly)) {
            const R *Xs = a.xi + fs.soff[ks];
            X = Xs[ly * T + lx];
            Y = Xs[T * T + ly * T + lx];
            if (X == X) Pv = phi_eta(X, Y, lx, ly, fr, fs.srq[ks]);
        }
        sX[ks * PN + p] = X; sY[ks * PN + p] = Y; sP[ks * PN + p] = Pv;
        bX[ks * PN + p] = R(0); bY[ks * PN + p] = R(0); bP[ks * PN + p] = R(0);
    }
    {
        const int lt = threadIdx.x;
        const int i = i0 + (lt & (TX - 1)), j = j0 + (lt >> sp.lx);
        const bool in = i < sp.nx && j < sp.ny;
        const long long c = (long long)j * sp.nx + i;
        nF[lt] = (in && a.Fb) ? a.Fb[c] : R(0);
        nF[TILE_N + lt] = (in && a.Fb) ? a.Fb[sp.P + c] : R(0);
        nF[2 * TILE_N + lt] = in ? a.Db[c] : R(0);
    }
    __syncthreads();
    // Node terms: Delta rho = sum lam drho_s / max(1, L), A_y = sum lam a_s / max(1, L).
    {
        const int lt = threadIdx.x, cx = lt & (TX - 1), cy = lt >> sp.lx;
        const int p = (cy + 1) * PX + cx + 1;
        const R Dbar = nF[2 * TILE_N + lt], Aybar = nF[TILE_N + lt];
        if (Dbar != R(0) || Aybar != R(0)) {
            R L = 0, D = 0, Ay = 0;
            for (int ks = 0; ks < n; ks++) {
                const R ph = sP[ks * PN + p];
                if (!(ph == ph)) continue;
                const R lam = R(1) - heaviside<R>(ph, eps);
                L += lam; D += lam * fs.sD[ks]; Ay += lam * fs.sA[ks];
            }
            R Dr = Dbar, Ar = Aybar, Lb = R(0);
            if (L > R(1)) {
                Dr = Dbar / L; Ar = Aybar / L;
                Lb = -(Dbar * (D / L) + Aybar * (Ay / L)) / L;
            }
            for (int ks = 0; ks < n; ks++) {
                const R ph = sP[ks * PN + p];
                if (!(ph == ph)) continue;
                const R lam = R(1) - heaviside<R>(ph, eps);
                const R lamb = Dr * fs.sD[ks] + Ar * fs.sA[ks] + Lb;
                atomicAdd(&bP[ks * PN + p], -dheaviside<R>(ph, eps) * lamb);
                // drho_s = rho_f (r - 1), a_s = -(1 - 1/r) g with r = rho_s / rho_f
                const SolidDesc &sd = a.solids[fs.ids[ks]];
                const double r = sd.rho_s / sp.rho_f;
                atomicAdd(&sRb[ks], (double)lam * ((double)Dr * (double)rho_f - (double)Ar * sp.gravity / (r * r)));
            }
        }
    }
    if (node_only) {
        __syncthreads();
        if (threadIdx.x < n) atomicAdd(&a.Rb[fs.ids[threadIdx.x]], sRb[threadIdx.x]);
        __syncthreads();
        return;
    }
    // Edge stress adjoints from the tile's nodes: F_x = d_x tau_xx + d_y tau_xy, F_y = d_x tau_xy + d_y tau_yy.
    for (int e = threadIdx.x; e < NXE + NYE; e += blockDim.x) {
        R bxx = 0, bxy = 0, byy = 0;
        if (e < NXE) {
            const int ex = e % (TX + 1), ey = e / (TX + 1);
            if (ex >= 1) { const int l = ey * TX + ex - 1; bxx += nF[l]; bxy += nF[TILE_N + l]; }
            if (ex < TX) { const int r = ey * TX + ex; bxx -= nF[r]; bxy -= nF[TILE_N + r]; }
        } else {
            const int f = e - NXE, ex = f % TX, ey = f / TX;
            if (ey >= 1) { const int b = (ey - 1) * TX + ex; bxy += nF[b]; byy += nF[TILE_N + b]; }
            if (ey < sp.ty) { const int t = ey * TX + ex; bxy -= nF[t]; byy -= nF[TILE_N + t]; }
        }
        eTb[3 * e] = bxx; eTb[3 * e + 1] = bxy; eTb[3 * e + 2] = byy;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NXE + NYE; e += blockDim.x) {
        const R tbxx = eTb[3 * e], tbxy = eTb[3 * e + 1], tbyy = eTb[3 * e + 2];
        if (tbxx == R(0) && tbxy == R(0) && tbyy == R(0)) continue;
        int pa[3], pb[3];
        const bool xedge = e < NXE;
        if (xedge) {
            const int ex = e % (TX + 1), ey = e / (TX + 1);
            for (int k = 0; k < 3; k++) { pa[k] = (ey + k) * PX + ex; pb[k] = (ey + k) * PX + ex + 1; }
        } else {
            const int f = e - NXE, ex = f % TX, ey = f / TX;
            for (int k = 0; k < 3; k++) { pa[k] = ey * PX + ex + k; pb[k] = (ey + 1) * PX + ex + k; }
        }
        // pass 1: the blended solid stress and sum lambda
        R Sxx = 0, Sxy = 0, Syy = 0, L = 0;
        unsigned okm = 0;
        for (int ks = 0; ks < n; ks++) {
            const R *X = sX + ks * PN, *Y = sY + ks * PN, *Pp = sP + ks * PN;
            bool ok = true;
            for (int k = 0; k < 3; k++) ok = ok && (Pp[pa[k]] == Pp[pa[k]]) && (Pp[pb[k]] == Pp[pb[k]]);
            if (!ok) continue;
            const R ph = R(0.5) * (Pp[pa[1]] + Pp[pb[1]]);
            if (!(ph < eps)) continue;  // lambda = 0 and dlambda/dphi = 0: as the forward, no terms
            const R lam = R(1) - heaviside<R>(ph, eps);
            R dXn, dXt, dYn, dYt, txx, txy, tyy;
            edge_grad<R>(X[pa[0]], X[pa[1]], X[pa[2]], X[pb[0]], X[pb[1]], X[pb[2]], dXn, dXt);
            edge_grad<R>(Y[pa[0]], Y[pa[1]], Y[pa[2]], Y[pb[0]], Y[pb[1]], Y[pb[2]], dYn, dYt);
            const bool good = xedge ? stress_from_grad<R>(dXn, dXt, dYn, dYt, fs.sG[ks], txx, txy, tyy)
                                    : stress_from_grad<R>(dXt, dXn, dYt, dYn, fs.sG[ks], txx, txy, tyy);
            if (!good) continue;
            okm |= 1u << ks;
            Sxx += lam * txx; Sxy += lam * txy; Syy += lam * tyy; L += lam;
        }
        R Sbxx = tbxx, Sbxy = tbxy, Sbyy = tbyy, Lb = R(0);
        if (L > R(1)) {
            Sbxx /= L; Sbxy /= L; Sbyy /= L;
            Lb = -(tbxx * Sxx + tbxy * Sxy + tbyy * Syy) / (L * L);
        }
        // pass 2: each solid's stress and weight
        for (int ks = 0; ks < n; ks++) {
            if (!((okm >> ks) & 1u)) continue;
            const R *X = sX + ks * PN, *Y = sY + ks * PN, *Pp = sP + ks * PN;
            const R ph = R(0.5) * (Pp[pa[1]] + Pp[pb[1]]);
            const R lam = R(1) - heaviside<R>(ph, eps);
            R dXn, dXt, dYn, dYt, h_xx, h_xy, h_yy;
            edge_grad<R>(X[pa[0]], X[pa[1]], X[pa[2]], X[pb[0]], X[pb[1]], X[pb[2]], dXn, dXt);
            edge_grad<R>(Y[pa[0]], Y[pa[1]], Y[pa[2]], Y[pb[0]], Y[pb[1]], Y[pb[2]], dYn, dYt);
            const R Axx = xedge ? dXn : dXt, Axy = xedge ? dXt : dXn, Ayx = xedge ? dYn : dYt, Ayy = xedge ? dYt : dYn;
            stress_from_grad<R>(Axx, Axy, Ayx, Ayy, R(1), h_xx, h_xy, h_yy);  // stress per unit G
            const R G = fs.sG[ks];
            const R lamb = G * (Sbxx * h_xx + Sbxy * h_xy + Sbyy * h_yy) + Lb;
            atomicAdd(&sGb[ks], (double)(lam * (Sbxx * h_xx + Sbxy * h_xy + Sbyy * h_yy)));
            R Abxx = 0, Abxy = 0, Abyx = 0, Abyy = 0;
            stress_adjoint<R>(Axx, Axy, Ayx, Ayy, G, lam * Sbxx, lam * Sbxy, lam * Sbyy, Abxx, Abxy, Abyx, Abyy);
            // back to the 2x3 stencils: dn = b1 - a1, dt = (b2 + a2 - b0 - a0) / 4
            const R bXn = xedge ? Abxx : Abxy, bXt = xedge ? Abxy : Abxx;
            const R bYn = xedge ? Abyx : Abyy, bYt = xedge ? Abyy : Abyx;
            R *gX = bX + ks * PN, *gY = bY + ks * PN, *gP = bP + ks * PN;
            atomicAdd(&gX[pb[1]], bXn); atomicAdd(&gX[pa[1]], -bXn);
            atomicAdd(&gX[pb[2]], bXt / R(4)); atomicAdd(&gX[pa[2]], bXt / R(4));
            atomicAdd(&gX[pb[0]], -bXt / R(4)); atomicAdd(&gX[pa[0]], -bXt / R(4));
            atomicAdd(&gY[pb[1]], bYn); atomicAdd(&gY[pa[1]], -bYn);
            atomicAdd(&gY[pb[2]], bYt / R(4)); atomicAdd(&gY[pa[2]], bYt / R(4));
            atomicAdd(&gY[pb[0]], -bYt / R(4)); atomicAdd(&gY[pa[0]], -bYt / R(4));
            const R phb = -dheaviside<R>(ph, eps) * lamb;
            atomicAdd(&gP[pa[1]], R(0.5) * phb);
            atomicAdd(&gP[pb[1]], R(0.5) * phb);
        }
        // pass 3: contact pairs (Eq. 3_6_collision_stress), not normalised
        for (int ks = 0; ks < n; ks++) {
            if (!((okm >> ks) & 1u)) continue;
            const R *Ps = sP + ks * PN;
            const R phs = R(0.5) * (Ps[pa[1]] + Ps[pb[1]]);
            if (!(phs < eps)) continue;
            for (int kt = ks + 1; kt < n; kt++) {
                if (!((okm >> kt) & 1u)) continue;
                const R *Pt = sP + kt * PN;
                const R pht = R(0.5) * (Pt[pa[1]] + Pt[pb[1]]);
                if (!(pht < eps)) continue;
                const R fsv = R(0.5) * (R(1) - phs / eps), ftv = R(0.5) * (R(1) - pht / eps);
                const bool take_s = fsv < ftv;
                const R fm = take_s ? fsv : ftv;
                R gn, gt;
                edge_grad<R>(Ps[pa[0]] - Pt[pa[0]], Ps[pa[1]] - Pt[pa[1]], Ps[pa[2]] - Pt[pa[2]],
                             Ps[pb[0]] - Pt[pb[0]], Ps[pb[1]] - Pt[pb[1]], Ps[pb[2]] - Pt[pb[2]], gn, gt);
                const R gxx = xedge ? gn : gt, gyy = xedge ? gt : gn;
                const R nrm = rsqrt_<R>(gxx * gxx + gyy * gyy);
                if (nrm == R(0)) continue;
                const R nx_ = gxx / nrm, ny_ = gyy / nrm;
                const R Gst = fs.sG[ks] + fs.sG[kt];
                const R kk = -eta * fm * Gst;
                const R kkb = tbxx * (nx_ * nx_ - R(0.5)) + tbxy * (nx_ * ny_) + tbyy * (ny_ * ny_ - R(0.5));
                const R nbx = kk * (R(2) * tbxx * nx_ + tbxy * ny_), nby = kk * (tbxy * nx_ + R(2) * tbyy * ny_);
                const R gG = -eta * fm * kkb;
                atomicAdd(&sGb[ks], (double)gG);
                atomicAdd(&sGb[kt], (double)gG);
                const R fmb = -eta * Gst * kkb;
                const int kw = take_s ? ks : kt;
                const R phw = -fmb / (R(2) * eps);  // f = (1 - phi / eps) / 2
                atomicAdd(&bP[kw * PN + pa[1]], R(0.5) * phw);
                atomicAdd(&bP[kw * PN + pb[1]], R(0.5) * phw);
                const R nd = nx_ * nbx + ny_ * nby;
                const R gbx = (nbx - nx_ * nd) / nrm, gby = (nby - ny_ * nd) / nrm;
                const R gbn = xedge ? gbx : gby, gbt = xedge ? gby : gbx;
                // (gn, gt) = edge_grad(P_s - P_t)
                const int ksk[2] = {ks, kt};
                for (int w = 0; w < 2; w++) {
                    const R sgn = w == 0 ? R(1) : R(-1);
                    R *gP = bP + ksk[w] * PN;
                    atomicAdd(&gP[pb[1]], sgn * gbn); atomicAdd(&gP[pa[1]], -sgn * gbn);
                    atomicAdd(&gP[pb[2]], sgn * gbt / R(4)); atomicAdd(&gP[pa[2]], sgn * gbt / R(4));
                    atomicAdd(&gP[pb[0]], -sgn * gbt / R(4)); atomicAdd(&gP[pa[0]], -sgn * gbt / R(4));
                }
            }
        }
    }
    __syncthreads();
    // phi = phi_0(xi): push the level-set adjoint onto xi and flush to the solids' adjoint tiles
    for (int idx = threadIdx.x; idx < n * PN; idx += blockDim.x) {
        const int ks = idx / PN, p = idx % PN;
        R gx_ = bX[ks * PN + p], gy_ = bY[ks * PN + p];
        const R pb_ = bP[ks * PN + p];
        const R X = sX[ks * PN + p], Y = sY[ks * PN + p];
        if (!(X == X)) continue;
        const int px = p % PX, py = p / PX;
        const Frame fr = fs.sfr[ks];
        const int gxg = i0 - 1 + px, gyg = j0 - 1 + py;
        const int lx = sp.wall_x ? gxg - fr.ox : wrapi(gxg - fr.ox, sp.nx);
        const int ly = sp.wall_y ? gyg - fr.oy : wrapi(gyg - fr.oy, sp.ny);
        if (pb_ != R(0)) {
            R dx_, dy_;
            dphi_deta<R>(X, Y, lx, ly, fr, dx_, dy_);
            gx_ += pb_ * dx_;
            gy_ += pb_ * dy_;
        }
        if (gx_ == R(0) && gy_ == R(0)) continue;
        const int T = fs.sT[ks];
        R *Xb = a.xib + fs.soff[ks];
        atomicAdd(&Xb[ly * T + lx], gx_);
        atomicAdd(&Xb[T * T + ly * T + lx], gy_);
    }
    __syncthreads();
    if (threadIdx.x < n) {
        atomicAdd(&a.Gb[fs.ids[threadIdx.x]], sGb[threadIdx.x]);
        atomicAdd(&a.Rb[fs.ids[threadIdx.x]], sRb[threadIdx.x]);
    }
    __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(TILE_N) force_adjoint_kernel(SimParams sp, ForceAdjArgs<R> a, int node_only) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ForceShared<R> fs;
    __shared__ double sGb[KMAX], sRb[KMAX];
    const int nact = *a.reg_nactive;
    for (int it = blockIdx.x; it < nact; it += gridDim.x)
        force_adjoint_tile<R>(sp, a, a.reg_active[it], fs, sGb, sRb, reinterpret_cast<R *>(smem), node_only != 0);
}

// ---------------------------------------------------------------------------
// K2 reverse: one solid per CTA.
// ---------------------------------------------------------------------------
template <class R>
struct RmtAdjArgs {
    const R *xi_in, *xi_out;            // xi^n and xi^{n+1} tiles
    const Frame *frame_in, *frame_out;  // their frames
    const R *tape;                      // rho^n, ux^n, uy^n (first 3 of 5 planes)
    R *xib_out;                         // adjoint of xi^{n+1}: complete on entry, passed down the layers
    R *xib_in;                          // adjoint of xi^n, accumulated
    R *fb, *cb;                         // adjoint of f^n and of the half-force of step n, accumulated
    const SolidDesc *solids;
};

// Normal of phi^n at input-frame node (ix, iy) from central differences, as the forward.
template <class R>
__device__ __forceinline__ bool adj_normal(const R *Xi, const R *Yi, int T, int ix, int iy, const Frame &fi,
                                           const Rsq<R> &rq, R &nhx, R &nhy, R &gxp, R &gyp, R &nn) {
    if (!(ix > fi.bx0 && iy > fi.by0 && ix < fi.bx1 && iy < fi.by1)) return false;
    const int k0 = iy * T + ix;
    const R Xe = Xi[k0 + 1], Xw = Xi[k0 - 1], Xn = Xi[k0 + T], Xs = Xi[k0 - T];
    if (!(Xe == Xe && Xw == Xw && Xn == Xn && Xs == Xs)) return false;
    const R pe = phi_eta(Xe, Yi[k0 + 1], ix + 1, iy, fi, rq), pw = phi_eta(Xw, Yi[k0 - 1], ix - 1, iy, fi, rq);
    const R pn = phi_eta(Xn, Yi[k0 + T], ix, iy + 1, fi, rq), ps = phi_eta(Xs, Yi[k0 - T], ix, iy - 1, fi, rq);
    gxp = (pe - pw) / R(2);
    gyp = (pn - ps) / R(2);
    nn = rsqrt_<R>(gxp * gxp + gyp * gyp);
    if (!(nn > R(0))) return false;
    nhx = gxp / nn;
    nhy = gyp / nn;
    return true;
}

// Weight of valid node (dx, dy) relative to the target (0 if the node is not used).
template <class R>
__device__ __forceinline__ R adj_weight(const signed char *lab, int k, int l, int dx, int dy, bool use_n, R nhx,
                                        R nhy, R &dn) {
    const int L = lab[k];
    dn = R(0);
    if (!(L >= 0 && L < l)) return R(0);
    R wt = pow2neg<R>(abs(dx) + abs(dy));
    if (use_n) {
        dn = (R(-dx) * nhx + R(-dy) * nhy) * rinv_tab<R>(dx, dy);
        wt = dn > R(COS_TIE) ? dn * wt : R(0);
    }
    return wt;
}

// Reverse of one extrapolated target (tx, ty) of layer l: pass its adjoint
// (xb, yb) to the nodes of its fit and, for the directional weights, return
// the adjoint of the unit normal.
template <class R>
__device__ void extrapolate_adjoint(const SimParams &sp, const signed char *lab, const R *X, const R *Y, R *Xb,
                                    int T, int tx, int ty, int l, bool use_n, R nhx, R nhy, R xb, R yb, R &nbx,
                                    R &nby) {
    nbx = R(0);
    nby = R(0);
    // the same window growth as the forward fit
    int nvalid = 0, n = 0, sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0;
    R a = 0, b = 0, c = 0, d = 0, e = 0, fw = 0;
    int rsel = -1;
    for (int r = 2; r <= sp.rmax && rsel < 0; r++) {
        for (int dy = -r; dy <= r; dy++)
            for (int dx = -r; dx <= r; dx++) {
                if (r > 2 && abs(dx) != r && abs(dy) != r) continue;  // only the new ring
                if (tx + dx < 0 || ty + dy < 0 || tx + dx >= T || ty + dy >= T) continue;
                const int k = (ty + dy) * T + tx + dx;
                const int L = lab[k];
                if (!(L >= 0 && L < l)) continue;
                nvalid++;
                R dn;
                const R wt = adj_weight<R>(lab, k, l, dx, dy, use_n, nhx, nhy, dn);
                if (!(wt > R(0))) continue;
                n++; sx += dx; sy += dy; sxx += dx * dx; syy += dy * dy; sxy += dx * dy;
                const R x = R(dx), y = R(dy), wx = wt * x, wy = wt * y;
                a += wx * x; b += wx * y; c += wx; d += wy * y; e += wy; fw += wt;
            }
        if (nvalid < 3 || n < 3) continue;
        const long long g1 = (long long)n * sxx - (long long)sx * sx;
        const long long g2 = (long long)n * syy - (long long)sy * sy;
        const long long g3 = (long long)n * sxy - (long long)sx * sy;
        if (g1 * g2 - g3 * g3 == 0) continue;
        const R det = a * (d * fw - e * e) - b * (b * fw - c * e) + c * (b * e - c * d);
        if (!(det != R(0))) continue;
        rsel = r;
    }
    if (rsel < 0) return;  // the forward flagged it and wrote NaN
    // full inverse of the symmetric normal matrix M = [[a b c],[b d e],[c e fw]]
    const R C11 = d * fw - e * e, C12 = c * e - b * fw, C13 = b * e - c * d;
    const R C22 = a * fw - c * c, C23 = b * c - a * e, C33 = a * d - b * b;
    const R det = a * C11 + b * C12 + c * C13;
    const R id = R(1) / det;
    const R g0 = C13 * id, g1v = C23 * id, g2 = C33 * id;  // M^-1 e3
    // fit coefficients (needed for the residuals of the weight derivatives)
    R cX[3] = {0, 0, 0}, cY[3] = {0, 0, 0}, xref = 0, yref = 0;
    if (use_n) {
        R bx0 = 0, bx1 = 0, bx2 = 0, by0 = 0, by1 = 0, by2 = 0;
        bool have = false;
        for (int dy = -rsel; dy <= rsel; dy++)
            for (int dx = -rsel; dx <= rsel; dx++) {
                if (tx + dx < 0 || ty + dy < 0 || tx + dx >= T || ty + dy >= T) continue;
                const int k = (ty + dy) * T + tx + dx;
                R dn;
                const R wt = adj_weight<R>(lab, k, l, dx, dy, use_n, nhx, nhy, dn);
                if (!(wt > R(0))) continue;
                if (!have) { xref = X[k]; yref = Y[k]; have = true; }
                const R Xv = X[k] - xref, Yv = Y[k] - yref;
                const R wx = wt * R(dx), wy = wt * R(dy);
                bx0 += wx * Xv; bx1 += wy * Xv; bx2 += wt * Xv;
                by0 += wx * Yv; by1 += wy * Yv; by2 += wt * Yv;
            }
        cX[0] = (C11 * bx0 + C12 * bx1 + C13 * bx2) * id;
        cX[1] = (C12 * bx0 + C22 * bx1 + C23 * bx2) * id;
        cX[2] = (C13 * bx0 + C23 * bx1 + C33 * bx2) * id;
        cY[0] = (C11 * by0 + C12 * by1 + C13 * by2) * id;
        cY[1] = (C12 * by0 + C22 * by1 + C23 * by2) * id;
        cY[2] = (C13 * by0 + C23 * by1 + C33 * by2) * id;
    }
    for (int dy = -rsel; dy <= rsel; dy++)
        for (int dx = -rsel; dx <= rsel; dx++) {
            if (tx + dx < 0 || ty + dy < 0 || tx + dx >= T || ty + dy >= T) continue;
            const int k = (ty + dy) * T + tx + dx;
            R dn;
            const R wt = adj_weight<R>(lab, k, l, dx, dy, use_n, nhx, nhy, dn);
            if (!(wt > R(0))) continue;
            const R gp = g0 * R(dx) + g1v * R(dy) + g2;  // (M^-1 e3) . (dx, dy, 1)
            const R al = wt * gp;
            atomicAdd(&Xb[k], al * xb);
            atomicAdd(&Xb[T * T + k], al * yb);
            if (use_n) {
                // d value / d w_k = gp * residual_k; w_k = 2^-(|dx|+|dy|) * dn
                const R rx = (X[k] - xref) - (cX[0] * R(dx) + cX[1] * R(dy) + cX[2]);
                const R ry = (Y[k] - yref) - (cY[0] * R(dx) + cY[1] * R(dy) + cY[2]);
                const R wb = gp * (xb * rx + yb * ry);
                const R dnb = wb * pow2neg<R>(abs(dx) + abs(dy)) * rinv_tab<R>(dx, dy);
                nbx += -R(dx) * dnb;
                nby += -R(dy) * dnb;
            }
        }
}

template <class R>
__device__ void rmt_adjoint_solid(const SimParams &sp, const RmtAdjArgs<R> &a);

template <class R>
__global__ void __launch_bounds__(RMT_THREADS) rmt_adjoint_kernel(SimParams sp, RmtAdjArgs<R> a) {
    rmt_adjoint_solid<R>(sp, a);
}

// 1024-thread CTAs for FP32 simulations with few solids (as the forward kernel).
template <class R>
__global__ void __launch_bounds__(RMT_THREADS_BIG, 1) rmt_adjoint_kernel_big(SimParams sp, RmtAdjArgs<R> a) {
    rmt_adjoint_solid<R>(sp, a);
}

template <class R>
__device__ void rmt_adjoint_solid(const SimParams &sp, const RmtAdjArgs<R> &a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int bb[4];
    __shared__ int lcnt[24], loff[24];
    const int s = blockIdx.x;
    const SolidDesc sd = a.solids[s];
    const int T = sd.T, TT = T * T;
    const int lane = threadIdx.x & 31;
    signed char *lab = reinterpret_cast<signed char *>(smem);
    const Frame fo = a.frame_out[s], fi = a.frame_in[s];
    const int2 oo = make_int2(fo.ox, fo.oy);
    const int shx = fo.ox - fi.ox, shy = fo.oy - fi.oy;
    const Rsq<R> rq(sd);
    const R *Xi = a.xi_in + sd.off, *Yi = Xi + TT;
    const R *Xo = a.xi_out + sd.off, *Yo = Xo + TT;
    R *XbO = a.xib_out + sd.off;
    R *XbI = a.xib_in + sd.off;
    const R eps = pick<R>(sp.eps, sp.eps_f);
    const long long P = sp.P;
    if (threadIdx.x < 4) bb[threadIdx.x] = (threadIdx.x & 1) ? -(1 << 29) : (1 << 29);
    if (threadIdx.x < 24) lcnt[threadIdx.x] = 0;
    for (int k = threadIdx.x; k < (TT + 15) >> 4; k += blockDim.x)
        reinterpret_cast<int4 *>(lab)[k] = make_int4(-1, -1, -1, -1);
    int sb[4] = {1 << 29, -(1 << 29), 1 << 29, -(1 << 29)};
    __syncthreads();
    // the advected set S^n and its stencil conditions, as the forward
    {
        const int bw = fi.bx1 - fi.bx0 + 1, bn = (fi.bx1 >= fi.bx0 && fi.by1 >= fi.by0) ? bw * (fi.by1 - fi.by0 + 1) : 0;
        for (int kk = threadIdx.x; kk < bn; kk += blockDim.x) {
            const int ix = fi.bx0 + kk % bw, iy = fi.by0 + kk / bw;
            const int lx = ix - shx, ly = iy - shy, gx = oo.x + lx, gy = oo.y + ly;
            const int k = iy * T + ix;
            const R ex = Xi[k];
            if (!(ex == ex)) continue;
            const R phi = phi_eta(ex, Yi[k], ix, iy, fi, rq);
            if (!(phi < eps) || !domain_cell(sp, gx, gy)) continue;
            if (lx < 0 || ly < 0 || lx >= T || ly >= T) continue;
            if (!(phi < -R(PHI_TIE))) continue;
            const long long c = (long long)wrapi(gy, sp.ny) * sp.nx + wrapi(gx, sp.nx);
            const R u = a.tape[P + c], v = a.tape[2 * P + c];
            const int sx = (u >= R(0)) ? -1 : 1, sy = (v >= R(0)) ? -1 : 1;
            const int x2 = ix + 2 * sx, y2 = iy + 2 * sy;
            if (x2 < fi.bx0 || x2 > fi.bx1 || y2 < fi.by0 || y2 > fi.by1) continue;
            lab[ly * T + lx] = 0;
            sb[0] = min(sb[0], lx); sb[1] = max(sb[1], lx); sb[2] = min(sb[2], ly); sb[3] = max(sb[3], ly);
        }
    }
    for (int k = 0; k < 4; k++) warp_minmax(sb[k], (k & 1) == 0);
    if (lane == 0) { atomicMin(&bb[0], sb[0]); atomicMax(&bb[1], sb[1]); atomicMin(&bb[2], sb[2]); atomicMax(&bb[3], sb[3]); }
    __syncthreads();
    const int sx0 = bb[0], sx1 = bb[1], sy0 = bb[2], sy1 = bb[3];
    if (sx0 > sx1) return;
    const int NL = sp.n_layers;
    // the layers, as the forward, listed so that a layer's targets fill whole warps
    int *lists = reinterpret_cast<int *>(smem + ((TT + 15) & ~15));
    label_layers_l1(sp, lab, T, sx0, sx1, sy0, sy1, oo, NL, lcnt);
    __syncthreads();
    const bool listed = list_layers(lab, T, max(sx0 - NL, 0), min(sx1 + NL, T - 1), max(sy0 - NL, 0),
                                    min(sy1 + NL, T - 1), NL, lcnt, loff, lists, 2 * LIST_CAP);
    // extrapolated layers in reverse order
    for (int l = NL; l >= 1; l--) {
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
            const R xb = XbO[t], yb = XbO[TT + t];
            if (xb == R(0) && yb == R(0)) continue;
            bool use_n = false;
            R nhx = 0, nhy = 0, gxp = 0, gyp = 0, nn = 0;
            const int ix = lx + shx, iy = ly + shy;
            if (l <= 2) use_n = adj_normal<R>(Xi, Yi, T, ix, iy, fi, rq, nhx, nhy, gxp, gyp, nn);
            R nbx, nby;
            extrapolate_adjoint<R>(sp, lab, Xo, Yo, XbO, T, lx, ly, l, use_n, nhx, nhy, xb, yb, nbx, nby);
            if (use_n && (nbx != R(0) || nby != R(0))) {
                // n = g / |g|, g = central differences of phi^n
                const R ndot = nhx * nbx + nhy * nby;
                const R gbx = (nbx - nhx * ndot) / nn, gby = (nby - nhy * ndot) / nn;
                const int k0 = iy * T + ix;
                const int kn[4] = {k0 + 1, k0 - 1, k0 + T, k0 - T};
                const int nxo[4] = {1, -1, 0, 0}, nyo[4] = {0, 0, 1, -1};
                const R pbv[4] = {gbx / R(2), -gbx / R(2), gby / R(2), -gby / R(2)};
                for (int m = 0; m < 4; m++) {
                    R dx_, dy_;
                    dphi_deta<R>(Xi[kn[m]], Yi[kn[m]], ix + nxo[m], iy + nyo[m], fi, dx_, dy_);
                    atomicAdd(&XbI[kn[m]], pbv[m] * dx_);
                    atomicAdd(&XbI[TT + kn[m]], pbv[m] * dy_);
                }
            }
        }
        __syncthreads();
    }
    // advected nodes: eta^{n+1} = eta - (u - dd) - u d_x eta - v d_y eta (one-sided, upwind)
    {
        const int w = sx1 - sx0 + 1, nb = w * (sy1 - sy0 + 1);
        for (int k = threadIdx.x; k < nb; k += blockDim.x) {
            const int lx = sx0 + k % w, ly = sy0 + k / w, t = ly * T + lx;
            if (lab[t] != 0) continue;
            const R Xb = XbO[t], Yb = XbO[TT + t];
            if (Xb == R(0) && Yb == R(0)) continue;
            const int ix = lx + shx, iy = ly + shy, kk = iy * T + ix;
            const int gx = oo.x + lx, gy = oo.y + ly;
            const long long c = (long long)wrapi(gy, sp.ny) * sp.nx + wrapi(gx, sp.nx);
            const R rho = a.tape[c], u = a.tape[P + c], v = a.tape[2 * P + c];
            const int sx = (u >= R(0)) ? -1 : 1, sy = (v >= R(0)) ? -1 : 1;
            const int k1 = kk + sx, k2 = kk + 2 * sx, k3 = kk + sy * T, k4 = kk + 2 * sy * T;
            const R hx = R(-sx) * R(0.5), hy = R(-sy) * R(0.5);
            const R ex = Xi[kk], ey = Yi[kk];
            const R dXdx = hx * (R(3) * ex - R(4) * Xi[k1] + Xi[k2]), dYdx = hx * (R(3) * ey - R(4) * Yi[k1] + Yi[k2]);
            const R dXdy = hy * (R(3) * ex - R(4) * Xi[k3] + Xi[k4]), dYdy = hy * (R(3) * ey - R(4) * Yi[k3] + Yi[k4]);
            const R c0 = R(1) - R(3) * (u * hx + v * hy);
            atomicAdd(&XbI[kk], Xb * c0); atomicAdd(&XbI[TT + kk], Yb * c0);
            atomicAdd(&XbI[k1], Xb * R(4) * u * hx); atomicAdd(&XbI[TT + k1], Yb * R(4) * u * hx);
            atomicAdd(&XbI[k2], -Xb * u * hx); atomicAdd(&XbI[TT + k2], -Yb * u * hx);
            atomicAdd(&XbI[k3], Xb * R(4) * v * hy); atomicAdd(&XbI[TT + k3], Yb * R(4) * v * hy);
            atomicAdd(&XbI[k4], -Xb * v * hy); atomicAdd(&XbI[TT + k4], -Yb * v * hy);
            const R ub = -Xb * (R(1) + dXdx) - Yb * dYdx;
            const R vb = -Xb * dXdy - Yb * (R(1) + dYdy);
            // u = (sum c f + half-force) / rho
            const R inv = R(1) / rho;
#pragma unroll
            for (int q = 0; q < 9; q++)
                atomicAdd(&a.fb[q * P + c], ((R(cxq(q)) - u) * ub + (R(cyq(q)) - v) * vb) * inv);
            atomicAdd(&a.cb[c], ub * inv);
            atomicAdd(&a.cb[P + c], vb * inv);
        }
    }
}

// ---------------------------------------------------------------------------
// Centroid c_s = sum lambda x / sum lambda (lambda = 1 - H(phi), domain nodes
// of the solid's tile) and the adjoint of xi for a given dL/dc_s.
// ---------------------------------------------------------------------------
template <class R>
__global__ void centroid_seed_kernel(SimParams sp, const R *xi, const Frame *frames, const SolidDesc *solids,
                                     const double *dLdc, R *xib) {
    __shared__ double red[32 * 3];
    __shared__ double tot[3];
    const int s = blockIdx.x;
    const SolidDesc sd = solids[s];
    const Frame fr = frames[s];
    const Rsq<R> rq(sd);
    const int T = sd.T, TT = T * T;
    const R eps = pick<R>(sp.eps, sp.eps_f);
    const R *X = xi + sd.off, *Y = X + TT;
    double st[3] = {0, 0, 0};
    for (int t = threadIdx.x; t < TT; t += blockDim.x) {
        const int lx = t % T, ly = t / T;
        if (!in_box(fr, lx, ly) || !domain_cell(sp, fr.ox + lx, fr.oy + ly)) continue;
        if (!(X[t] == X[t])) continue;
        const R phi = phi_eta(X[t], Y[t], lx, ly, fr, rq);
        if (!(phi < eps)) continue;
        const double lam = 1.0 - (double)heaviside<R>(phi, eps);
        st[0] += lam; st[1] += lam * (fr.ox + lx); st[2] += lam * (fr.oy + ly);
    }
    block_sum<double, 3>(st, red);
    if (threadIdx.x == 0) { tot[0] = st[0]; tot[1] = st[1]; tot[2] = st[2]; }
    __syncthreads();
    const double lsum = tot[0];
    if (lsum <= 0.0) return;
    const double cx = tot[1] / lsum, cy = tot[2] / lsum;
    const double gx = dLdc[2 * s], gy = dLdc[2 * s + 1];
    R *Xb = xib + sd.off;
    for (int t = threadIdx.x; t < TT; t += blockDim.x) {
        const int lx = t % T, ly = t / T;
        if (!in_box(fr, lx, ly) || !domain_cell(sp, fr.ox + lx, fr.oy + ly)) continue;
        if (!(X[t] == X[t])) continue;
        const R phi = phi_eta(X[t], Y[t], lx, ly, fr, rq);
        if (!(phi < eps)) continue;
        const R lamb = R((gx * (fr.ox + lx - cx) + gy * (fr.oy + ly - cy)) / lsum);
        const R phb = -dheaviside<R>(phi, eps) * lamb;
        R dx_, dy_;
        dphi_deta<R>(X[t], Y[t], lx, ly, fr, dx_, dy_);
        Xb[t] += phb * dx_;
        Xb[TT + t] += phb * dy_;
    }
}

}  // namespace lbrmt
