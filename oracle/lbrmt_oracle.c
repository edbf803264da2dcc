/*
 * lbrmt_oracle.c -- TEST INFRASTRUCTURE ONLY (the parity oracle).
 *
 * A plain, slow, FP64 CPU implementation of one time step of the lattice
 * Boltzmann reference map technique (LBRMT) of Sun & Rycroft, "A
 * fully-integrated lattice Boltzmann method for fluid-structure interaction"
 * (arXiv 2402.12696).  It follows Algorithm 1 step by step:
 *
 *   advect xi (Sec. 3.1, Eqs. 3_1_refmap_adv / 3_1_eno)
 *   extrapolate xi layer by layer (Sec. 3.2, Eq. 3_2_extrap_weight)
 *   relabel phi = phi_0(xi) (Sec. 3.2)
 *   divergence of the blended solid stress + contact (Sec. 3.3, Sec. 3.6,
 *     Eqs. 3_3_refmap_jacobian .. 3_3_div_solid_stress, 2_4_F_divs,
 *     3_6_collision_stress .. 3_6_global_stress)
 *   equilibrium with smooth flux correction (Eqs. 2_3_drho, 2_3_feq_sfc)
 *   Guo forcing term (Eq. 2_2_Fi, times rho as in the expanded Eq. 3_4_Fi)
 *   BGK collision (Eq. 2_2_bgk_force), wall conditions (Sec. 3.5),
 *   streaming, moments with the half-force (Sec. 3.4).
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load this file.  It shares no code, header or constant with the
 * CUDA path.  Where the paper is silent the readings are:
 *   - u == 0 takes the u > 0 (backward) upwind branch;
 *   - the advected set is {domain nodes with phi^n < 0}; a node whose level
 *     set lies within PHI_TIE = 1e-9 of zero counts as not solid, so that
 *     nodes exactly on the initial interface (a disk centred on a node) are
 *     classified the same way whatever the rounding of later steps;
 *   - a directional extrapolation weight whose cosine d.n/|d| is at most
 *     COS_TIE = 1e-9 is zero (the same rule for a node exactly abeam the
 *     target);
 *   - the extrapolation's "ill-defined" fit means fewer than three nodes of
 *     positive weight, or all of them on one line (det M = 0);
 *   - the surface normal of Eq. 3_2_extrap_weight is the central-difference
 *     gradient of the previous step's phi at the target, dropped when a
 *     neighbour is missing or the gradient vanishes;
 *   - Eq. 3_3_refmap_jacobian's printed first y-term xi_{i,j} is read as
 *     xi_{i,j+1} (six-node stencil of Fig. 3_lbrmt B; F = I gives zero stress);
 *   - Eq. 3_4_Fi's F_2 / F_4 "9 v F_x" is read as 9 v F_y (from Eq. 2_2_Fi);
 *   - the half-edge solid fraction uses phi averaged over the edge's two nodes;
 *   - contact acts on half-edges where both solids have phi < eps, the normal
 *     from the same six-node stencil applied to phi_s - phi_t;
 *   - multi-solid density and external accelerations are blended with the
 *     same normalisation as the stress (Eq. 3_6_global_stress);
 *   - moving-wall halfway bounce-back adds 2 w_i rho (c_i . u_w) / c_s^2 with
 *     rho the node's density; a population crossing a side wall and the lid
 *     is treated as crossing the lid;
 *   - initial populations are the SFC equilibrium at rest with rho = rho_t.
 * Parity pins: see tests/test_oracle_pins.py (closed forms, invariants and
 * brute force).  The in-layer weight choice of the extrapolation is "parity
 * unpinned" beyond its exactness on linear fields.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 9
static const int CX[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WQ[NQ] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[NQ] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#define PHI_TIE 1e-9
#define COS_TIE 1e-9

typedef struct {
    int nx, ny, wall_x, wall_y;
    double tau, rho_f, lid_u, eps;
    int n_layers;
    double eta, gravity;
    int force_kind;
    double force_a[2];
    int rmax;
    double *bfield;  /* force_kind 3: per-node body force, x plane then y plane */
    int force_mode;  /* 0: rho F in the Guo term (Eq. 3_4_Fi as printed); 1: rho on the accelerations only */
} ocfg_t;

typedef struct {
    double xc, yc, R, rho_s, G;  /* R: radius of the disk, circumscribed radius of other shapes */
    int shape;                   /* 0 disk, 1 axis-aligned ellipse, 2 axis-aligned rectangle */
    double a, b;                 /* semi-axes / half-sides along x and y */
    int x0, y0, w, h;  /* window in unwrapped coordinates */
    double *X, *Y, *phi;
    signed char *lab;  /* -1 outside S u band, 0 advected solid set, l = layer */
} osolid_t;

typedef struct {
    ocfg_t c;
    int ns, cap;
    osolid_t *s;
    double *f, *fh, *Fi;   /* 9 planes of nx*ny */
    double *rho, *ux, *uy; /* moments */
    double *Fx, *Fy, *drho;/* force density and density difference of the last step */
    double *Fsx, *Fsy;     /* its stress-divergence part (solid and contact stresses) */
    double *Fax, *Fay;     /* and the rest: blended accelerations and body force */
    double *ex, *ey;       /* half-edge accumulators, 7 values per edge */
    double *nl, *nd, *na;  /* node accumulators: sum lambda, sum lambda(rho_s-rho_f), sum lambda a (2) */
    long step;
    int err;
    char msg[256];
} osim_t;

/* ------------------------------------------------------------------------ */
/* Pointwise pieces of the method                                           */
/* ------------------------------------------------------------------------ */

/* Smoothed Heaviside, Eq. 2_3_heaviside. */
double oracle_heaviside(double phi, double eps) {
    if (phi <= -eps) return 0.0;
    if (phi >= eps) return 1.0;
    return 0.5 * (1.0 + phi / eps + sin(M_PI * phi / eps) / M_PI);
}

/* Contact force function f of Eq. 3_6_collision_force. */
static double contact_f(double phi, double eps) {
    return phi < eps ? 0.5 * (1.0 - phi / eps) : 0.0;
}

/* Equilibrium with smooth flux correction, Eq. 2_3_feq_sfc (c_s^2 = 1/3). */
void oracle_feq(double rho, double u, double v, double drho, double out[NQ]) {
    const double cs2 = 1.0 / 3.0;
    double vv = u * u + v * v;
    double sum_w = 0.0;
    for (int i = 1; i < NQ; i++) sum_w += WQ[i];
    for (int i = 0; i < NQ; i++) {
        double cu = CX[i] * u + CY[i] * v;
        double e = WQ[i] * rho * (1.0 + cu / cs2 + (cu * cu - cs2 * vv) / (2.0 * cs2 * cs2));
        if (i == 0) e += sum_w * drho;
        else e -= WQ[i] * drho;
        out[i] = e;
    }
}

/* Guo forcing term, Eq. 2_2_Fi, multiplied by rho as in Eq. 3_4_Fi. */
void oracle_guo(double rho, double u, double v, double Fx, double Fy, double out[NQ]) {
    const double cs2 = 1.0 / 3.0;
    for (int i = 0; i < NQ; i++) {
        double cv = CX[i] * u + CY[i] * v;
        double ax = (CX[i] - u) / cs2 + cv * CX[i] / (cs2 * cs2);
        double ay = (CY[i] - v) / cs2 + cv * CY[i] / (cs2 * cs2);
        out[i] = rho * WQ[i] * (ax * Fx + ay * Fy);
    }
}

/* Incompressible neo-Hookean plane-strain deviatoric stress, Eq. 3_3_solid_stress,
 * from the Jacobian J = d xi / d x (F = J^{-1}, Eq. 3_3_refmap_deformation).
 * tau = (xx, xy, yy). Returns 0 if J is singular. */
int oracle_stress_from_jacobian(double Jxx, double Jxy, double Jyx, double Jyy, double G,
                                double tau[3]) {
    double det = Jxx * Jyy - Jxy * Jyx;
    if (det == 0.0) return 0;
    double Fxx = Jyy / det, Fxy = -Jxy / det, Fyx = -Jyx / det, Fyy = Jxx / det;
    double Bxx = Fxx * Fxx + Fxy * Fxy;
    double Bxy = Fxx * Fyx + Fxy * Fyy;
    double Byy = Fyx * Fyx + Fyy * Fyy;
    double tr = (Bxx + Byy + 1.0) / 3.0;
    tau[0] = G * (Bxx - tr);
    tau[1] = G * Bxy;
    tau[2] = G * (Byy - tr);
    return 1;
}

/* Half-edge Jacobian, Eq. 3_3_refmap_jacobian.  The six nodes are given as
 * a[k], b[k] for k = 0 (row below), 1 (edge row), 2 (row above); for an
 * x-edge (i-1/2, j) a = column i-1 and b = column i.  For a y-edge the caller
 * passes the transposed stencil and swaps the result. */
static void edge_grad(const double a[3], const double b[3], double *dn, double *dt) {
    *dn = b[1] - a[1];
    *dt = (b[2] + a[2] - b[0] - a[0]) / 4.0;
}

/* Contact stress, Eq. 3_6_collision_stress, for normal (nx, ny). */
static void contact_stress(double fmin, double Gs, double Gt, double eta, double nx, double ny,
                           double tau[3]) {
    double k = -eta * fmin * (Gs + Gt);
    tau[0] = k * (nx * nx - 0.5);
    tau[1] = k * (nx * ny);
    tau[2] = k * (ny * ny - 0.5);
}

void oracle_contact_stress(double phi_s, double phi_t, double Gs, double Gt, double eta,
                           double eps, double gx, double gy, double tau[3]) {
    double fm = fmin(contact_f(phi_s, eps), contact_f(phi_t, eps));
    double nrm = sqrt(gx * gx + gy * gy);
    tau[0] = tau[1] = tau[2] = 0.0;
    if (fm <= 0.0 || nrm == 0.0) return;
    contact_stress(fm, Gs, Gt, eta, gx / nrm, gy / nrm, tau);
}

/* Solve the 3x3 system M p = b (two right-hand sides) by Gaussian
 * elimination with partial pivoting.  Returns 0 if a pivot vanishes. */
static int solve3(double M[3][3], double b1[3], double b2[3]) {
    for (int c = 0; c < 3; c++) {
        int p = c;
        for (int r = c + 1; r < 3; r++)
            if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
        if (M[p][c] == 0.0) return 0;
        if (p != c) {
            for (int k = 0; k < 3; k++) { double t = M[c][k]; M[c][k] = M[p][k]; M[p][k] = t; }
            double t = b1[c]; b1[c] = b1[p]; b1[p] = t;
            t = b2[c]; b2[c] = b2[p]; b2[p] = t;
        }
        for (int r = c + 1; r < 3; r++) {
            double m = M[r][c] / M[c][c];
            for (int k = c; k < 3; k++) M[r][k] -= m * M[c][k];
            b1[r] -= m * b1[c];
            b2[r] -= m * b2[c];
        }
    }
    for (int r = 2; r >= 0; r--) {
        for (int k = r + 1; k < 3; k++) { b1[r] -= M[r][k] * b1[k]; b2[r] -= M[r][k] * b2[k]; }
        b1[r] /= M[r][r];
        b2[r] /= M[r][r];
    }
    return 1;
}

/* Weighted least-squares extrapolation of one target node (Sec. 3.2 steps
 * (i)-(iii)).  The grid is w*h with labels lab (-1: not valid, 0: solid,
 * l>0: band layer l) and values X, Y.  Valid nodes for a target of layer l
 * are those with 0 <= lab < l.  (use_normal, nhx, nhy) is the surface normal
 * for l <= 2.  Returns the final window half-width r, or -1 if r would exceed
 * rmax. */
int oracle_extrap_target(int w, int h, const signed char *lab, const double *X,
                         const double *Y, int tx, int ty, int l, int use_normal,
                         double nhx, double nhy, int rmax, double *outX, double *outY) {
    for (int r = 2; r <= rmax; r++) {
        int nvalid = 0;
        for (int dy = -r; dy <= r; dy++)
            for (int dx = -r; dx <= r; dx++) {
                int x = tx + dx, y = ty + dy;
                if (x < 0 || y < 0 || x >= w || y >= h) continue;
                int L = lab[y * w + x];
                if (L >= 0 && L < l) nvalid++;
            }
        if (nvalid < 3) continue;
        double M[3][3] = {{0}}, bX[3] = {0}, bY[3] = {0};
        int npos = 0, p0x = 0, p0y = 0, p1x = 0, p1y = 0, have1 = 0, noncol = 0;
        for (int dy = -r; dy <= r; dy++)
            for (int dx = -r; dx <= r; dx++) {
                int x = tx + dx, y = ty + dy;
                if (x < 0 || y < 0 || x >= w || y >= h) continue;
                int L = lab[y * w + x];
                if (!(L >= 0 && L < l)) continue;
                double wt = ldexp(1.0, -(abs(dx) + abs(dy)));
                if (l <= 2 && use_normal) {
                    /* d = target - valid node */
                    double ddx = -dx, ddy = -dy;
                    double dn = (ddx * nhx + ddy * nhy) / sqrt(ddx * ddx + ddy * ddy);
                    wt = dn > COS_TIE ? dn * wt : 0.0;
                }
                if (!(wt > 0.0)) continue;
                /* collinearity bookkeeping on integer offsets */
                if (npos == 0) { p0x = dx; p0y = dy; }
                else if (!have1) { p1x = dx; p1y = dy; have1 = 1; }
                else if (!noncol) {
                    long cr = (long)(p1x - p0x) * (dy - p0y) - (long)(p1y - p0y) * (dx - p0x);
                    if (cr != 0) noncol = 1;
                }
                npos++;
                double xv = dx, yv = dy, v[3] = {xv, yv, 1.0};
                for (int a = 0; a < 3; a++) {
                    for (int b = 0; b < 3; b++) M[a][b] += wt * v[a] * v[b];
                    bX[a] += wt * v[a] * X[y * w + x];
                    bY[a] += wt * v[a] * Y[y * w + x];
                }
            }
        if (npos < 3 || !noncol) continue;
        if (!solve3(M, bX, bY)) continue;
        *outX = bX[2];
        *outY = bY[2];
        return r;
    }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* Simulation state                                                         */
/* ------------------------------------------------------------------------ */

static int wrapi(int g, int n) { int r = g % n; return r < 0 ? r + n : r; }

/* Distance from (y0, y1), y0, y1 >= 0, to the ellipse (x/e0)^2 + (y/e1)^2 = 1
 * with e0 >= e1 > 0.  The closest point is x_i = e_i^2 y_i / (t + e_i^2) for
 * the root t of sum_i (e_i y_i / (t + e_i^2))^2 = 1; in s = t / e1^2 that root
 * is bracketed and found by bisection to full precision (Eberly's method for
 * the distance from a point to an ellipse). */
static double ellipse_dist_q1(double e0, double e1, double y0, double y1) {
    if (y1 > 0) {
        if (y0 > 0) {
            double z0 = y0 / e0, z1 = y1 / e1, g = z0 * z0 + z1 * z1 - 1.0;
            if (g == 0.0) return 0.0;
            double r0 = (e0 / e1) * (e0 / e1), n0 = r0 * z0;
            double s0 = z1 - 1.0, s1 = g < 0 ? 0.0 : hypot(n0, z1) - 1.0, sm = 0.0;
            for (int it = 0; it < 2000; it++) {
                sm = 0.5 * (s0 + s1);
                if (sm == s0 || sm == s1) break;
                double ra = n0 / (sm + r0), rb = z1 / (sm + 1.0), f = ra * ra + rb * rb - 1.0;
                if (f > 0) s0 = sm;
                else if (f < 0) s1 = sm;
                else break;
            }
            double x0 = r0 * y0 / (sm + r0), x1 = y1 / (sm + 1.0);
            return hypot(x0 - y0, x1 - y1);
        }
        return fabs(y1 - e1);
    }
    double numer0 = e0 * y0, denom0 = e0 * e0 - e1 * e1;
    if (numer0 < denom0) {
        double xde0 = numer0 / denom0, x0 = e0 * xde0, x1 = e1 * sqrt(1.0 - xde0 * xde0);
        return hypot(x0 - y0, x1);
    }
    return fabs(y0 - e0);
}

/* Signed distance (negative inside) of (qx, qy) relative to the centre to an
 * axis-aligned shape: 0 disk of radius a, 1 ellipse with semi-axes a (x) and
 * b (y), 2 rectangle with half-sides a and b. */
double oracle_phi0(int shape, double a, double b, double qx, double qy) {
    if (shape == 1) {
        double y0 = fabs(qx), y1 = fabs(qy), e0 = a, e1 = b;
        if (e0 < e1) { double t = e0; e0 = e1; e1 = t; t = y0; y0 = y1; y1 = t; }
        double d = ellipse_dist_q1(e0, e1, y0, y1);
        return (y0 / e0) * (y0 / e0) + (y1 / e1) * (y1 / e1) < 1.0 ? -d : d;
    }
    if (shape == 2) {
        double dx = fabs(qx) - a, dy = fabs(qy) - b;
        return hypot(fmax(dx, 0.0), fmax(dy, 0.0)) + fmin(fmax(dx, dy), 0.0);
    }
    return hypot(qx, qy) - a;
}

static double phi0(const osolid_t *s, double X, double Y) {
    return oracle_phi0(s->shape, s->a, s->b, X - s->xc, Y - s->yc);
}

static int seterr(osim_t *m, const char *msg) {
    if (!m->err) { m->err = 1; snprintf(m->msg, sizeof m->msg, "%s", msg); }
    return -1;
}

/* Band cells may not go beyond the two pad layers of a no-slip side. */
static int allowed(const ocfg_t *c, int gx, int gy) {
    if (c->wall_x && (gx < -2 || gx > c->nx + 1)) return 0;
    if (c->wall_y && (gy < -2 || gy > c->ny + 1)) return 0;
    return 1;
}

static int in_domain(const ocfg_t *c, int gx, int gy) {
    if (c->wall_x && (gx < 0 || gx >= c->nx)) return 0;
    if (c->wall_y && (gy < 0 || gy >= c->ny)) return 0;
    return 1;
}

static int widx(const osolid_t *s, int gx, int gy) {
    int lx = gx - s->x0, ly = gy - s->y0;
    if (lx < 0 || ly < 0 || lx >= s->w || ly >= s->h) return -1;
    return ly * s->w + lx;
}

/* Window index of the image of grid node (x, y) (periodic coordinates wrapped
 * to [0, n), wall coordinates raw) inside solid s's unwrapped window; -1 if
 * none. Writes the unwrapped coordinates. */
static int lookup(const ocfg_t *c, const osolid_t *s, int x, int y, int *gx, int *gy) {
    int ux = c->wall_x ? x : s->x0 + wrapi(x - s->x0, c->nx);
    int uy = c->wall_y ? y : s->y0 + wrapi(y - s->y0, c->ny);
    *gx = ux; *gy = uy;
    return widx(s, ux, uy);
}

static void free_window(osolid_t *s) {
    free(s->X); free(s->Y); free(s->phi); free(s->lab);
    s->X = s->Y = s->phi = NULL; s->lab = NULL;
}

static int alloc_window(osolid_t *s, int x0, int y0, int w, int h) {
    s->x0 = x0; s->y0 = y0; s->w = w; s->h = h;
    size_t n = (size_t)w * h;
    s->X = malloc(n * sizeof(double));
    s->Y = malloc(n * sizeof(double));
    s->phi = malloc(n * sizeof(double));
    s->lab = malloc(n);
    if (!s->X || !s->Y || !s->phi || !s->lab) return -1;
    for (size_t k = 0; k < n; k++) { s->X[k] = s->Y[k] = s->phi[k] = NAN; s->lab[k] = -1; }
    return 0;
}

/* Window of bbox(S) grown by the layer count (+1), clipped to the pads. */
static int window_for(const osim_t *m, int bx0, int by0, int bx1, int by1,
                      int *x0, int *y0, int *w, int *h) {
    const ocfg_t *c = &m->c;
    int g = c->n_layers + 1;
    int a0 = bx0 - g, a1 = bx1 + g, b0 = by0 - g, b1 = by1 + g;
    if (c->wall_x) { if (a0 < -2) a0 = -2; if (a1 > c->nx + 1) a1 = c->nx + 1; }
    if (c->wall_y) { if (b0 < -2) b0 = -2; if (b1 > c->ny + 1) b1 = c->ny + 1; }
    *x0 = a0; *y0 = b0; *w = a1 - a0 + 1; *h = b1 - b0 + 1;
    if ((!c->wall_x && *w >= c->nx) || (!c->wall_y && *h >= c->ny)) return -1;
    return 0;
}

/* Mark layers 1..L by 4-neighbour dilation of the solid set and extrapolate
 * each layer from the valid nodes (Sec. 3.2).  old: previous window (for the
 * surface normal from phi^n), may be NULL at initialisation (then the values
 * are simply xi = x and no fit is needed). */
static int layers_and_extrapolate(osim_t *m, osolid_t *s, const osolid_t *old, int init) {
    const ocfg_t *c = &m->c;
    int w = s->w, h = s->h;
    signed char *cand = malloc((size_t)w * h);
    if (!cand) return seterr(m, "out of memory");
    for (int l = 1; l <= c->n_layers; l++) {
        memset(cand, 0, (size_t)w * h);
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                if (s->lab[y * w + x] != -1) continue;
                if (!allowed(c, s->x0 + x, s->y0 + y)) continue;
                static const int nb[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
                for (int k = 0; k < 4; k++) {
                    int xx = x + nb[k][0], yy = y + nb[k][1];
                    if (xx < 0 || yy < 0 || xx >= w || yy >= h) continue;
                    if (s->lab[yy * w + xx] == l - 1) { cand[y * w + x] = 1; break; }
                }
            }
        for (int k = 0; k < w * h; k++)
            if (cand[k]) s->lab[k] = (signed char)l;
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                int k = y * w + x;
                if (s->lab[k] != l) continue;
                int gx = s->x0 + x, gy = s->y0 + y;
                if (init) { s->X[k] = gx; s->Y[k] = gy; continue; }
                int use_n = 0;
                double nhx = 0, nhy = 0;
                if (l <= 2 && old) {
                    int ke = widx(old, gx + 1, gy), kw = widx(old, gx - 1, gy);
                    int kn = widx(old, gx, gy + 1), ks = widx(old, gx, gy - 1);
                    if (ke >= 0 && kw >= 0 && kn >= 0 && ks >= 0 && old->lab[ke] >= 0 &&
                        old->lab[kw] >= 0 && old->lab[kn] >= 0 && old->lab[ks] >= 0) {
                        double gxp = (old->phi[ke] - old->phi[kw]) / 2.0;
                        double gyp = (old->phi[kn] - old->phi[ks]) / 2.0;
                        double nn = sqrt(gxp * gxp + gyp * gyp);
                        if (nn > 0.0) { use_n = 1; nhx = gxp / nn; nhy = gyp / nn; }
                    }
                }
                double ox, oy;
                int r = oracle_extrap_target(w, h, s->lab, s->X, s->Y, x, y, l, use_n, nhx, nhy,
                                             c->rmax, &ox, &oy);
                if (r < 0) { free(cand); return seterr(m, "extrapolation window exceeded rmax"); }
                s->X[k] = ox;
                s->Y[k] = oy;
            }
    }
    free(cand);
    /* relabel: phi = phi_0(xi) on S u band */
    for (int k = 0; k < w * h; k++)
        if (s->lab[k] >= 0) s->phi[k] = phi0(s, s->X[k], s->Y[k]);
    return 0;
}

static int init_solid(osim_t *m, osolid_t *s) {
    const ocfg_t *c = &m->c;
    /* solid set S0 = domain nodes with phi_0(x) < 0 (unwrapped around the centre) */
    int bx0 = (int)floor(s->xc - s->R) - 1, bx1 = (int)ceil(s->xc + s->R) + 1;
    int by0 = (int)floor(s->yc - s->R) - 1, by1 = (int)ceil(s->yc + s->R) + 1;
    int sx0 = 1 << 30, sx1 = -(1 << 30), sy0 = 1 << 30, sy1 = -(1 << 30);
    for (int gy = by0; gy <= by1; gy++)
        for (int gx = bx0; gx <= bx1; gx++)
            if (in_domain(c, gx, gy) && phi0(s, gx, gy) < -PHI_TIE) {
                if (gx < sx0) { sx0 = gx; }
                if (gx > sx1) { sx1 = gx; }
                if (gy < sy0) { sy0 = gy; }
                if (gy > sy1) { sy1 = gy; }
            }
    if (sx0 > sx1) return seterr(m, "solid covers no node");
    int x0, y0, w, h;
    if (window_for(m, sx0, sy0, sx1, sy1, &x0, &y0, &w, &h)) return seterr(m, "solid window too large");
    if (alloc_window(s, x0, y0, w, h)) return seterr(m, "out of memory");
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            int gx = x0 + x, gy = y0 + y;
            if (in_domain(c, gx, gy) && phi0(s, gx, gy) < -PHI_TIE) {
                int k = y * w + x;
                s->lab[k] = 0; s->X[k] = gx; s->Y[k] = gy;
            }
        }
    return layers_and_extrapolate(m, s, NULL, 1);
}

/* Steps 1-3 of the loop of Algorithm 1 for one solid. */
static int update_solid(osim_t *m, osolid_t *s) {
    const ocfg_t *c = &m->c;
    int nx = c->nx;
    /* advected set S = domain nodes with phi^n < 0 */
    int sx0 = 1 << 30, sx1 = -(1 << 30), sy0 = 1 << 30, sy1 = -(1 << 30);
    for (int y = 0; y < s->h; y++)
        for (int x = 0; x < s->w; x++) {
            int k = y * s->w + x, gx = s->x0 + x, gy = s->y0 + y;
            if (s->lab[k] >= 0 && s->phi[k] < -PHI_TIE && in_domain(c, gx, gy)) {
                if (gx < sx0) { sx0 = gx; }
                if (gx > sx1) { sx1 = gx; }
                if (gy < sy0) { sy0 = gy; }
                if (gy > sy1) { sy1 = gy; }
            }
        }
    if (sx0 > sx1) return seterr(m, "solid vanished");
    osolid_t old = *s, nw = *s;
    int x0, y0, w, h;
    if (window_for(m, sx0, sy0, sx1, sy1, &x0, &y0, &w, &h)) return seterr(m, "solid window too large");
    if (alloc_window(&nw, x0, y0, w, h)) return seterr(m, "out of memory");
    /* advection, Eqs. 3_1_refmap_adv and 3_1_eno (Jacobi: reads xi^n only) */
    for (int y = 0; y < s->h; y++)
        for (int x = 0; x < s->w; x++) {
            int k = y * s->w + x, gx = s->x0 + x, gy = s->y0 + y;
            if (!(s->lab[k] >= 0 && s->phi[k] < -PHI_TIE && in_domain(c, gx, gy))) continue;
            int cell = wrapi(gy, c->ny) * nx + wrapi(gx, nx);
            double u = m->ux[cell], v = m->uy[cell];
            int sx = (u >= 0.0) ? -1 : 1; /* backward for u >= 0 */
            int sy = (v >= 0.0) ? -1 : 1;
            int k1 = widx(s, gx + sx, gy), k2 = widx(s, gx + 2 * sx, gy);
            int k3 = widx(s, gx, gy + sy), k4 = widx(s, gx, gy + 2 * sy);
            if (k1 < 0 || k2 < 0 || k3 < 0 || k4 < 0 || s->lab[k1] < 0 || s->lab[k2] < 0 ||
                s->lab[k3] < 0 || s->lab[k4] < 0) {
                free_window(&nw);
                return seterr(m, "advection stencil leaves the band");
            }
            /* (3 xi_0 - 4 xi_1 + xi_2) / 2 with the sign of the one-sided direction */
            double dXdx = -sx * (3.0 * s->X[k] - 4.0 * s->X[k1] + s->X[k2]) / 2.0;
            double dYdx = -sx * (3.0 * s->Y[k] - 4.0 * s->Y[k1] + s->Y[k2]) / 2.0;
            double dXdy = -sy * (3.0 * s->X[k] - 4.0 * s->X[k3] + s->X[k4]) / 2.0;
            double dYdy = -sy * (3.0 * s->Y[k] - 4.0 * s->Y[k3] + s->Y[k4]) / 2.0;
            int kn = widx(&nw, gx, gy);
            nw.X[kn] = s->X[k] - (u * dXdx + v * dXdy);
            nw.Y[kn] = s->Y[k] - (u * dYdx + v * dYdy);
            nw.lab[kn] = 0;
        }
    int rc = layers_and_extrapolate(m, &nw, &old, 0);
    free_window(&old);
    *s = nw;
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Force density (Sec. 3.3, 3.6) and LB update (Sec. 3.4, 3.5)              */
/* ------------------------------------------------------------------------ */

#define EV 7 /* per edge: sum lambda*tau (3), sum lambda, contact tau (3) */

/* External body force of node (i, j) (Eq. 2_4_F_divs), acting on all phases. */
static void body_force(const ocfg_t *c, int i, int j, double *fx, double *fy) {
    *fx = *fy = 0.0;
    if (c->force_kind == 1) { *fx = c->force_a[0]; *fy = c->force_a[1]; }
    else if (c->force_kind == 2) *fx = c->force_a[0] * sin(2.0 * M_PI * j / c->ny);
    else if (c->force_kind == 3 && c->bfield) {
        long cell = (long)j * c->nx + i;
        *fx = c->bfield[cell];
        *fy = c->bfield[(long)c->nx * c->ny + cell];
    }
}

/* Edge array index of the x-edge (dir 0) between (gx-1, gy) and (gx, gy), or the
 * y-edge (dir 1) between (gx, gy-1) and (gx, gy); -1 if not a domain edge. */
static long edge_index(const ocfg_t *c, int dir, int gx, int gy) {
    int nx = c->nx, ny = c->ny;
    int ex = gx, ey = gy;
    if (dir == 0) {
        if (c->wall_x) { if (ex < 0 || ex > nx) return -1; } else ex = wrapi(ex, nx);
        if (c->wall_y) { if (ey < 0 || ey >= ny) return -1; } else ey = wrapi(ey, ny);
    } else {
        if (c->wall_x) { if (ex < 0 || ex >= nx) return -1; } else ex = wrapi(ex, nx);
        if (c->wall_y) { if (ey < 0 || ey > ny) return -1; } else ey = wrapi(ey, ny);
    }
    return (long)ey * (nx + 1) + ex;
}

/* Do the windows [a0, a0 + aw) and [b0, b0 + bw) share a coordinate, the
 * periodic images of the second included? */
static int windows_meet_1d(int a0, int aw, int b0, int bw, int n, int periodic) {
    for (int k = periodic ? -2 : 0; k <= (periodic ? 2 : 0); k++) {
        const int lo = b0 + k * n;
        if (a0 < lo + bw && lo < a0 + aw) return 1;
    }
    return 0;
}

/* Do two solids' windows share a grid node? */
static int windows_meet(const ocfg_t *c, const osolid_t *s, const osolid_t *t) {
    return windows_meet_1d(s->x0, s->w, t->x0, t->w, c->nx, !c->wall_x) &&
           windows_meet_1d(s->y0, s->h, t->y0, t->h, c->ny, !c->wall_y);
}

/* Exported for the tests: do the windows (x0a, y0a, wa x ha) and
 * (x0b, y0b, wb x hb) of a grid nx x ny (walls per axis) share a node? */
int oracle_windows_meet(int x0a, int y0a, int wa, int ha, int x0b, int y0b, int wb, int hb, int nx, int ny,
                        int wall_x, int wall_y) {
    return windows_meet_1d(x0a, wa, x0b, wb, nx, !wall_x) && windows_meet_1d(y0a, ha, y0b, hb, ny, !wall_y);
}

/* Gather the 2x3 stencil of an edge for one solid.  For dir 0 (x-edge at
 * (gx-1/2, gy)): a = column gx-1, b = column gx, rows gy-1..gy+1.  For dir 1
 * (y-edge at (gx, gy-1/2)): a = row gy-1, b = row gy, columns gx-1..gx+1.
 * Returns 0 if a node is not valid. */
static int edge_stencil(const osolid_t *s, int dir, int gx, int gy, double aX[3], double bX[3],
                        double aY[3], double bY[3], double ap[3], double bp[3]) {
    for (int t = 0; t < 3; t++) {
        int ax, ay, bx, by;
        if (dir == 0) { ax = gx - 1; bx = gx; ay = by = gy - 1 + t; }
        else { ay = gy - 1; by = gy; ax = bx = gx - 1 + t; }
        int ka = widx(s, ax, ay), kb = widx(s, bx, by);
        if (ka < 0 || kb < 0 || s->lab[ka] < 0 || s->lab[kb] < 0) return 0;
        aX[t] = s->X[ka]; bX[t] = s->X[kb];
        aY[t] = s->Y[ka]; bY[t] = s->Y[kb];
        ap[t] = s->phi[ka]; bp[t] = s->phi[kb];
    }
    return 1;
}

/* Contact stress of the pair (s, t) on the half-edge of direction dir at s's
 * unwrapped node (gx, gy) (Eqs. 3_6_collision_stress .. 3_6_normal): nonzero
 * where both solids' six-node stencils lie in their bands and both edge means
 * of phi are below eps.  Returns 0 where the pair has no contact stress. */
static int pair_edge_stress(const osim_t *m, const osolid_t *s, const osolid_t *t, int dir, int gx, int gy,
                            double tau[3]) {
    const ocfg_t *c = &m->c;
    double aX[3], bX[3], aY[3], bY[3], ap[3], bp[3];
    if (!edge_stencil(s, dir, gx, gy, aX, bX, aY, bY, ap, bp)) return 0;
    int wx = c->wall_x ? gx : wrapi(gx, c->nx);
    int wy = c->wall_y ? gy : wrapi(gy, c->ny);
    int tx, ty;
    lookup(c, t, wx, wy, &tx, &ty);
    double tX[3], uX[3], tY[3], uY[3], tp[3], up[3];
    if (!edge_stencil(t, dir, tx, ty, tX, uX, tY, uY, tp, up)) return 0;
    double phs = 0.5 * (ap[1] + bp[1]), pht = 0.5 * (tp[1] + up[1]);
    double fm = fmin(contact_f(phs, c->eps), contact_f(pht, c->eps));
    if (!(fm > 0.0)) return 0;
    double pa[3], pb[3];
    for (int q = 0; q < 3; q++) { pa[q] = ap[q] - tp[q]; pb[q] = bp[q] - up[q]; }
    double gn, gt;
    edge_grad(pa, pb, &gn, &gt);
    double gxx = dir == 0 ? gn : gt, gyy = dir == 0 ? gt : gn;
    double nrm = sqrt(gxx * gxx + gyy * gyy);
    if (nrm == 0.0) return 0;
    contact_stress(fm, s->G, t->G, c->eta, gxx / nrm, gyy / nrm, tau);
    return 1;
}

static void compute_force(osim_t *m) {
    const ocfg_t *c = &m->c;
    int nx = c->nx, ny = c->ny;
    long N = (long)nx * ny;
    long NE = (long)(nx + 1) * (ny + 1);
    memset(m->ex, 0, sizeof(double) * EV * NE);
    memset(m->ey, 0, sizeof(double) * EV * NE);
    memset(m->nl, 0, sizeof(double) * N);
    memset(m->nd, 0, sizeof(double) * N);
    memset(m->na, 0, sizeof(double) * 2 * N);
    /* solid stresses at half-edges, accumulated in solid order */
    for (int si = 0; si < m->ns; si++) {
        const osolid_t *s = &m->s[si];
        for (int dir = 0; dir < 2; dir++)
            for (int y = 0; y < s->h; y++)
                for (int x = 0; x < s->w; x++) {
                    int gx = s->x0 + x, gy = s->y0 + y;
                    long e = edge_index(c, dir, gx, gy);
                    if (e < 0) continue;
                    double aX[3], bX[3], aY[3], bY[3], ap[3], bp[3];
                    if (!edge_stencil(s, dir, gx, gy, aX, bX, aY, bY, ap, bp)) continue;
                    /* beyond the blur zone the solid's stress has weight lambda = 0 in
                     * Eq. 3_6_global_stress: it is not formed (nor its Jacobian checked) */
                    if (!(0.5 * (ap[1] + bp[1]) < c->eps)) continue;
                    double lam = 1.0 - oracle_heaviside(0.5 * (ap[1] + bp[1]), c->eps);
                    double dXn, dXt, dYn, dYt, tau[3] = {0, 0, 0};
                    edge_grad(aX, bX, &dXn, &dXt);
                    edge_grad(aY, bY, &dYn, &dYt);
                    int ok;
                    if (dir == 0) ok = oracle_stress_from_jacobian(dXn, dXt, dYn, dYt, s->G, tau);
                    else ok = oracle_stress_from_jacobian(dXt, dXn, dYt, dYn, s->G, tau);
                    if (!ok) { seterr(m, "singular reference-map Jacobian"); continue; }
                    double *E = (dir == 0 ? m->ex : m->ey) + EV * e;
                    E[0] += lam * tau[0]; E[1] += lam * tau[1]; E[2] += lam * tau[2];
                    E[3] += lam;
                }
        /* node terms: solid fraction, density difference, solid acceleration */
        for (int y = 0; y < s->h; y++)
            for (int x = 0; x < s->w; x++) {
                int k = y * s->w + x, gx = s->x0 + x, gy = s->y0 + y;
                if (s->lab[k] < 0 || !in_domain(c, gx, gy)) continue;
                int cell = wrapi(gy, ny) * nx + wrapi(gx, nx);
                double lam = 1.0 - oracle_heaviside(s->phi[k], c->eps);
                double fbx, fby;
                body_force(c, wrapi(gx, nx), wrapi(gy, ny), &fbx, &fby);
                double ax = fbx, ay = fby - (1.0 - c->rho_f / s->rho_s) * c->gravity;
                m->nl[cell] += lam;
                m->nd[cell] += lam * (s->rho_s - c->rho_f);
                m->na[2 * cell] += lam * ax;
                m->na[2 * cell + 1] += lam * ay;
            }
    }
    /* contact stress between every pair of solids (Sec. 3.6); a pair whose
     * windows share no grid node has no edge whose stencil lies in both, so it
     * contributes nothing and is passed over */
    for (int si = 0; si < m->ns; si++)
        for (int ti = si + 1; ti < m->ns; ti++) {
            const osolid_t *s = &m->s[si], *t = &m->s[ti];
            if (!windows_meet(c, s, t)) continue;
            for (int dir = 0; dir < 2; dir++)
                for (int y = 0; y < s->h; y++)
                    for (int x = 0; x < s->w; x++) {
                        int gx = s->x0 + x, gy = s->y0 + y;
                        long e = edge_index(c, dir, gx, gy);
                        if (e < 0) continue;
                        double tau[3];
                        if (!pair_edge_stress(m, s, t, dir, gx, gy, tau)) continue;
                        double *E = (dir == 0 ? m->ex : m->ey) + EV * e;
                        E[4] += tau[0]; E[5] += tau[1]; E[6] += tau[2];
                    }
        }
    /* divergence of the global solid stress (Eq. 3_3_div_solid_stress) and
     * the smoothed force density (Eq. 2_4_F_divs with Eq. 3_6_global_stress) */
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            double tl[3], tr[3], tb[3], tt[3];
            const double *E[4] = {m->ex + EV * edge_index(c, 0, i, j),
                                  m->ex + EV * edge_index(c, 0, i + 1, j),
                                  m->ey + EV * edge_index(c, 1, i, j),
                                  m->ey + EV * edge_index(c, 1, i, j + 1)};
            double *T[4] = {tl, tr, tb, tt};
            for (int q = 0; q < 4; q++) {
                double L = E[q][3];
                for (int a = 0; a < 3; a++) {
                    double sol = L > 1.0 ? E[q][a] / L : E[q][a];
                    T[q][a] = sol + E[q][4 + a];
                }
            }
            double fsx = (tr[0] - tl[0]) + (tt[1] - tb[1]);
            double fsy = (tr[1] - tl[1]) + (tt[2] - tb[2]);
            long cell = (long)j * nx + i;
            double L = m->nl[cell];
            double ax = m->na[2 * cell], ay = m->na[2 * cell + 1], dr = m->nd[cell];
            if (L > 1.0) { ax /= L; ay /= L; dr /= L; }
            double Hf = 1.0 - fmin(1.0, L);
            double fbx, fby;
            body_force(c, i, j, &fbx, &fby);
            m->Fx[cell] = fsx + ax + Hf * fbx;
            m->Fy[cell] = fsy + ay + Hf * fby;
            m->Fsx[cell] = fsx;
            m->Fsy[cell] = fsy;
            m->Fax[cell] = ax + Hf * fbx;
            m->Fay[cell] = ay + Hf * fby;
            m->drho[cell] = dr;
        }
}

static void lb_update(osim_t *m) {
    const ocfg_t *c = &m->c;
    int nx = c->nx, ny = c->ny;
    long N = (long)nx * ny;
    double tau = c->tau;
    /* equilibrium, forcing, collision (Eq. 2_2_bgk_force) */
#pragma omp parallel for schedule(static)
    for (long cell = 0; cell < N; cell++) {
        double feq[NQ], Fi[NQ];
        oracle_feq(m->rho[cell], m->ux[cell], m->uy[cell], m->drho[cell], feq);
        if (c->force_mode == 1) {
            /* conservative form: the stress divergence without rho, the
             * accelerations with it (the Guo term is linear in rho F) */
            double Fs[NQ];
            oracle_guo(m->rho[cell], m->ux[cell], m->uy[cell], m->Fax[cell], m->Fay[cell], Fi);
            oracle_guo(1.0, m->ux[cell], m->uy[cell], m->Fsx[cell], m->Fsy[cell], Fs);
            for (int q = 0; q < NQ; q++) Fi[q] += Fs[q];
        } else {
            oracle_guo(m->rho[cell], m->ux[cell], m->uy[cell], m->Fx[cell], m->Fy[cell], Fi);
        }
        for (int q = 0; q < NQ; q++) {
            double fq = m->f[q * N + cell];
            m->fh[q * N + cell] = fq - (fq - feq[q]) / tau + (1.0 - 1.0 / (2.0 * tau)) * Fi[q];
            m->Fi[q * N + cell] = Fi[q];
        }
    }
    /* wall conditions and streaming (pull form of the buffer-node copy, Sec. 3.5) */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            long cell = (long)j * nx + i;
            for (int q = 0; q < NQ; q++) {
                int sx = i - CX[q], sy = j - CY[q];
                int out_x = sx < 0 || sx >= nx, out_y = sy < 0 || sy >= ny;
                int wall = (out_x && c->wall_x) || (out_y && c->wall_y);
                if (wall) {
                    double uwx = 0.0, uwy = 0.0;
                    if (out_y && c->wall_y && sy >= ny) uwx = c->lid_u; /* top wall is the lid */
                    double cu = CX[q] * uwx + CY[q] * uwy;
                    m->f[q * N + cell] = m->fh[OPP[q] * N + cell] + 2.0 * WQ[q] * m->rho[cell] * cu * 3.0;
                } else {
                    long src = (long)wrapi(sy, ny) * nx + wrapi(sx, nx);
                    m->f[q * N + cell] = m->fh[q * N + src];
                }
            }
        }
    /* moments with the half-force correction (Sec. 3.4) */
#pragma omp parallel for schedule(static)
    for (long cell = 0; cell < N; cell++) {
        double r = 0, jx = 0, jy = 0, hx = 0, hy = 0;
        for (int q = 0; q < NQ; q++) {
            double fq = m->f[q * N + cell], Fq = m->Fi[q * N + cell];
            r += fq; jx += CX[q] * fq; jy += CY[q] * fq;
            hx += CX[q] * Fq; hy += CY[q] * Fq;
        }
        m->rho[cell] = r;
        m->ux[cell] = jx / r + hx / (2.0 * r);
        m->uy[cell] = jy / r + hy / (2.0 * r);
    }
}

/* ------------------------------------------------------------------------ */
/* Public API (ctypes)                                                      */
/* ------------------------------------------------------------------------ */

void *oracle_create(int nx, int ny, int wall_x, int wall_y, double tau, double rho_f,
                    double lid_u, double eps, int n_layers, double eta, double gravity,
                    int force_kind, double fa0, double fa1, int rmax) {
    osim_t *m = calloc(1, sizeof(osim_t));
    if (!m) return NULL;
    ocfg_t *c = &m->c;
    c->nx = nx; c->ny = ny; c->wall_x = wall_x; c->wall_y = wall_y;
    c->tau = tau; c->rho_f = rho_f; c->lid_u = lid_u; c->eps = eps;
    c->n_layers = n_layers; c->eta = eta; c->gravity = gravity;
    c->force_kind = force_kind; c->force_a[0] = fa0; c->force_a[1] = fa1;
    c->rmax = rmax;
    long N = (long)nx * ny, NE = (long)(nx + 1) * (ny + 1);
    m->f = calloc(NQ * N, sizeof(double));
    m->fh = calloc(NQ * N, sizeof(double));
    m->Fi = calloc(NQ * N, sizeof(double));
    m->rho = calloc(N, sizeof(double));
    m->ux = calloc(N, sizeof(double));
    m->uy = calloc(N, sizeof(double));
    m->Fx = calloc(N, sizeof(double));
    m->Fy = calloc(N, sizeof(double));
    m->drho = calloc(N, sizeof(double));
    m->Fsx = calloc(N, sizeof(double));
    m->Fsy = calloc(N, sizeof(double));
    m->Fax = calloc(N, sizeof(double));
    m->Fay = calloc(N, sizeof(double));
    m->ex = calloc(EV * NE, sizeof(double));
    m->ey = calloc(EV * NE, sizeof(double));
    m->nl = calloc(N, sizeof(double));
    m->nd = calloc(N, sizeof(double));
    m->na = calloc(2 * N, sizeof(double));
    if (!m->f || !m->fh || !m->Fi || !m->rho || !m->ux || !m->uy || !m->Fx || !m->Fy ||
        !m->drho || !m->ex || !m->ey || !m->nl || !m->nd || !m->na || !m->Fsx || !m->Fsy || !m->Fax ||
        !m->Fay) {
        free(m);
        return NULL;
    }
    m->step = -1; /* not initialised */
    return m;
}

/* Form of the Guo term (Sec. 3.4): 0 multiplies the whole force density by
 * rho, as the expanded Eq. 3_4_Fi prints it; 1 leaves the stress divergence
 * (Eqs. 3_3_div_solid_stress, 3_6_global_stress) without rho, so its net
 * force telescopes to zero in a periodic box. */
int oracle_set_force_mode(void *h, int mode) {
    osim_t *m = h;
    if (mode != 0 && mode != 1) return seterr(m, "force_mode must be 0 or 1");
    m->c.force_mode = mode;
    return 0;
}

int oracle_add_solid(void *h, double xc, double yc, double R, double rho_s, double G) {
    osim_t *m = h;
    if (m->step >= 0) return seterr(m, "solids must be added before the first step");
    if (m->ns == m->cap) {
        int nc = m->cap ? 2 * m->cap : 8;
        osolid_t *ns = realloc(m->s, nc * sizeof(osolid_t));
        if (!ns) return seterr(m, "out of memory");
        m->s = ns; m->cap = nc;
    }
    osolid_t *s = &m->s[m->ns];
    memset(s, 0, sizeof *s);
    s->xc = xc; s->yc = yc; s->R = R; s->rho_s = rho_s; s->G = G;
    s->shape = 0; s->a = R; s->b = R;
    return m->ns++;
}

/* A solid of shape 0 (disk, radius a), 1 (ellipse, semi-axes a, b) or 2
 * (rectangle, half-sides a, b), axis-aligned, centred at (xc, yc). */
int oracle_add_solid_shape(void *h, int shape, double xc, double yc, double a, double b, double rho_s, double G) {
    if (shape < 0 || shape > 2 || !(a > 0) || !(b > 0)) return seterr((osim_t *)h, "bad shape");
    double R = shape == 0 ? a : shape == 1 ? fmax(a, b) : hypot(a, b);
    int id = oracle_add_solid(h, xc, yc, R, rho_s, G);
    if (id < 0) return id;
    osim_t *m = h;
    m->s[id].shape = shape;
    m->s[id].a = shape == 0 ? a : a;
    m->s[id].b = shape == 0 ? a : b;
    return id;
}

/* Algorithm 1, initialisation: xi_0 = x on solid + band, phi = phi_0(xi_0),
 * rho = rho_t, v = 0, f = f^eq,SFC(rho_t, 0), no stored forcing. */
int oracle_init(void *h) {
    osim_t *m = h;
    const ocfg_t *c = &m->c;
    long N = (long)c->nx * c->ny;
    int rc = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : rc)
    for (int si = 0; si < m->ns; si++) rc |= init_solid(m, &m->s[si]) ? 1 : 0;
    if (rc || m->err) return -1;
    compute_force(m); /* gives drho from phi_0; the stress vanishes at xi = x */
    for (long cell = 0; cell < N; cell++) {
        double feq[NQ];
        double rho_t = c->rho_f + m->drho[cell];
        m->rho[cell] = rho_t; m->ux[cell] = 0.0; m->uy[cell] = 0.0;
        oracle_feq(rho_t, 0.0, 0.0, m->drho[cell], feq);
        for (int q = 0; q < NQ; q++) { m->f[q * N + cell] = feq[q]; m->Fi[q * N + cell] = 0.0; }
    }
    m->step = 0;
    return m->err ? -1 : 0;
}

int oracle_step(void *h, int nsteps) {
    osim_t *m = h;
    if (m->step < 0 && oracle_init(h)) return -1;
    for (int n = 0; n < nsteps; n++) {
        int rc = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : rc)
        for (int si = 0; si < m->ns; si++) rc |= update_solid(m, &m->s[si]) ? 1 : 0;
        if (rc || m->err) return -1;
        compute_force(m);
        if (m->err) return -1;
        lb_update(m);
        m->step++;
    }
    return 0;
}

/* Fields: 0 rho, 1 ux, 2 uy, 3 Fx, 4 Fy, 5 drho (last step's force density and
 * density difference), 10 xi_x, 11 xi_y, 12 phi, 13 layer label (per solid,
 * NaN / -1 where the node is not in the solid's band), 20+q population q. */
/* Deformation measures for a Jacobian J = d xi / dx (row-major, J[0] = dX/dx,
 * J[1] = dX/dy, J[2] = dY/dx, J[3] = dY/dy): out[0] = det F - 1 with F = J^-1
 * (volumetric deviation), out[1] = von Mises stress of the neo-Hookean stress
 * tau = G (F F^T - (tr(F F^T) + 1)/3 I) of Eq. 3_3_solid_stress in plane strain,
 * whose out-of-plane component is G (1 - (tr(F F^T) + 1)/3).  Returns -1 if J
 * is singular. */
int oracle_deformation(const double *J, double G, double *out) {
    double det = J[0] * J[3] - J[1] * J[2];
    if (det == 0.0) return -1;
    double F[4] = {J[3] / det, -J[1] / det, -J[2] / det, J[0] / det};
    double Bxx = F[0] * F[0] + F[1] * F[1], Bxy = F[0] * F[2] + F[1] * F[3], Byy = F[2] * F[2] + F[3] * F[3];
    double tr = (Bxx + Byy + 1.0) / 3.0;
    double txx = G * (Bxx - tr), tyy = G * (Byy - tr), tzz = G * (1.0 - tr), txy = G * Bxy;
    out[0] = 1.0 / det - 1.0;
    out[1] = sqrt(1.5 * (txx * txx + tyy * tyy + tzz * tzz + 2.0 * txy * txy));
    return 0;
}

/* Central-difference Jacobian of solid s's reference map at window node (x, y);
 * -1 unless the node is solid (phi < 0) and its four neighbours are in the band. */
static int node_jacobian(const osim_t *m, const osolid_t *s, int x, int y, double *J) {
    const ocfg_t *c = &m->c;
    if (x < 1 || y < 1 || x >= s->w - 1 || y >= s->h - 1) return -1;
    int k = y * s->w + x;
    if (s->lab[k] < 0 || !(s->phi[k] < -PHI_TIE) || !in_domain(c, s->x0 + x, s->y0 + y)) return -1;
    if (s->lab[k - 1] < 0 || s->lab[k + 1] < 0 || s->lab[k - s->w] < 0 || s->lab[k + s->w] < 0) return -1;
    J[0] = 0.5 * (s->X[k + 1] - s->X[k - 1]);
    J[1] = 0.5 * (s->X[k + s->w] - s->X[k - s->w]);
    J[2] = 0.5 * (s->Y[k + 1] - s->Y[k - 1]);
    J[3] = 0.5 * (s->Y[k + s->w] - s->Y[k - s->w]);
    return 0;
}

int oracle_read_field(void *h, int field, int solid, double *out) {
    osim_t *m = h;
    const ocfg_t *c = &m->c;
    long N = (long)c->nx * c->ny;
    if (m->step < 0 && oracle_init(h)) return -1;
    const double *src = NULL;
    switch (field) {
    case 0: src = m->rho; break;
    case 1: src = m->ux; break;
    case 2: src = m->uy; break;
    case 3: src = m->Fx; break;
    case 4: src = m->Fy; break;
    case 5: src = m->drho; break;
    default: break;
    }
    if (src) { memcpy(out, src, N * sizeof(double)); return 0; }
    if (field >= 20 && field < 20 + NQ) { memcpy(out, m->f + (field - 20) * N, N * sizeof(double)); return 0; }
    if (field == 14 || field == 15) {
        if (solid < 0 || solid >= m->ns) return seterr(m, "bad solid id");
        const osolid_t *s = &m->s[solid];
        for (long k = 0; k < N; k++) out[k] = NAN;
        for (int y = 0; y < s->h; y++)
            for (int x = 0; x < s->w; x++) {
                double J[4], d[2];
                if (node_jacobian(m, s, x, y, J) || oracle_deformation(J, s->G, d)) continue;
                long cell = (long)wrapi(s->y0 + y, c->ny) * c->nx + wrapi(s->x0 + x, c->nx);
                out[cell] = field == 14 ? d[0] : d[1];
            }
        return 0;
    }
    if (field >= 10 && field <= 13) {
        if (solid < 0 || solid >= m->ns) return seterr(m, "bad solid id");
        const osolid_t *s = &m->s[solid];
        for (long k = 0; k < N; k++) out[k] = field == 13 ? -1.0 : NAN;
        for (int y = 0; y < s->h; y++)
            for (int x = 0; x < s->w; x++) {
                int k = y * s->w + x, gx = s->x0 + x, gy = s->y0 + y;
                if (s->lab[k] < 0 || !in_domain(c, gx, gy)) continue;
                long cell = (long)wrapi(gy, c->ny) * c->nx + wrapi(gx, c->nx);
                out[cell] = field == 10 ? s->X[k] : field == 11 ? s->Y[k] : field == 12 ? s->phi[k] : (double)s->lab[k];
            }
        return 0;
    }
    return seterr(m, "bad field id");
}

/* Per-solid statistics at the current time: lambda = 1 - H(phi) over domain
 * nodes; out[0..7] = sum lambda, centroid x, centroid y (unwrapped frame),
 * sum lambda rho, sum lambda rho u, sum lambda rho v, and over the solid nodes
 * (phi < 0) the maximum and the lambda-weighted mean of |det F - 1|. */
/* Net contact force on solid s (a reading: the paper defines the contact
 * stress, Sec. 3.6, but no per-solid force): for every other solid t, the
 * divergence (Eq. 3_3_div_solid_stress) of the pair's contact stress at each
 * domain node, counted for s where the node is nearer to s than to t
 * (phi_s < phi_t; half each where equal; a node outside t's band is nearer to
 * s).  Summed over the pairs.  The divergence of one pair's stress sums to
 * zero over a periodic box, so the forces on s and t from their contact are
 * equal and opposite. */
static void oracle_contact_force(const osim_t *m, int solid, double *out) {
    const ocfg_t *c = &m->c;
    const osolid_t *s = &m->s[solid];
    out[0] = out[1] = 0.0;
    for (int ti = 0; ti < m->ns; ti++) {
        if (ti == solid) continue;
        const osolid_t *t = &m->s[ti];
        if (!windows_meet(c, s, t)) continue;
        for (int y = 0; y < s->h; y++)
            for (int x = 0; x < s->w; x++) {
                int k = y * s->w + x, gx = s->x0 + x, gy = s->y0 + y;
                if (s->lab[k] < 0 || !in_domain(c, gx, gy)) continue;
                int tx, ty;
                int kt = lookup(c, t, c->wall_x ? gx : wrapi(gx, c->nx), c->wall_y ? gy : wrapi(gy, c->ny), &tx, &ty);
                double pt = (kt >= 0 && t->lab[kt] >= 0) ? t->phi[kt] : INFINITY;
                double w = s->phi[k] < pt ? 1.0 : (s->phi[k] == pt ? 0.5 : 0.0);
                if (w == 0.0) continue;
                double tl[3] = {0, 0, 0}, tr[3] = {0, 0, 0}, tb[3] = {0, 0, 0}, tt[3] = {0, 0, 0};
                int any = pair_edge_stress(m, s, t, 0, gx, gy, tl);
                any |= pair_edge_stress(m, s, t, 0, gx + 1, gy, tr);
                any |= pair_edge_stress(m, s, t, 1, gx, gy, tb);
                any |= pair_edge_stress(m, s, t, 1, gx, gy + 1, tt);
                if (!any) continue;
                out[0] += w * ((tr[0] - tl[0]) + (tt[1] - tb[1]));
                out[1] += w * ((tr[1] - tl[1]) + (tt[2] - tb[2]));
            }
    }
}

int oracle_solid_stats(void *h, int solid, double *out) {
    osim_t *m = h;
    const ocfg_t *c = &m->c;
    if (m->step < 0 && oracle_init(h)) return -1;
    if (solid < 0 || solid >= m->ns) return seterr(m, "bad solid id");
    const osolid_t *s = &m->s[solid];
    double L = 0, Lx = 0, Ly = 0, Lr = 0, Lu = 0, Lv = 0, Dmax = 0, Dsum = 0, Dw = 0;
    for (int y = 0; y < s->h; y++)
        for (int x = 0; x < s->w; x++) {
            int k = y * s->w + x, gx = s->x0 + x, gy = s->y0 + y;
            if (s->lab[k] < 0 || !in_domain(c, gx, gy)) continue;
            if (!(s->phi[k] < c->eps)) continue;
            long cell = (long)wrapi(gy, c->ny) * c->nx + wrapi(gx, c->nx);
            double lam = 1.0 - oracle_heaviside(s->phi[k], c->eps);
            L += lam; Lx += lam * gx; Ly += lam * gy;
            Lr += lam * m->rho[cell];
            Lu += lam * m->rho[cell] * m->ux[cell];
            Lv += lam * m->rho[cell] * m->uy[cell];
            double J[4], d[2];
            if (node_jacobian(m, s, x, y, J) == 0 && oracle_deformation(J, s->G, d) == 0) {
                double a = fabs(d[0]);
                if (a > Dmax) Dmax = a;
                Dsum += lam * a;
                Dw += lam;
            }
        }
    out[0] = L; out[1] = Lx / L; out[2] = Ly / L; out[3] = Lr; out[4] = Lu; out[5] = Lv;
    out[6] = Dmax; out[7] = Dw > 0 ? Dsum / Dw : 0.0;
    oracle_contact_force(m, solid, out + 8);
    return 0;
}

/* Overwrite the populations (9 planes of nx*ny) and recompute the moments with
 * no stored forcing; used by tests that start from a prescribed state. */
int oracle_set_populations(void *h, const double *f) {
    osim_t *m = h;
    const ocfg_t *c = &m->c;
    long N = (long)c->nx * c->ny;
    if (m->step < 0 && oracle_init(h)) return -1;
    memcpy(m->f, f, NQ * N * sizeof(double));
    for (long cell = 0; cell < N; cell++) {
        double r = 0, jx = 0, jy = 0;
        for (int q = 0; q < NQ; q++) {
            double fq = f[q * N + cell];
            r += fq; jx += CX[q] * fq; jy += CY[q] * fq;
            m->Fi[q * N + cell] = 0.0;
        }
        m->rho[cell] = r; m->ux[cell] = jx / r; m->uy[cell] = jy / r;
    }
    return 0;
}

long oracle_steps_done(void *h) { return ((osim_t *)h)->step; }
/* Overwrite a solid's reference map on its solid and band nodes with the
 * values of the grids X, Y (nx*ny doubles each, absolute reference
 * coordinates of the grid nodes), then relabel phi = phi_0(xi) there (Sec.
 * 3.2).  The labels (solid set and layers) are kept.  A node of the unwrapped
 * window at gx takes X[i] + (gx - i) for its grid node i, so the map stays
 * continuous across a periodic edge.  For tests that prescribe a deformation. */
int oracle_set_refmap(void *h, int solid, const double *X, const double *Y) {
    osim_t *m = h;
    if (m->step < 0) return seterr(m, "the simulation is not initialised");
    if (solid < 0 || solid >= m->ns) return seterr(m, "no such solid");
    const ocfg_t *c = &m->c;
    osolid_t *s = &m->s[solid];
    for (int y = 0; y < s->h; y++)
        for (int x = 0; x < s->w; x++) {
            int k = y * s->w + x, gx = s->x0 + x, gy = s->y0 + y;
            if (s->lab[k] < 0) continue;
            int i = wrapi(gx, c->nx), j = wrapi(gy, c->ny);
            long cell = (long)j * c->nx + i;
            s->X[k] = X[cell] + (gx - i);
            s->Y[k] = Y[cell] + (gy - j);
            s->phi[k] = phi0(s, s->X[k], s->Y[k]);
        }
    return 0;
}

int oracle_num_solids(void *h) { return ((osim_t *)h)->ns; }
const char *oracle_error(void *h) { return ((osim_t *)h)->err ? ((osim_t *)h)->msg : ""; }

void oracle_destroy(void *h) {
    osim_t *m = h;
    if (!m) return;
    for (int si = 0; si < m->ns; si++) free_window(&m->s[si]);
    free(m->s);
    free(m->f); free(m->fh); free(m->Fi); free(m->rho); free(m->ux); free(m->uy);
    free(m->Fx); free(m->Fy); free(m->drho); free(m->ex); free(m->ey);
    free(m->Fsx); free(m->Fsy); free(m->Fax); free(m->Fay);
    free(m->nl); free(m->nd); free(m->na);
    free(m->c.bfield);
    free(m);
}

/* force_kind 3: copy the body force field (2*nx*ny doubles, x plane then y plane). */
int oracle_set_body_force(void *h, const double *bxy) {
    osim_t *m = h;
    long n = 2L * m->c.nx * m->c.ny;
    if (m->c.force_kind != 3) return seterr(m, "force_kind is not 3 (field)");
    if (!m->c.bfield) m->c.bfield = malloc(n * sizeof(double));
    if (!m->c.bfield) return seterr(m, "out of memory");
    memcpy(m->c.bfield, bxy, n * sizeof(double));
    return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
