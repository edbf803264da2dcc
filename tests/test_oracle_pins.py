"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
printed tables and expanded formulas (tests/golden/), conservation laws the
paper derives (Appendix C), closed-form flows (Couette, Poiseuille), exact
properties of the discretisations (upwind stencil and least-squares fit are
exact on linear fields, F = I gives zero stress) and brute force with an
independent least-squares routine.
"""
import math
import os

import numpy as np
import pytest

import oracle
import scenarios

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _table(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return np.array(rows)


D2Q9 = _table("d2q9_table.txt")
CX = D2Q9[:, 1]
CY = D2Q9[:, 2]
W = D2Q9[:, 3] / D2Q9[:, 4]


# --------------------------------------------------------------------------
# Equilibrium with smooth flux correction (Eqs. 2_3_feq_sfc, 3_4_feq; App. C)
# --------------------------------------------------------------------------

def test_d2q9_table_consistency():
    # Table d2q9: weights sum to one, isotropy gives c_s^2 = 1/3 (Sec. 2.2)
    assert abs(W.sum() - 1.0) < 1e-15
    assert abs((W * CX * CX).sum() - 1.0 / 3.0) < 1e-15
    assert abs((W * CX * CY).sum()) < 1e-15


@pytest.mark.parametrize("seed", range(5))
def test_feq_moments_and_sfc_conservation(seed):
    rng = np.random.default_rng(seed)
    for _ in range(50):
        rho = rng.uniform(0.5, 2.0)
        u, v = rng.uniform(-0.1, 0.1, 2)
        drho = rng.uniform(-0.5, 1.0)
        f = oracle.feq(rho, u, v, drho)
        # Appendix C: the SFC terms cancel in mass and momentum
        assert abs(f.sum() - rho) < 1e-14
        assert abs((CX * f).sum() - rho * u) < 1e-15
        assert abs((CY * f).sum() - rho * v) < 1e-15
        # second moment of the uncorrected part: sum c c f = rho (cs2 I + v v)
        f0 = oracle.feq(rho, u, v, 0.0)
        assert abs((CX * CX * f0).sum() - rho * (1 / 3 + u * u)) < 1e-14
        assert abs((CX * CY * f0).sum() - rho * u * v) < 1e-14


def test_feq_matches_expanded_eq_3_4_feq():
    T = _table("feq_expanded.txt")
    rng = np.random.default_rng(7)
    for _ in range(100):
        rho = rng.uniform(0.5, 2.0)
        u, v = rng.uniform(-0.2, 0.2, 2)
        drho = rng.uniform(-0.5, 1.0)
        f = oracle.feq(rho, u, v, drho)
        for row in T:
            i, den, a0, au, av, auu, avv, auv, kn, kd = row
            e = rho * (a0 + au * u + av * v + auu * u * u + avv * v * v + auv * u * v) / den + kn / kd * drho
            assert abs(f[int(i)] - e) < 1e-15


# --------------------------------------------------------------------------
# Guo forcing (Eqs. 2_2_Fi, 3_4_Fi)
# --------------------------------------------------------------------------

def test_guo_moments_and_expanded_form():
    T = _table("guo_expanded.txt")
    rng = np.random.default_rng(3)
    for _ in range(100):
        rho = rng.uniform(0.5, 2.0)
        u, v = rng.uniform(-0.2, 0.2, 2)
        fx, fy = rng.uniform(-1e-3, 1e-3, 2)
        F = oracle.guo(rho, u, v, fx, fy)
        assert abs(F.sum()) < 1e-18
        assert abs((CX * F).sum() - rho * fx) < 1e-18
        assert abs((CY * F).sum() - rho * fy) < 1e-18
        # second moments of the Guo term: rho (v F + F v)
        assert abs((CX * CX * F).sum() - 2 * rho * u * fx) < 1e-18
        assert abs((CX * CY * F).sum() - rho * (u * fy + v * fx)) < 1e-18
        assert abs((CY * CY * F).sum() - 2 * rho * v * fy) < 1e-18
        for row in T:
            i, den, bx, by, bux, bvx, buy, bvy = row
            e = rho / den * (bx * fx + by * fy + bux * u * fx + bvx * v * fx + buy * u * fy + bvy * v * fy)
            assert abs(F[int(i)] - e) < 1e-18


def test_printed_F2_term_would_break_momentum():
    # As printed, F_2 and F_4 of Eq. 3_4_Fi carry 9 v F_x; that version breaks
    # the second moment sum c_y c_y F_i = 2 rho v F_y that Eq. 2_2_Fi gives,
    # which is why the oracle reads 9 v F_y.
    rho, u, v, fx, fy = 1.1, 0.03, -0.02, 1e-3, 2e-3
    F = oracle.guo(rho, u, v, fx, fy).copy()
    F_print = F.copy()
    F_print[2] = rho / 9 * (-3 * u * fx + 3 * (1 - v) * fy + 9 * v * fx)
    F_print[4] = rho / 9 * (-3 * u * fx + 3 * (-1 - v) * fy + 9 * v * fx)
    assert abs((CY * CY * F).sum() - 2 * rho * v * fy) < 1e-18
    assert abs((CY * CY * F_print).sum() - 2 * rho * v * fy) > 1e-6


# --------------------------------------------------------------------------
# Heaviside (Eq. 2_3_heaviside)
# --------------------------------------------------------------------------

def test_heaviside_properties():
    eps = 1.5
    H = oracle.heaviside
    assert H(0.0, eps) == 0.5
    assert H(-eps, eps) == 0.0 and H(eps, eps) == 1.0
    xs = np.linspace(-2 * eps, 2 * eps, 401)
    vals = np.array([H(x, eps) for x in xs])
    assert np.all(np.diff(vals) >= -1e-16)
    assert vals.min() >= 0 and vals.max() <= 1
    for x in xs:
        assert abs(H(x, eps) + H(-x, eps) - 1.0) < 1e-15
    # continuity at the blur-zone edges
    d = 1e-9
    assert abs(H(eps - d, eps) - 1.0) < 1e-12
    assert abs(H(-eps + d, eps)) < 1e-12


# --------------------------------------------------------------------------
# Solid stress (Eqs. 3_3_refmap_deformation, 3_3_solid_stress) and contact
# --------------------------------------------------------------------------

def test_stress_zero_for_identity_and_rotation():
    G = 0.37
    assert np.all(oracle.stress_from_jacobian([[1, 0], [0, 1]], G) == 0.0)
    for th in np.linspace(-3, 3, 13):
        R = [[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]]
        assert np.abs(oracle.stress_from_jacobian(R, G)).max() < 1e-15


@pytest.mark.parametrize("a", [0.5, 0.9, 1.3, 2.0])
def test_stress_uniaxial_stretch_closed_form(a):
    G = 0.1
    # J = d xi/dx = F^{-1} for F = diag(a, 1/a)
    tau = oracle.stress_from_jacobian([[1 / a, 0], [0, a]], G)
    tr = (a * a + 1 / (a * a) + 1) / 3
    assert np.allclose(tau, [G * (a * a - tr), 0.0, G * (1 / (a * a) - tr)], rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("gam", [-0.4, 0.05, 0.3])
def test_stress_simple_shear_closed_form(gam):
    G = 0.02
    # F = [[1, gam], [0, 1]] => J = [[1, -gam], [0, 1]]; B = F F^T
    tau = oracle.stress_from_jacobian([[1, -gam], [0, 1]], G)
    assert np.allclose(tau, [2 / 3 * G * gam * gam, G * gam, -G * gam * gam / 3], rtol=1e-13, atol=1e-18)


def test_contact_stress_properties():
    eps, eta = 1.5, 1.0
    rng = np.random.default_rng(1)
    for _ in range(50):
        ps, pt = rng.uniform(-1.4, 1.4, 2)
        gx, gy = rng.normal(size=2)
        t = oracle.contact_stress(ps, pt, 0.01, 0.02, eta, eps, gx, gy)
        assert abs(t[0] + t[2]) < 1e-17          # traceless
        t2 = oracle.contact_stress(pt, ps, 0.02, 0.01, eta, eps, -gx, -gy)
        assert np.allclose(t, t2, rtol=0, atol=1e-18)  # swap invariance
        # repulsive: normal stress along n is -k/2 < 0 times (-1) ... sign check
        n = np.array([gx, gy]) / math.hypot(gx, gy)
        tn = t[0] * n[0] ** 2 + 2 * t[1] * n[0] * n[1] + t[2] * n[1] ** 2
        fm = min(0.5 * (1 - ps / eps), 0.5 * (1 - pt / eps))
        assert abs(tn - (-eta * fm * 0.03 * 0.5)) < 1e-15
    assert np.all(oracle.contact_stress(1.5, -1.0, 0.01, 0.01, eta, eps, 1, 0) == 0)
    assert np.all(oracle.contact_stress(-1.0, 2.0, 0.01, 0.01, eta, eps, 1, 0) == 0)


def test_contact_pair_window_test_matches_brute_force():
    # The contact sum (Sec. 3.6) passes over solid pairs whose windows share no
    # grid node.  The window test against explicit node sets (periodic images
    # folded into the grid) on random windows of small periodic and walled
    # grids; windows start within one window width of the domain, as a
    # solid's window does (its centre lies in the domain).
    rng = np.random.default_rng(5)
    met = 0
    for _ in range(600):
        nx, ny = int(rng.integers(6, 24)), int(rng.integers(6, 24))
        wall_x, wall_y = bool(rng.integers(2)), bool(rng.integers(2))

        def window():
            w, h = int(rng.integers(1, nx)), int(rng.integers(1, ny))
            return (int(rng.integers(-w + 1, nx)), int(rng.integers(-h + 1, ny)), w, h)

        def nodes(win):
            x0, y0, w, h = win
            xs = [x if wall_x else x % nx for x in range(x0, x0 + w)]
            ys = [y if wall_y else y % ny for y in range(y0, y0 + h)]
            return {(x, y) for x in xs for y in ys}

        a, b = window(), window()
        expect = bool(nodes(a) & nodes(b))
        met += expect
        assert oracle.windows_meet(a, b, nx, ny, wall_x, wall_y) == expect, (a, b, nx, ny, wall_x, wall_y)
    assert 100 < met < 500  # both outcomes exercised


# --------------------------------------------------------------------------
# Extrapolation (Sec. 3.2, Eq. 3_2_extrap_weight)
# --------------------------------------------------------------------------

def _lsq_reference(lab, X, tx, ty, layer, r, normal):
    """Independent weighted least squares with numpy.linalg.lstsq."""
    h, w = lab.shape
    rows, rhs = [], []
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            x, y = tx + dx, ty + dy
            if not (0 <= x < w and 0 <= y < h):
                continue
            if not (0 <= lab[y, x] < layer):
                continue
            wt = 2.0 ** -(abs(dx) + abs(dy))
            if layer <= 2 and normal is not None:
                d = np.array([-dx, -dy], float)
                cos = d @ np.asarray(normal) / np.linalg.norm(d)
                wt = cos * wt if cos > 1e-9 else 0.0
            if wt <= 0:
                continue
            s = math.sqrt(wt)
            rows.append([s * dx, s * dy, s])
            rhs.append(s * X[y, x])
    p = np.linalg.lstsq(np.array(rows), np.array(rhs), rcond=None)[0]
    return p[2]


def _random_region(rng, h=13, w=13):
    lab = -np.ones((h, w), np.int8)
    cx, cy, R = rng.uniform(4, 8), rng.uniform(4, 8), rng.uniform(2.5, 4)
    yy, xx = np.mgrid[0:h, 0:w]
    lab[(xx - cx) ** 2 + (yy - cy) ** 2 < R * R] = 0
    # two dilation layers
    for l in (1, 2, 3):
        prev = lab == l - 1
        nb = np.zeros_like(prev)
        nb[1:] |= prev[:-1]; nb[:-1] |= prev[1:]; nb[:, 1:] |= prev[:, :-1]; nb[:, :-1] |= prev[:, 1:]
        lab[(lab == -1) & nb] = l
    return lab, (cx, cy)


@pytest.mark.parametrize("seed", range(6))
def test_extrapolation_exact_on_linear_fields(seed):
    rng = np.random.default_rng(seed)
    lab, (cx, cy) = _random_region(rng)
    A = rng.normal(size=(2, 2)); b = rng.normal(size=2) * 10
    yy, xx = np.mgrid[0:lab.shape[0], 0:lab.shape[1]].astype(float)
    X = A[0, 0] * xx + A[0, 1] * yy + b[0]
    Y = A[1, 0] * xx + A[1, 1] * yy + b[1]
    for ty, tx in zip(*np.nonzero(lab > 0)):
        l = int(lab[ty, tx])
        n = np.array([tx - cx, ty - cy]); n /= np.linalg.norm(n)
        r, ox, oy = oracle.extrap_target(lab, X, Y, tx, ty, l, normal=n)
        assert r >= 2
        assert abs(ox - X[ty, tx]) < 1e-12 and abs(oy - Y[ty, tx]) < 1e-12


@pytest.mark.parametrize("seed", range(6))
def test_extrapolation_matches_independent_lstsq(seed):
    rng = np.random.default_rng(100 + seed)
    lab, (cx, cy) = _random_region(rng)
    X = rng.normal(size=lab.shape)
    Y = rng.normal(size=lab.shape)
    for ty, tx in zip(*np.nonzero(lab > 0)):
        l = int(lab[ty, tx])
        n = np.array([tx - cx, ty - cy]); n /= np.linalg.norm(n)
        r, ox, oy = oracle.extrap_target(lab, X, Y, tx, ty, l, normal=n)
        assert abs(ox - _lsq_reference(lab, X, tx, ty, l, r, n)) < 1e-11
        assert abs(oy - _lsq_reference(lab, Y, tx, ty, l, r, n)) < 1e-11


def test_extrapolation_window_growth():
    # fewer than three valid nodes within r = 2 -> r grows to 3
    lab = -np.ones((9, 9), np.int8)
    lab[4, 0] = 0; lab[4, 1] = 0; lab[0, 0] = 0
    lab[4, 4] = 1
    X = np.arange(81, dtype=float).reshape(9, 9)
    r, ox, _ = oracle.extrap_target(lab, X, X, 4, 4, 3)
    assert r == 4  # (0,0) is at Chebyshev distance 4
    assert abs(ox - X[4, 4]) < 1e-12
    # three collinear valid nodes: ill-posed fit, the window must grow
    lab = -np.ones((9, 9), np.int8)
    lab[4, 1] = lab[4, 2] = lab[4, 3] = 0
    lab[1, 1] = 0
    lab[4, 5] = 1
    r, ox, _ = oracle.extrap_target(lab, X, X, 5, 4, 3)
    assert r == 4 and abs(ox - X[4, 5]) < 1e-12
    # the directional weight of layers 1-2 keeps only nodes behind the target
    lab = -np.ones((9, 9), np.int8)
    lab[3, 2] = lab[5, 2] = lab[4, 3] = 0   # behind the target (x < 4)
    lab[3, 6] = lab[4, 6] = lab[5, 6] = 0   # ahead of the target
    lab[0, 4] = 0                           # below, at Chebyshev distance 4
    lab[4, 4] = 1
    r, ox, _ = oracle.extrap_target(lab, X, X, 4, 4, 1, normal=(1.0, 0.0))
    assert r == 2 and abs(ox - X[4, 4]) < 1e-12
    # normal along +y: only (2,3), (6,3) have positive weight within r = 2, so
    # the window grows until (4,0) joins at r = 4
    r2, ox2, _ = oracle.extrap_target(lab, X, X, 4, 4, 1, normal=(0.0, 1.0))
    assert r2 == 4 and abs(ox2 - X[4, 4]) < 1e-12


# --------------------------------------------------------------------------
# Whole-step invariants
# --------------------------------------------------------------------------

def _total(o):
    return o.field("rho").sum()


def test_rest_is_a_fixed_point():
    sc = scenarios.settling_small(seed=1, gravity=0.0)
    o = oracle.Oracle(sc)
    f0 = o.populations()
    o.step(30)
    assert np.abs(o.populations() - f0).max() < 1e-12  # round-off over 30 steps
    assert np.abs(o.field("ux")).max() < 1e-13 and np.abs(o.field("uy")).max() < 1e-13
    x = np.arange(sc["nx"])[None, :].repeat(sc["ny"], 0)
    for s in range(len(sc["solids"])):
        xi = o.field("xi_x", s)
        m = np.isfinite(xi)
        d = (xi[m] - x[m] + sc["nx"] / 2) % sc["nx"] - sc["nx"] / 2  # unwrapped frame
        assert np.abs(d).max() < 1e-10


@pytest.mark.parametrize("seed", range(3))
def test_mass_conserved_periodic_with_forcing(seed):
    sc = scenarios.mixing_small(seed=seed)
    o = oracle.Oracle(sc)
    m0 = _total(o)
    o.step(40)
    assert abs(_total(o) - m0) < 1e-11 * m0


def test_momentum_gain_per_step():
    # Periodic box.  The collision (Eq. 2_2_bgk_force) changes sum c_i f_i by
    # (1/tau)(rho v - sum c f) + (1 - 1/(2 tau)) rho^n F^n (sum c F_i = rho F,
    # Eq. 2_2_Fi); in Algorithm 1 the velocity v^n of f^eq carries the half-force
    # of the previous step, rho v^n = sum c f + rho^{n-1} F^{n-1} / 2.  So the
    # gain is exactly sum[rho^{n-1} F^{n-1} / (2 tau) + (1 - 1/(2 tau)) rho^n F^n].
    sc = scenarios.mixing_small(seed=2)
    tau = sc["tau"]
    o = oracle.Oracle(sc)
    o.step(4)
    rho_prev = o.populations().sum(0)
    o.step(1)
    prev = (rho_prev * o.field("Fx"), rho_prev * o.field("Fy"))
    for _ in range(3):
        f = o.populations()
        rho = f.sum(0)
        px = (CX[:, None, None] * f).sum()
        py = (CY[:, None, None] * f).sum()
        o.step(1)
        f1 = o.populations()
        cur = (rho * o.field("Fx"), rho * o.field("Fy"))
        gx = (prev[0] / (2 * tau) + (1 - 1 / (2 * tau)) * cur[0]).sum()
        gy = (prev[1] / (2 * tau) + (1 - 1 / (2 * tau)) * cur[1]).sum()
        assert abs(gx) > 1e-6
        assert abs((CX[:, None, None] * f1).sum() - px - gx) < 1e-11
        assert abs((CY[:, None, None] * f1).sum() - py - gy) < 1e-11
        prev = cur


def test_rigid_translation_keeps_xi_exact():
    # neutrally buoyant disk in uniform flow: upwind advection and the LSQ fit are
    # exact on linear xi, so xi = x - n U on the whole band; stress stays zero
    sc = scenarios.fluid_only(64, 48, 0, 0, 0.7)
    sc["solids"].append({"x": 30.3, "y": 23.6, "r": 9.0, "rho_s": 1.0, "G": 0.05})
    o = oracle.Oracle(sc)
    U, V = 0.02, -0.013
    f = np.zeros((9, 48, 64))
    feq = oracle.feq(1.0, U, V, 0.0)
    f[:] = feq[:, None, None]
    o.set_populations(f)
    n = 6
    o.step(n)
    x = np.arange(64)[None, :].repeat(48, 0).astype(float)
    y = np.arange(48)[:, None].repeat(64, 1).astype(float)
    xi, yi = o.field("xi_x"), o.field("xi_y")
    m = np.isfinite(xi)
    assert m.sum() > 500
    assert np.abs(xi[m] - (x[m] - n * U)).max() < 1e-10
    assert np.abs(yi[m] - (y[m] - n * V)).max() < 1e-10
    assert np.abs(o.field("Fx")).max() < 1e-12 and np.abs(o.field("Fy")).max() < 1e-12


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0])
def test_couette_exact_linear_profile(tau):
    ny, U = 8, 0.01
    o = oracle.Oracle(scenarios.fluid_only(4, ny, 0, 1, tau, lid_u=U))
    o.step(5000)
    u = o.field("ux")[:, 0]
    assert np.abs(u - U * (np.arange(ny) + 0.5) / ny).max() < 1e-13
    assert np.abs(o.field("uy")).max() < 1e-13


@pytest.mark.parametrize("tau", [0.6, 1.0])
def test_poiseuille_parabola(tau):
    g = 1e-6
    nu = (tau - 0.5) / 3
    slips = []
    for ny in (8, 16):
        o = oracle.Oracle(scenarios.fluid_only(4, ny, 0, 1, tau, force_kind=1, force_a=(g, 0.0)))
        o.step(int(12 * ny * ny / nu))
        u = o.field("ux")[:, 0]
        d2 = u[2:] - 2 * u[1:-1] + u[:-2]
        assert np.abs(d2 * nu / g + 1.0).max() < 1e-8        # curvature exactly -g/nu
        y = np.arange(ny) + 0.5
        ex = g / (2 * nu) * y * (ny - y)
        dev = u - ex
        assert np.ptp(dev) < 1e-8 * ex.max()                  # uniform wall slip
        slips.append(abs(dev.mean()) / ex.max())
    assert slips[1] < slips[0] / 3.5                          # slip error is O(1/H^2)


def test_mirror_symmetry_settling_disk():
    nx, ny = 48, 64
    sc = scenarios.fluid_only(nx, ny, 0, 1, 0.7)
    sc["gravity"] = 5e-4
    # centre on the mirror line x = (nx - 1)/2 of the node lattice
    sc["solids"].append({"x": (nx - 1) / 2, "y": 30.4, "r": 8.5, "rho_s": 1.6, "G": 0.02})
    o = oracle.Oracle(sc)
    o.step(60)
    u, v = o.field("ux"), o.field("uy")
    assert np.abs(v).max() > 1e-4
    assert np.abs(u + u[:, ::-1]).max() < 1e-10 * np.abs(v).max()
    assert np.abs(v - v[:, ::-1]).max() < 1e-10 * np.abs(v).max()
    xi = o.field("xi_x")
    m = np.isfinite(xi)
    assert np.array_equal(m, m[:, ::-1])
    assert np.abs((xi - (nx - 1) / 2) + (xi[:, ::-1] - (nx - 1) / 2))[m].max() < 1e-10


def test_band_has_eleven_layers_and_pads():
    sc = scenarios.ldc_disk_64()
    o = oracle.Oracle(sc)
    lab = o.field("label")
    assert lab.max() == 11
    phi = o.field("phi")
    assert np.all(phi[lab == 0] < 0)
    o.step(3)
    lab = o.field("label")
    assert set(np.unique(lab[lab >= 0]).astype(int)) == set(range(12))


def test_body_force_field_uniform_equals_constant_force():
    # A per-node body force field (force_kind 3) that is uniform must give
    # exactly the pinned constant-force path (force_kind 1): the field only
    # replaces where f of Eq. 2_4_F_divs is read from.
    sc1 = scenarios.mixing_small(seed=3)
    sc1["force_kind"], sc1["force_a"] = 1, [2e-5, -1e-5]
    sc3 = dict(sc1)
    sc3["force_kind"] = 3
    n = sc1["nx"] * sc1["ny"]
    sc3["body_field"] = np.concatenate([np.full(n, 2e-5), np.full(n, -1e-5)])
    a, b = oracle.Oracle(sc1), oracle.Oracle(sc3)
    a.step(15)
    b.step(15)
    for name in ("rho", "ux", "uy", "Fx", "Fy"):
        assert np.array_equal(a.field(name), b.field(name)), name
    assert np.array_equal(a.field("xi_x", 1), b.field("xi_x", 1), equal_nan=True)


def test_body_force_field_momentum_gain():
    # Momentum gain per step with a non-uniform field (periodic box): the
    # identity of test_momentum_gain_per_step with F including the field.
    sc = scenarios.fluid_only(48, 40, 0, 0, 0.7)
    sc["force_kind"] = 3
    sc["body_field"] = scenarios.smooth_body_field(5, 48, amp=3e-5)[:, :40, :]
    tau = sc["tau"]
    o = oracle.Oracle(sc)
    o.step(2)
    rho_prev = o.populations().sum(0)
    o.step(1)
    prev = (rho_prev * o.field("Fx"), rho_prev * o.field("Fy"))
    f = o.populations()
    rho = f.sum(0)
    px, py = (CX[:, None, None] * f).sum(), (CY[:, None, None] * f).sum()
    o.step(1)
    f1 = o.populations()
    # no solid: F is the field itself
    assert np.array_equal(o.field("Fx"), sc["body_field"][0])
    cur = (rho * o.field("Fx"), rho * o.field("Fy"))
    gx = (prev[0] / (2 * tau) + (1 - 1 / (2 * tau)) * cur[0]).sum()
    gy = (prev[1] / (2 * tau) + (1 - 1 / (2 * tau)) * cur[1]).sum()
    assert abs((CX[:, None, None] * f1).sum() - px - gx) < 1e-11
    assert abs((CY[:, None, None] * f1).sum() - py - gy) < 1e-11


def test_deformation_closed_forms():
    # det F - 1 and the von Mises stress of tau = G (F F^T - (tr(F F^T) + 1)/3 I)
    # in plane strain (tau_zz = G (1 - (tr + 1)/3)), for Jacobians J = d xi/dx
    G = 0.7
    assert oracle.deformation(np.eye(2), G) == (0.0, 0.0)
    for th in (0.3, -1.1, 2.5):  # rigid rotation: F = R^T, F F^T = I
        J = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        d, vm = oracle.deformation(J, G)
        assert abs(d) < 1e-15 and vm < 1e-15
    for a in (0.8, 1.25, 2.0):  # F = diag(a, 1/a): isochoric stretch
        J = np.diag([1 / a, a])
        d, vm = oracle.deformation(J, G)
        tr = (a * a + 1 / (a * a) + 1) / 3
        t = np.array([a * a - tr, 1 / (a * a) - tr, 1 - tr]) * G
        assert abs(d) < 1e-15
        assert abs(vm - np.sqrt(1.5 * (t ** 2).sum())) < 1e-14
    for s in (0.9, 1.1):  # pure dilation: F = s I, deviatoric stress from the z direction only
        d, vm = oracle.deformation(np.eye(2) / s, G)
        assert abs(d - (s * s - 1)) < 1e-14
        tr = (2 * s * s + 1) / 3
        t = np.array([s * s - tr, s * s - tr, 1 - tr]) * G
        assert abs(vm - np.sqrt(1.5 * (t ** 2).sum())) < 1e-14
    g = 0.4  # simple shear F = [[1, g], [0, 1]]: B = [[1 + g^2, g], [g, 1]],
    # tau = G (2g^2/3, -g^2/3, -g^2/3; g), von Mises = G g sqrt(g^2 + 3)
    J = np.linalg.inv(np.array([[1.0, g], [0.0, 1.0]]))
    d, vm = oracle.deformation(J, G)
    assert abs(d) < 1e-15
    assert abs(vm - G * g * np.sqrt(g * g + 3)) < 1e-14


def test_initial_solid_is_undeformed():
    # xi = x at initialisation: J = I on every solid node, det F = 1, no stress
    sc = scenarios.settling_small(0)
    o = oracle.Oracle(sc)
    for s in range(len(sc["solids"])):
        d, vm = o.field("detF_dev", s), o.field("von_mises", s)
        m = np.isfinite(d)
        assert m.sum() > 100
        assert np.abs(d[m]).max() < 1e-13 and np.abs(vm[m]).max() < 1e-14
        st = o.solid_stats(s)
        assert st[6] < 1e-13 and st[7] < 1e-13


def _boundary_points(shape, a, b, n=400000):
    t = np.linspace(0, 2 * np.pi, n, endpoint=False)
    if shape == "ellipse":
        return np.stack([a * np.cos(t), b * np.sin(t)], 1)
    # rectangle perimeter, uniformly
    per = 4 * (a + b)
    s = np.linspace(0, per, n, endpoint=False)
    pts = np.empty((n, 2))
    for k, v in enumerate(s):
        if v < 2 * a:
            pts[k] = (-a + v, -b)
        elif v < 2 * a + 2 * b:
            pts[k] = (a, -b + (v - 2 * a))
        elif v < 4 * a + 2 * b:
            pts[k] = (a - (v - 2 * a - 2 * b), b)
        else:
            pts[k] = (-a, b - (v - 4 * a - 2 * b))
    corners = np.array([[-a, -b], [a, -b], [a, b], [-a, b]])  # the nearest point may be a corner
    return np.concatenate([pts, corners])


@pytest.mark.parametrize("shape,a,b", [("ellipse", 11.0, 6.0), ("ellipse", 4.0, 9.5), ("rect", 9.0, 5.0),
                                       ("rect", 6.0, 6.0)])
def test_shape_signed_distance_brute_force(shape, a, b):
    # phi_0 is the signed distance to the boundary (negative inside): checked
    # against the nearest of 4e5 boundary samples (spacing < 2e-4, so the
    # sampled distance is within ~1e-8 of the exact one away from the samples)
    rng = np.random.default_rng(7)
    pts = _boundary_points(shape, a, b)
    q = rng.uniform(-1.6 * max(a, b), 1.6 * max(a, b), size=(60, 2))
    for qx, qy in q:
        d = np.sqrt(((pts - (qx, qy)) ** 2).sum(1)).min()
        inside = ((qx / a) ** 2 + (qy / b) ** 2 < 1) if shape == "ellipse" else (abs(qx) < a and abs(qy) < b)
        ref = -d if inside else d
        assert abs(oracle.phi0(shape, a, b, qx, qy) - ref) < 1e-6, (qx, qy)


def test_shape_signed_distance_special_cases():
    # an ellipse with equal semi-axes is the disk; points on the axes and at corners
    for qx, qy in [(0.3, -2.0), (7.5, 1.0), (-12.0, 3.0), (0.0, 0.0)]:
        assert abs(oracle.phi0("ellipse", 6, 6, qx, qy) - (np.hypot(qx, qy) - 6)) < 1e-12
        assert abs(oracle.phi0("disk", 6, 6, qx, qy) - (np.hypot(qx, qy) - 6)) < 1e-15
    assert oracle.phi0("ellipse", 10, 5, 0, 0) == -5.0
    assert abs(oracle.phi0("ellipse", 10, 5, 12, 0) - 2.0) < 1e-15
    assert abs(oracle.phi0("ellipse", 10, 5, 0, -7) - 2.0) < 1e-15
    assert abs(oracle.phi0("rect", 4, 2, 5, 3) - np.sqrt(2)) < 1e-15  # off a corner
    assert oracle.phi0("rect", 4, 2, 1, 0.5) == -1.5                  # inside: distance to the nearer side
    assert oracle.phi0("rect", 4, 2, 6, 0) == 2.0


def test_shapes_initial_area_and_rest():
    # the initial solid set of each shape covers its area (to the perimeter's
    # order), and rest stays an exact fixed point with non-circular solids
    sc = scenarios.shapes_small(0, gravity=0.0)
    o = oracle.Oracle(sc)
    for k, s in enumerate(sc["solids"]):
        lab = o.field("label", k)
        n = int((lab == 0).sum())
        shape = s.get("shape", "disk")
        area = {"disk": np.pi * s["r"] ** 2, "ellipse": np.pi * s.get("a", 0) * s.get("b", 0),
                "rect": 4 * s.get("a", 0) * s.get("b", 0)}[shape]
        per = 2 * np.pi * _shape_r(s) if shape != "rect" else 4 * (s["a"] + s["b"])
        assert abs(n - area) < per, (shape, n, area)
    f0 = o.populations()
    o.step(25)
    assert np.abs(o.populations() - f0).max() < 1e-12
    assert np.abs(o.field("ux")).max() < 1e-13 and np.abs(o.field("uy")).max() < 1e-13


def _shape_r(s):
    return s["r"] if s.get("shape", "disk") == "disk" else max(s["a"], s["b"])


# --------------------------------------------------------------------------
# Upwind side, overlap normalisation and divergence assembly on prescribed
# reference maps (oracle.set_refmap writes xi on the solid and band nodes)
# --------------------------------------------------------------------------
def _grid(nx, ny):
    return (np.arange(nx)[None, :].repeat(ny, 0).astype(float),
            np.arange(ny)[:, None].repeat(nx, 1).astype(float))


@pytest.mark.parametrize("U", [0.02, -0.02])
def test_upwind_side_on_a_quartic_reference_map(U):
    # Eq. 3_1_eno differences against the flow: (3 xi_0 - 4 xi_-1 + xi_-2) / 2 for
    # u > 0 and (-3 xi_0 + 4 xi_1 - xi_2) / 2 for u < 0.  Both are exact on
    # quadratics and share the h^2 term; on a quartic they differ in the h^3
    # term, exactly: backward = xi' - xi'''/3 + xi''''/4, forward = xi' - xi'''/3
    # - xi''''/4.  So one advection step of xi_x = x + a (x - x0)^4 in a uniform
    # flow (U, V) is xi_x - U (xi' - xi'''/3 + s xi''''/4), s = sign of U, on
    # every node of the advected set (xi_x does not vary in y, so the y
    # difference is exactly zero).
    nx, ny, x0, a, V = 64, 48, 31.0, 1e-6, 0.013
    sc = scenarios.fluid_only(nx, ny, 0, 0, 0.7)
    sc["solids"].append({"x": 31.0, "y": 24.0, "r": 9.0, "rho_s": 1.0, "G": 0.0})
    o = oracle.Oracle(sc)
    f = np.zeros((9, ny, nx))
    f[:] = oracle.feq(1.0, U, V, 0.0)[:, None, None]
    o.set_populations(f)
    x, y = _grid(nx, ny)
    X = x + a * (x - x0) ** 4
    o.set_refmap(0, X, y)
    phi = o.field("phi", 0)
    S = np.isfinite(phi) & (phi < -1e-9)
    assert S.sum() > 200
    o.step(1)
    xi = o.field("xi_x", 0)
    s = x - x0
    d1, d3, d4 = 1 + 4 * a * s ** 3, 24 * a * s, 24 * a
    side = 1.0 if U > 0 else -1.0
    expect = X - U * (d1 - d3 / 3 + side * d4 / 4)
    wrong = X - U * (d1 - d3 / 3 - side * d4 / 4)  # the stencil from the downwind side
    assert np.abs(xi[S] - expect[S]).max() < 1e-12
    assert np.abs(xi[S] - wrong[S]).min() > 0.5 * abs(U) * 12 * a
    o.close()


def _edge_weights(phi, eps, c=lambda lam: lam):
    """Blend weights c(lambda) of the x-edges left/right and y-edges
    below/above every node, lambda = 1 - H(mean phi of the edge's two nodes)
    (zero where a node has no value: beyond the band lambda is zero)."""
    H = np.vectorize(lambda p: oracle.heaviside(p, eps) if np.isfinite(p) else 1.0)
    lx = c(1.0 - H(0.5 * (phi + np.roll(phi, 1, axis=1))))   # edge (i - 1/2, j)
    ly = c(1.0 - H(0.5 * (phi + np.roll(phi, 1, axis=0))))   # edge (i, j - 1/2)
    return lx, np.roll(lx, -1, axis=1), ly, np.roll(ly, -1, axis=0)


def _stretched(sc, stretch, copies):
    """Oracle with `copies` coincident copies of the scenario's solid, each
    given the uniform stretch xi = c + diag(1/stretch, stretch) (x - c)."""
    sc = dict(sc, solids=sc["solids"] * copies)
    o = oracle.Oracle(sc)
    x, y = _grid(sc["nx"], sc["ny"])
    s0 = sc["solids"][0]
    for k in range(copies):
        o.set_refmap(k, s0["x"] + (x - s0["x"]) / stretch, s0["y"] + (y - s0["y"]) * stretch)
    return o


def test_overlap_blend_is_normalised_by_sum_lambda():
    # Eq. 3_6_global_stress: the blended solid stress sum lambda_s tau_s is divided
    # by sum lambda where that exceeds one; Delta rho (Eq. 2_3_drho) and the solid
    # accelerations are blended the same way.  Two coincident copies of one
    # uniformly stretched solid have lambda_1 = lambda_2 = lambda everywhere, so
    # every blended quantity is min(1, 2 lambda) / lambda times the single
    # copy's, and with the stretch's uniform tau_s (its closed form is pinned
    # above) the force at a node is tau_s applied to the differences of the
    # edge weights.  The copies' contact stress vanishes (phi_s - phi_t has no
    # gradient).
    stretch, G, rho_s = 1.03, 0.01, 1.4
    sc = scenarios.fluid_only(64, 64, 0, 0, 0.8)
    sc["solids"].append({"x": 32.2, "y": 31.7, "r": 10.0, "rho_s": rho_s, "G": G})
    J = [[1.0 / stretch, 0.0], [0.0, stretch]]
    txx, txy, tyy = oracle.stress_from_jacobian(J, G)
    assert abs(txx) > 1e-4 and abs(txy) < 1e-18
    one, two = _stretched(sc, stretch, 1), _stretched(sc, stretch, 2)
    one.step(1)
    two.step(1)
    phi = one.field("phi", 0)
    assert np.array_equal(np.isfinite(phi), np.isfinite(two.field("phi", 1)))
    lam = np.where(np.isfinite(phi), 1.0 - np.vectorize(lambda p: oracle.heaviside(p, 1.5))(np.nan_to_num(phi, nan=9.0)), 0.0)
    assert ((2 * lam > 1) & (lam < 1)).any() and ((2 * lam < 1) & (lam > 0)).any()
    # Delta rho at the nodes
    d1, d2 = one.field("drho"), two.field("drho")
    assert np.abs(d1 - lam * (rho_s - 1.0)).max() < 1e-14
    assert np.abs(d2 - np.minimum(1.0, 2 * lam) * (rho_s - 1.0)).max() < 1e-14
    # force density: divergence of the blended uniform stress
    for o, c in ((one, lambda l: l), (two, lambda l: np.minimum(1.0, 2 * l))):
        wl, wr, wb, wt = _edge_weights(phi, 1.5, c)
        fx = txx * (wr - wl) + txy * (wt - wb)
        fy = txy * (wr - wl) + tyy * (wt - wb)
        # (the band's least-squares fits reproduce the linear map to ~1e-13)
        assert np.abs(o.field("Fx") - fx).max() < 1e-12
        assert np.abs(o.field("Fy") - fy).max() < 1e-12
    assert np.abs(two.field("Fx") - one.field("Fx")).max() > 1e-6  # the normalisation acts
    one.close(); two.close()
    # solid accelerations (G = 0: no stress): a_s = -(1 - rho_f / rho_s) g
    g = 1e-4
    sc0 = dict(sc, gravity=g, solids=[dict(sc["solids"][0], G=0.0)])
    one, two = _stretched(sc0, stretch, 1), _stretched(sc0, stretch, 2)
    one.step(1)
    two.step(1)
    a_s = -(1.0 - 1.0 / rho_s) * g
    assert np.abs(one.field("Fy") - lam * a_s).max() < 1e-18
    assert np.abs(two.field("Fy") - np.minimum(1.0, 2 * lam) * a_s).max() < 1e-18
    one.close(); two.close()


def test_divergence_of_a_sinusoidal_shear():
    # Eqs. 3_3_refmap_jacobian .. 3_3_div_solid_stress on a small shear
    # displacement u = (A sin(k y), 0) inside a large solid: xi = x - u, so
    # J = I - grad u, F = J^-1 = I + grad u + O(A^2) and the neo-Hookean stress is
    # tau_xy = G du_x/dy, tau_xx = tau_yy = O(A^2).  On the half-edge stencils the
    # y-edge difference of xi_x is -2 A sin(k/2) cos(k (j - 1/2)), so the divergence
    # at a node of the solid's interior is F_x = -4 G A sin^2(k/2) sin(k j), the
    # discrete form of G d^2 u_x / dy^2, and F_y = O(A^2).  A swapped face, a
    # transposed component or a sign slip in the assembly fails this.
    nx = ny = 96
    A, k, G = 1e-5, 2 * np.pi / 12, 0.02
    sc = scenarios.fluid_only(nx, ny, 0, 0, 0.8)
    sc["solids"].append({"x": 48.3, "y": 47.6, "r": 30.0, "rho_s": 1.0, "G": G})
    o = oracle.Oracle(sc)
    x, y = _grid(nx, ny)
    o.set_refmap(0, x - A * np.sin(k * y), y)
    o.step(1)
    phi = o.field("phi", 0)
    inner = np.isfinite(phi) & (phi < -(1.5 + 3.0))
    assert inner.sum() > 1500
    fx = -4 * G * A * np.sin(k / 2) ** 2 * np.sin(k * y)
    amp = 4 * G * A * np.sin(k / 2) ** 2
    assert np.abs(o.field("Fx")[inner] - fx[inner]).max() < 1e-3 * amp
    assert np.abs(o.field("Fy")[inner]).max() < 1e-3 * amp
    assert np.abs(o.field("Fx")[inner]).max() > 0.9 * amp
    o.close()


def test_conservative_force_mode_conserves_momentum():
    # force_mode 1 leaves the stress divergence without rho in the Guo term and
    # the half-force moments (Sec. 3.4).  The divergence of the blended stress
    # telescopes to zero over a periodic box (Eq. 3_3_div_solid_stress sums
    # differences of half-edge stresses), so with no external force the total
    # momentum sum rho u is conserved to round-off while the solid deforms; the
    # literal form (mode 0) multiplies the divergence by the non-uniform rho and
    # changes it.
    n, U = 48, 2e-3
    base = scenarios.fluid_only(n, n, 0, 0, 0.8)
    base["solids"].append({"x": 23.4, "y": 24.2, "r": 8.0, "rho_s": 1.3, "G": 0.01})
    y = np.arange(n)[:, None].repeat(n, 1)
    drift = {}
    for mode in (0, 1):
        o = oracle.Oracle(dict(base, force_mode=mode))
        f = np.stack([oracle.feq(1.0, U * math.sin(2 * math.pi * yy / n), 0.0, 0.0) for yy in range(n)], axis=1)
        o.set_populations(np.repeat(f[:, :, None], n, axis=2))
        p0 = None
        worst = 0.0
        for _ in range(30):
            o.step(1)
            rho = o.field("rho")
            p = np.array([(rho * o.field("ux")).sum(), (rho * o.field("uy")).sum()])
            p0 = p if p0 is None else p0
            worst = max(worst, np.abs(p - p0).max())
        # the solid deforms: its stress divergence is not small
        assert np.abs(o.field("Fx")).max() > 1e-7
        assert abs(o.field("Fx").sum()) < 1e-15 and abs(o.field("Fy").sum()) < 1e-15
        drift[mode] = worst
        o.close()
    # momentum ~ U n^2 / pi = 1.5: round-off of its sum over n^2 nodes is ~1e-14
    assert drift[1] < 1e-13
    assert drift[0] > 1e-10


def test_contact_forces_are_equal_and_opposite():
    # The net contact force on a solid (the divergence of its pairs' contact
    # stresses, Eqs. 3_6_collision_stress .. 3_6_normal and 3_3_div_solid_stress,
    # over the nodes nearer to it) is a reading: the paper gives the stress, not
    # a per-solid force.  Whatever the split of the nodes, one pair's divergence
    # telescopes to zero over a periodic box, so the two forces cancel (Newton's
    # third law); they push the solids apart; a solid without a partner feels none.
    sc = scenarios.contact_pair(gap=0.8, nx=96, ny=64)
    o = oracle.Oracle(sc)
    o.step(1)
    a, b = o.solid_stats(0), o.solid_stats(1)
    fa, fb = a[8:10], b[8:10]
    assert np.linalg.norm(fa) > 1e-5
    assert np.abs(fa + fb).max() < 1e-14 * np.abs(fa).max() * 100
    ca, cb = a[1:3], b[1:3]
    assert np.dot(fa, ca - cb) > 0 and np.dot(fb, cb - ca) > 0  # repulsive
    o.close()
    far = scenarios.contact_pair(gap=8.0, nx=96, ny=64)
    o = oracle.Oracle(far)
    o.step(1)
    assert np.all(o.solid_stats(0)[8:10] == 0.0) and np.all(o.solid_stats(1)[8:10] == 0.0)
    o.close()
