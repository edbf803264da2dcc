"""Seeded synthetic inputs for the LBRMT time step.

This module is the one place both the CUDA path and the FP64 oracle take their
inputs from.  It holds no arithmetic of the method: it only draws solid
placements and material constants and returns plain dictionaries.  Both sides
consume the same dictionary (grid, walls, relaxation time, forcing, solids).

Lattice units throughout: dx = dt = 1 and rho_f = 1 (paper, Sec. 4 intro and
Appendix A).  The blur-zone half-width eps = 1.5 and the 11 extrapolation
layers are the values the paper uses for every result (Sec. 4 intro).

Scenario keys
-------------
nx, ny        grid nodes in x and y
wall_x/wall_y 0 = periodic, 1 = no-slip halfway bounce-back walls (Sec. 3.5)
tau, rho_f    BGK relaxation time and fluid density
lid_u         speed of the top wall in +x (0 = static); lid-driven cavity, Sec. 4.1
eps, n_layers blur-zone half-width and extrapolation layers
eta           contact-stress constant of Eq. (3_6_collision_stress)
gravity       g > 0 acting in -y; a solid feels (1 - rho_f/rho_s) g (Sec. 4.3)
force_kind    0 none, 1 constant (force_a), 2 sinusoidal f_x = A sin(2 pi y / ny)
              applied to all phases
force_a       [fx, fy] for kind 1, [A, 0] for kind 2
solids        list of {"x", "y", "r", "rho_s", "G"} disks (centre, radius,
              density, small-strain shear modulus)
"""
from __future__ import annotations

import math
import numpy as np

EPS = 1.5
N_LAYERS = 11


def _base(nx, ny, wall_x, wall_y, tau, lid_u=0.0, gravity=0.0, force_kind=0,
          force_a=(0.0, 0.0), eta=1.0, name=""):
    return {
        "name": name, "nx": int(nx), "ny": int(ny),
        "wall_x": int(wall_x), "wall_y": int(wall_y),
        "tau": float(tau), "rho_f": 1.0, "lid_u": float(lid_u),
        "eps": EPS, "n_layers": N_LAYERS, "eta": float(eta),
        "gravity": float(gravity), "force_kind": int(force_kind),
        "force_a": [float(force_a[0]), float(force_a[1])],
        "solids": [],
    }


def _min_image(d, n, periodic):
    if periodic:
        d = (d + 0.5 * n) % n - 0.5 * n
    return d


def place_disks(rng, sc, count, r_lo, r_hi, rho_lo, rho_hi, g_lo, g_hi,
                max_tries=200, r_choice=None):
    """Rejection-sample non-overlapping disks.

    Surface gap between disks >= 2*eps + 1 = 4 cells; gap to a no-slip wall
    >= eps + 2 cells.  Disks that fail ``max_tries`` placements are dropped;
    the realised count is len(sc["solids"]).
    """
    nx, ny = sc["nx"], sc["ny"]
    px, py = sc["wall_x"] == 0, sc["wall_y"] == 0
    gap = 2 * EPS + 1
    wall_gap = EPS + 2
    placed = sc["solids"]
    for _ in range(count):
        r = float(rng.uniform(r_lo, r_hi)) if r_choice is None else float(rng.choice(r_choice))
        rho_s = float(rng.uniform(rho_lo, rho_hi))
        G = float(rng.uniform(g_lo, g_hi))
        for _t in range(max_tries):
            lo_x = 0.0 if px else r + wall_gap - 0.5
            hi_x = float(nx) if px else nx - 0.5 - r - wall_gap
            lo_y = 0.0 if py else r + wall_gap - 0.5
            hi_y = float(ny) if py else ny - 0.5 - r - wall_gap
            if hi_x <= lo_x or hi_y <= lo_y:
                break
            x = float(rng.uniform(lo_x, hi_x))
            y = float(rng.uniform(lo_y, hi_y))
            ok = True
            for s in placed:
                dx = _min_image(x - s["x"], nx, px)
                dy = _min_image(y - s["y"], ny, py)
                if math.hypot(dx, dy) < r + s["r"] + gap:
                    ok = False
                    break
            if ok:
                placed.append({"x": x, "y": y, "r": r, "rho_s": rho_s, "G": G})
                break
    return sc


# ---------------------------------------------------------------------------
# The five workloads (deterministic given the seed)
# ---------------------------------------------------------------------------

def ldc_disk_64():
    """Lid-driven cavity 64x64, lid 0.05, tau 0.8, one disk r=12 at (32,38),
    rho_s/rho_f = 1, G = 0.01 (template: the paper's Sec. 4.1 benchmark)."""
    sc = _base(64, 64, 1, 1, 0.8, lid_u=0.05, name="ldc_disk_64")
    sc["solids"].append({"x": 32.0, "y": 38.0, "r": 12.0, "rho_s": 1.0, "G": 0.01})
    return sc


def settling_512(seed=0):
    """512x512, periodic x, no-slip y, tau 0.7, 24 disks r~U[10,20],
    rho_s~U[1.2,2.0], G~U[0.005,0.02], gravity 1e-5, contact on (Sec. 4.3-4.4)."""
    rng = np.random.default_rng(seed)
    sc = _base(512, 512, 0, 1, 0.7, gravity=1e-5, name=f"settling_512_s{seed}")
    return place_disks(rng, sc, 24, 10, 20, 1.2, 2.0, 0.005, 0.02)


def mixing_4096(seed=0, n=4096, count=1024):
    """4096x4096 fully periodic, tau 0.6, f_x = 1e-5 sin(2 pi y/ny) on all
    phases, 1024 disks r~U[8,24], rho_s~U[1.0,1.5], G~U[0.002,0.02]."""
    rng = np.random.default_rng(seed)
    sc = _base(n, n, 0, 0, 0.6, force_kind=2, force_a=(1e-5, 0.0),
               name=f"mixing_{n}_s{seed}")
    return place_disks(rng, sc, count, 8, 24, 1.0, 1.5, 0.002, 0.02)


def ldc_ensemble(seed=0, count=96):
    """96 lid-driven cavities, side ~ U{128,192,256,384,512}, 1-8 disks each
    with r~U[8,40], G~U[0.005,0.05], lid_u~U[0.02,0.08]; tau 0.8, rho_s = 1."""
    rng = np.random.default_rng(seed)
    sims = []
    for k in range(count):
        side = int(rng.choice([128, 192, 256, 384, 512]))
        lid = float(rng.uniform(0.02, 0.08))
        sc = _base(side, side, 1, 1, 0.8, lid_u=lid, name=f"ldc_ens_{seed}_{k}")
        nd = int(rng.integers(1, 9))
        r_hi = min(40.0, side / 4.0)
        place_disks(rng, sc, nd, 8, r_hi, 1.0, 1.0, 0.005, 0.05)
        sims.append(sc)
    return sims


def adjoint_ldc_256():
    """256x256 lid-driven cavity, tau 0.8, one disk r=40 at (0.6L, 0.5L)."""
    sc = _base(256, 256, 1, 1, 0.8, lid_u=0.05, name="adjoint_ldc_256")
    sc["solids"].append({"x": 0.6 * 256, "y": 0.5 * 256, "r": 40.0, "rho_s": 1.0, "G": 0.01})
    return sc


def adjoint_ldc(n=256, r=40.0, G=0.01, rho_ratio=1.0, lid_u=0.05, body=None):
    """Lid-driven cavity of side n (tau 0.8) with one disk of radius r at
    (0.6n, 0.5n) and a per-node body force field (force_kind 3): ``body`` of
    shape (2, n, n), zero by default."""
    sc = _base(n, n, 1, 1, 0.8, lid_u=lid_u, force_kind=3, name=f"adjoint_ldc_{n}")
    sc["solids"].append({"x": 0.6 * n, "y": 0.5 * n, "r": float(r), "rho_s": float(rho_ratio) * sc["rho_f"],
                         "G": float(G)})
    sc["body_field"] = np.zeros((2, n, n)) if body is None else np.asarray(body, dtype=np.float64).reshape(2, n, n)
    return sc


def smooth_body_field(seed, n, amp=1e-5, modes=3):
    """Seeded smooth body force field (2, n, n): a few low Fourier modes per
    component with amplitudes up to ``amp``."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:n, 0:n] / float(n)
    out = np.zeros((2, n, n))
    for c in range(2):
        for _ in range(modes):
            kx, ky = rng.integers(1, 4, size=2)
            ph = rng.uniform(0, 2 * np.pi)
            out[c] += rng.uniform(-amp, amp) * np.sin(2 * np.pi * (kx * x + ky * y) + ph)
    return out


# ---------------------------------------------------------------------------
# Small seeded cases for parity tests (sizes the oracle finishes in seconds)
# ---------------------------------------------------------------------------

def settling_small(seed=0, nx=96, ny=80, count=3, gravity=2e-4):
    rng = np.random.default_rng(1000 + seed)
    sc = _base(nx, ny, 0, 1, 0.7, gravity=gravity, name=f"settling_small_s{seed}")
    return place_disks(rng, sc, count, 6, 10, 1.2, 2.0, 0.005, 0.02)


def mixing_small(seed=0, n=96, count=5, amp=2e-4):
    rng = np.random.default_rng(2000 + seed)
    sc = _base(n, n, 0, 0, 0.6, force_kind=2, force_a=(amp, 0.0),
               name=f"mixing_small_s{seed}")
    return place_disks(rng, sc, count, 6, 12, 1.0, 1.5, 0.002, 0.02)


def contact_pair(gap=1.0, nx=80, ny=48, speed=0.0):
    """Two disks whose blur zones overlap (surface gap < 2 eps), periodic box,
    pushed together by opposite body accelerations through gravity-free
    sinusoidal forcing off; exercises the contact stress."""
    sc = _base(nx, ny, 0, 0, 0.7, name=f"contact_pair_g{gap}")
    r = 9.0
    cx, cy = nx / 2.0, ny / 2.0 + 0.3
    sc["solids"].append({"x": cx - r - gap / 2 - 0.2, "y": cy, "r": r, "rho_s": 1.3, "G": 0.02})
    sc["solids"].append({"x": cx + r + gap / 2 + 0.1, "y": cy - 0.4, "r": r, "rho_s": 1.1, "G": 0.01})
    return sc


def ragged_wrap(nx=100, ny=74, walls=False):
    """A grid no registry tile shape divides, with disks that straddle the
    periodic boundaries (one across x = 0, one across y = 0 and x = nx, one
    inside); with walls=True no-slip walls in y instead, gravity, and the disks
    near the walls without touching them.  Sinusoidal body force, tau 0.7."""
    if walls:
        sc = _base(nx, ny, 0, 1, 0.7, gravity=1e-4, name=f"ragged_walls_{nx}x{ny}")
        sc["solids"].append({"x": 1.5, "y": 14.3, "r": 8.0, "rho_s": 1.4, "G": 0.01})
        sc["solids"].append({"x": nx - 3.2, "y": ny - 13.6, "r": 7.5, "rho_s": 1.2, "G": 0.02})
        sc["solids"].append({"x": 0.45 * nx, "y": 0.5 * ny, "r": 9.0, "rho_s": 1.3, "G": 0.015})
        return sc
    sc = _base(nx, ny, 0, 0, 0.7, force_kind=2, force_a=(2e-4, 0.0), name=f"ragged_wrap_{nx}x{ny}")
    sc["solids"].append({"x": 1.3, "y": 0.55 * ny, "r": 8.0, "rho_s": 1.3, "G": 0.01})
    sc["solids"].append({"x": nx - 2.6, "y": 1.7, "r": 7.0, "rho_s": 1.15, "G": 0.02})
    sc["solids"].append({"x": 0.5 * nx, "y": 0.3 * ny, "r": 6.5, "rho_s": 1.45, "G": 0.012})
    return sc


def fluid_only(nx, ny, wall_x, wall_y, tau, lid_u=0.0, force_kind=0, force_a=(0.0, 0.0)):
    return _base(nx, ny, wall_x, wall_y, tau, lid_u=lid_u, force_kind=force_kind,
                 force_a=force_a, name="fluid_only")


ALL = {
    "ldc_disk_64": ldc_disk_64,
    "settling_512": settling_512,
    "mixing_4096": mixing_4096,
    "adjoint_ldc_256": adjoint_ldc_256,
}


def _shape_radius(s):
    """Circumscribed radius of a solid dict."""
    shape = s.get("shape", "disk")
    if shape == "disk":
        return s["r"]
    return max(s["a"], s["b"]) if shape == "ellipse" else math.hypot(s["a"], s["b"])


def place_shapes(rng, sc, specs, rho_lo, rho_hi, g_lo, g_hi, max_tries=400):
    """Rejection-sample non-overlapping solids of the given shapes (dicts with
    'shape' and 'a', 'b' or 'r'), using their circumscribed radii for the
    surface gap >= 2 eps + 1 and the wall gap >= eps + 2."""
    nx, ny = sc["nx"], sc["ny"]
    px, py = sc["wall_x"] == 0, sc["wall_y"] == 0
    gap, wall_gap = 2 * EPS + 1, EPS + 2
    placed = sc["solids"]
    for spec in specs:
        r = _shape_radius(spec)
        rho_s = float(rng.uniform(rho_lo, rho_hi))
        G = float(rng.uniform(g_lo, g_hi))
        for _t in range(max_tries):
            lo_x, hi_x = (0.0, float(nx)) if px else (r + wall_gap - 0.5, nx - 0.5 - r - wall_gap)
            lo_y, hi_y = (0.0, float(ny)) if py else (r + wall_gap - 0.5, ny - 0.5 - r - wall_gap)
            if hi_x <= lo_x or hi_y <= lo_y:
                break
            x, y = float(rng.uniform(lo_x, hi_x)), float(rng.uniform(lo_y, hi_y))
            if all(math.hypot(_min_image(x - s["x"], nx, px), _min_image(y - s["y"], ny, py))
                   >= r + _shape_radius(s) + gap for s in placed):
                placed.append(dict(spec, x=x, y=y, r=r, rho_s=rho_s, G=G))
                break
    return sc


def heavy_disk_drift(n=96, r=12.0, tau=0.6, G=0.02, rho_s=1.5, accel=-1e-5):
    """A single disk in an n x n periodic box, everything driven by one uniform
    acceleration (force on all phases): the stiffest, heaviest disk of the
    4096^2 mixing workload at its tau, in the near-uniform part of its forcing."""
    sc = _base(n, n, 0, 0, tau, force_kind=1, force_a=(accel, 0.0), name=f"heavy_disk_drift_{n}")
    sc["solids"].append({"x": n / 2 + 0.3, "y": n / 2 + 0.17, "r": float(r), "rho_s": float(rho_s), "G": float(G)})
    return sc


def shapes_small(seed=0, nx=128, ny=96, gravity=2e-4):
    """128x96 box, periodic x, walls y, tau 0.7, gravity: a horizontal and a
    vertical ellipse, a square, a rectangle and a disk, rho_s~U[1.1,1.6],
    G~U[0.005,0.02]."""
    rng = np.random.default_rng(3000 + seed)
    sc = _base(nx, ny, 0, 1, 0.7, gravity=gravity, name=f"shapes_small_s{seed}")
    specs = [{"shape": "ellipse", "a": 11.0, "b": 6.0}, {"shape": "ellipse", "a": 5.0, "b": 10.0},
             {"shape": "rect", "a": 6.0, "b": 6.0}, {"shape": "rect", "a": 9.0, "b": 5.0},
             {"shape": "disk", "r": 7.0}]
    return place_shapes(rng, sc, specs, 1.1, 1.6, 0.005, 0.02)


def mixing_ellipses(seed=0, nx=800, ny=450, a=8.0, b=4.0, gravity=2e-5, G=0.05):
    """Mixing of 506 ellipses (Sec. 4, the 800x450 case): walls on all sides,
    tau 1, 242 heavier (rho_s 1.25) and 264 lighter (rho_s 0.83) ellipses with
    semi-axes a x b, lying and standing alternately on a 23 x 22 lattice (each
    jittered by up to half a node).  The paper gives neither the ellipse size
    nor gravity, and its G = 1 is in physical units (in lattice units it would
    break the shear-wave limit G <= rho_s of its Appendix A): a = 8, b = 4,
    g = 2e-5 and G = 0.05 (shear wave speed 0.2-0.25 nodes per step) are chosen."""
    rng = np.random.default_rng(4000 + seed)
    sc = _base(nx, ny, 1, 1, 1.0, gravity=gravity, name=f"mixing_ellipses_s{seed}")
    heavy = np.zeros(506, dtype=bool)
    heavy[rng.choice(506, 242, replace=False)] = True
    m = 11.5
    xs = m + np.arange(23) * (nx - 1 - 2 * m) / 22.0
    ys = m + np.arange(22) * (ny - 1 - 2 * m) / 21.0
    k = 0
    for iy, y in enumerate(ys):
        for ix, x in enumerate(xs):
            lying = (ix + iy) % 2 == 0
            sc["solids"].append({"shape": "ellipse", "a": a if lying else b, "b": b if lying else a,
                                 "r": max(a, b), "x": float(x + rng.uniform(-0.5, 0.5)),
                                 "y": float(y + rng.uniform(-0.5, 0.5)),
                                 "rho_s": 1.25 if heavy[k] else 0.83, "G": float(G)})
            k += 1
    return sc


def ldc_convergence(L, tau=0.8, re=100.0, g_over_rho_u2=0.1, t80=2000):
    """The grid-convergence case of Sec. 4.1 at resolution L: an L x L cavity with
    a disk of radius 0.2L at (0.6L, 0.5L), rho_s = rho_f, Re = U L / nu = 100.
    The paper gives the physical parameters only; in lattice units: tau 0.8
    (nu = 0.1), lid U = Re nu / L, and the shear modulus scaled with the lid's
    dynamic pressure, G = 0.1 rho_f U^2 (the paper's G = 0.1 read in lid
    units), so the same physical problem at every L under diffusive scaling
    (time steps ~ L^2, as the paper's 20000 steps at L = 80 and 1.28e6 at 640).
    The run length is t80 (L/80)^2 steps: the paper's full length carries the
    disk against the side wall, where the paper applies a solid-wall contact
    force that this library does not implement, so the study stops at 2000 (L/80)^2
    steps, before the disk nears a wall."""
    nu = (tau - 0.5) / 3.0
    U = re * nu / L
    sc = _base(L, L, 1, 1, tau, lid_u=U, name=f"ldc_convergence_{L}")
    sc["solids"].append({"x": 0.6 * L, "y": 0.5 * L, "r": 0.2 * L, "rho_s": 1.0,
                         "G": g_over_rho_u2 * U * U})
    sc["steps"] = int(round(t80 * (L / 80.0) ** 2))
    sc["deform_margin"] = 0.6  # the soft disk stretches along the flow
    return sc
