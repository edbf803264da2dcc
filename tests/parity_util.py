"""Helpers shared by the GPU parity tests: run the CUDA path and the FP64
oracle on the same scenario and compare field by field.

Error measure: relative L-infinity, max |gpu - oracle| / D, over nodes where
both are finite.  Vector fields (u, v) and (F_x, F_y) are compared as vectors:
D is the largest magnitude of the oracle's vector field.  D has a floor, the
magnitude below which a field is at the level of round-off of the method
itself (a fluid at rest, a force that is exactly zero after one step):
  rho - rho_f : 1e-4 rho_f        velocity : 1e-6
  force F     : 1e-6              drho     : 1e-6
  xi - x      : 1 lattice spacing (so the xi error is absolute, in cells)
The density floor is the FP32 resolution of the stored populations: their
deviations from w_q rho_f reach 6 w_q rho lid_u (8e-3 at a lid of 0.05), whose
FP32 rounding alone moves rho by ~1e-9, a relative 1e-5 of a density deviation
of 1e-4 (tests/test_fp32_floors.py shows it on the oracle's own populations).
"""
import numpy as np

import oracle
import scenarios  # noqa: F401  (re-exported for the tests)

FLOORS = {"rho": 1e-4, "u": 1e-6, "F": 1e-6, "drho": 1e-6, "xi": 1.0}


def rel_linf(a, b, floor=0.0, mask=None):
    m = np.isfinite(a) & np.isfinite(b)
    if mask is not None:
        m &= mask
    if not m.any():
        return 0.0
    den = max(np.abs(b[m]).max(), floor)
    return float(np.abs(a[m] - b[m]).max() / den) if den > 0 else float(np.abs(a[m] - b[m]).max())


def rel_linf_vec(ax, ay, bx, by, floor):
    m = np.isfinite(ax) & np.isfinite(bx) & np.isfinite(ay) & np.isfinite(by)
    if not m.any():
        return 0.0
    den = max(np.hypot(bx[m], by[m]).max(), floor)
    return float(np.hypot(ax[m] - bx[m], ay[m] - by[m]).max() / den)


def grid_x(sc):
    ny, nx = sc["ny"], sc["nx"]
    return (np.arange(nx)[None, :].repeat(ny, 0).astype(float),
            np.arange(ny)[:, None].repeat(nx, 1).astype(float))


def _abs_vec(ax, ay, bx, by):
    m = np.isfinite(ax) & np.isfinite(bx) & np.isfinite(ay) & np.isfinite(by)
    if not m.any():
        return 0.0, 0.0
    return float(np.hypot(ax[m] - bx[m], ay[m] - by[m]).max()), float(np.hypot(bx[m], by[m]).max())


def compare(sim, ref, sc, core_layers=4, solids=None):
    """Per-field errors (see module doc) and band-label mismatch counts.

    xi is compared on the solid and the first ``core_layers`` band layers
    (the nodes whose values enter the stress stencils and the advection
    stencils), and separately over the whole band (``xi_band``), for every
    solid or for the ids in ``solids``.  The absolute errors and the
    oracle's field magnitudes are returned too (``*_abs``, ``*_max``)."""
    out = {}
    rf = sc["rho_f"]
    ra, rb = sim.field_host("rho") - rf, ref.field("rho") - rf
    out["rho"] = rel_linf(ra, rb, FLOORS["rho"] * rf)
    out["rho_abs"] = float(np.abs(ra - rb).max())
    out["rho_max"] = float(np.abs(rb).max())
    ua = (sim.field_host("ux"), sim.field_host("uy"), ref.field("ux"), ref.field("uy"))
    out["u"] = rel_linf_vec(*ua, FLOORS["u"])
    out["u_abs"], out["u_max"] = _abs_vec(*ua)
    fa = (sim.field_host("Fx"), sim.field_host("Fy"), ref.field("Fx"), ref.field("Fy"))
    out["F"] = rel_linf_vec(*fa, FLOORS["F"])
    out["F_abs"], out["F_max"] = _abs_vec(*fa)
    out["drho"] = rel_linf(sim.field_host("drho"), ref.field("drho"), FLOORS["drho"])
    X, Y = grid_x(sc)
    nx, ny = sc["nx"], sc["ny"]
    core, band, mism = 0.0, 0.0, 0
    for s in (range(len(sc["solids"])) if solids is None else solids):
        xa, xb = sim.field_host("xi_x", s), ref.field("xi_x", s)
        ya, yb = sim.field_host("xi_y", s), ref.field("xi_y", s)
        lab = ref.field("label", s)
        ma, mb = np.isfinite(xa), np.isfinite(xb)
        mism += int((ma != mb).sum())
        both = ma & mb
        if not both.any():
            continue
        da = np.hypot(((xa - X + nx / 2) % nx - nx / 2) - ((xb - X + nx / 2) % nx - nx / 2),
                      ((ya - Y + ny / 2) % ny - ny / 2) - ((yb - Y + ny / 2) % ny - ny / 2))
        disp = np.hypot((xb - X + nx / 2) % nx - nx / 2, (yb - Y + ny / 2) % ny - ny / 2)
        den = max(disp[both].max(), FLOORS["xi"])
        band = max(band, float(da[both].max() / den))
        c = both & (lab <= core_layers)
        if c.any():
            core = max(core, float(da[c].max() / den))
    out["xi"] = core
    out["xi_band"] = band
    out["label_mismatch"] = mism
    return out


def run_pair(sc, precision, steps_list, **kw):
    """Run GPU and oracle side by side; return {steps: compare()}."""
    import paper_2402_12696_gb300 as pkg
    sim = pkg.Simulation(sc, precision=precision, **kw)
    ref = oracle.Oracle(sc)
    res = {}
    done = 0
    for n in steps_list:
        sim.step(n - done)
        ref.step(n - done)
        done = n
        sim.sync()
        res[n] = compare(sim, ref, sc)
    sim.close()
    ref.close()
    return res
