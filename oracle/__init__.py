"""FP64 CPU oracle of the LBRMT time step -- TEST INFRASTRUCTURE ONLY.

The oracle (``lbrmt_oracle.c``) is a plain C implementation of Algorithm 1 of
Sun & Rycroft (arXiv 2402.12696) in double precision.  It is used only by the
tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``.  The product path never imports this package and it shares no
code with the CUDA library.

``build()`` compiles ``liblbrmt_oracle.so`` in this directory with gcc
(OpenMP on); ``Oracle`` wraps one simulation built from a scenario dict of the
``scenarios`` module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbrmt_oracle.c")
_LIB = os.path.join(_HERE, "liblbrmt_oracle.so")
_lib = None

FIELDS = {"rho": 0, "ux": 1, "uy": 2, "Fx": 3, "Fy": 4, "drho": 5,
          "xi_x": 10, "xi_y": 11, "phi": 12, "label": 13, "detF_dev": 14, "von_mises": 15}
RMAX = 11


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp",
                               "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        d, i, p = C.c_double, C.c_int, C.c_void_p
        dp = C.POINTER(C.c_double)
        L.oracle_create.restype = p
        L.oracle_create.argtypes = [i, i, i, i, d, d, d, d, i, d, d, i, d, d, i]
        L.oracle_add_solid.argtypes = [p, d, d, d, d, d]
        L.oracle_set_force_mode.argtypes = [p, i]
        L.oracle_set_refmap.argtypes = [p, i, dp, dp]
        L.oracle_set_body_force.argtypes = [p, dp]
        L.oracle_deformation.argtypes = [dp, d, dp]
        L.oracle_add_solid_shape.argtypes = [p, i, d, d, d, d, d, d]
        L.oracle_phi0.argtypes = [i, d, d, d, d]
        L.oracle_phi0.restype = d
        L.oracle_init.argtypes = [p]
        L.oracle_step.argtypes = [p, i]
        L.oracle_read_field.argtypes = [p, i, i, dp]
        L.oracle_solid_stats.argtypes = [p, i, dp]
        L.oracle_set_populations.argtypes = [p, dp]
        L.oracle_steps_done.restype = C.c_long
        L.oracle_steps_done.argtypes = [p]
        L.oracle_error.restype = C.c_char_p
        L.oracle_error.argtypes = [p]
        L.oracle_destroy.argtypes = [p]
        L.oracle_heaviside.restype = d
        L.oracle_heaviside.argtypes = [d, d]
        L.oracle_feq.argtypes = [d, d, d, d, dp]
        L.oracle_guo.argtypes = [d, d, d, d, d, dp]
        L.oracle_stress_from_jacobian.restype = i
        L.oracle_stress_from_jacobian.argtypes = [d, d, d, d, d, dp]
        L.oracle_contact_stress.argtypes = [d, d, d, d, d, d, d, d, dp]
        L.oracle_windows_meet.argtypes = [C.c_int] * 12
        L.oracle_windows_meet.restype = C.c_int
        L.oracle_extrap_target.restype = i
        L.oracle_extrap_target.argtypes = [i, i, C.c_void_p, dp, dp, i, i, i, i, d, d, i, dp, dp]
        L.oracle_num_threads.restype = i
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


SHAPES = {"disk": 0, "ellipse": 1, "rect": 2}


def phi0(shape, a, b, qx, qy):
    """Signed distance of (qx, qy) (relative to the centre) to an axis-aligned
    disk (radius a), ellipse (semi-axes a, b) or rectangle (half-sides a, b)."""
    return lib().oracle_phi0(SHAPES[shape], float(a), float(b), float(qx), float(qy))


def deformation(J, G):
    """(det F - 1, von Mises stress) for the Jacobian J = d xi / dx (2x2)."""
    j = np.ascontiguousarray(np.asarray(J, dtype=np.float64).reshape(4))
    out = np.empty(2)
    if lib().oracle_deformation(_dp(j), float(G), _dp(out)) != 0:
        raise OracleError("singular Jacobian")
    return float(out[0]), float(out[1])


def heaviside(phi, eps):
    return lib().oracle_heaviside(float(phi), float(eps))


def feq(rho, u, v, drho):
    out = np.zeros(9)
    lib().oracle_feq(rho, u, v, drho, _dp(out))
    return out


def guo(rho, u, v, fx, fy):
    out = np.zeros(9)
    lib().oracle_guo(rho, u, v, fx, fy, _dp(out))
    return out


def stress_from_jacobian(J, G):
    out = np.zeros(3)
    ok = lib().oracle_stress_from_jacobian(J[0][0], J[0][1], J[1][0], J[1][1], G, _dp(out))
    return out if ok else None


def contact_stress(phi_s, phi_t, Gs, Gt, eta, eps, gx, gy):
    out = np.zeros(3)
    lib().oracle_contact_stress(phi_s, phi_t, Gs, Gt, eta, eps, gx, gy, _dp(out))
    return out


def windows_meet(a, b, nx, ny, wall_x, wall_y):
    """Do two solid windows (x0, y0, w, h) share a grid node (periodic images included)?"""
    return bool(lib().oracle_windows_meet(*a, *b, nx, ny, int(wall_x), int(wall_y)))


def extrap_target(lab, X, Y, tx, ty, layer, normal=None, rmax=RMAX):
    """Extrapolate one target of a small grid (lab: int8 [h, w])."""
    lab = np.ascontiguousarray(lab, dtype=np.int8)
    X = np.ascontiguousarray(X, dtype=np.float64)
    Y = np.ascontiguousarray(Y, dtype=np.float64)
    h, w = lab.shape
    ox, oy = C.c_double(), C.c_double()
    use_n = normal is not None
    nx, ny = (normal if use_n else (0.0, 0.0))
    r = lib().oracle_extrap_target(w, h, lab.ctypes.data, _dp(X), _dp(Y), tx, ty, layer,
                                   int(use_n), float(nx), float(ny), rmax,
                                   C.byref(ox), C.byref(oy))
    return r, ox.value, oy.value


def num_threads():
    return lib().oracle_num_threads()


class OracleError(RuntimeError):
    pass


class Oracle:
    """One FP64 oracle simulation built from a scenario dict."""

    def __init__(self, sc, rmax=RMAX):
        L = lib()
        self.sc = sc
        self.nx, self.ny = sc["nx"], sc["ny"]
        fa = sc.get("force_a", [0.0, 0.0])
        self.h = L.oracle_create(sc["nx"], sc["ny"], sc["wall_x"], sc["wall_y"], sc["tau"],
                                 sc["rho_f"], sc["lid_u"], sc["eps"], sc["n_layers"],
                                 sc["eta"], sc["gravity"], sc["force_kind"], fa[0], fa[1], rmax)
        if not self.h:
            raise OracleError("oracle_create failed (out of memory?)")
        for s in sc["solids"]:
            shape = SHAPES[s.get("shape", "disk")]
            a, b = (s["r"], s["r"]) if shape == 0 else (s["a"], s["b"])
            if L.oracle_add_solid_shape(self.h, shape, s["x"], s["y"], a, b, s["rho_s"], s["G"]) < 0:
                self._raise()
        if sc.get("force_mode", 0) and L.oracle_set_force_mode(self.h, int(sc["force_mode"])) != 0:
            self._raise()
        if sc["force_kind"] == 3:
            bf = np.ascontiguousarray(sc["body_field"], dtype=np.float64).reshape(2, self.ny, self.nx)
            if L.oracle_set_body_force(self.h, _dp(bf)) != 0:
                self._raise()
        if L.oracle_init(self.h) != 0:
            self._raise()

    def _raise(self):
        raise OracleError(lib().oracle_error(self.h).decode())

    def step(self, n=1):
        if lib().oracle_step(self.h, int(n)) != 0:
            self._raise()

    @property
    def steps_done(self):
        return lib().oracle_steps_done(self.h)

    def field(self, name, solid=0):
        out = np.empty(self.nx * self.ny)
        if lib().oracle_read_field(self.h, FIELDS[name], solid, _dp(out)) != 0:
            self._raise()
        return out.reshape(self.ny, self.nx)

    def populations(self):
        out = np.empty((9, self.ny, self.nx))
        for q in range(9):
            buf = np.empty(self.nx * self.ny)
            lib().oracle_read_field(self.h, 20 + q, 0, _dp(buf))
            out[q] = buf.reshape(self.ny, self.nx)
        return out

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if lib().oracle_set_populations(self.h, _dp(f)) != 0:
            self._raise()

    def set_refmap(self, solid, X, Y):
        """Prescribe a solid's reference map (absolute coordinates, (ny, nx)
        grids) on its solid and band nodes and relabel its level set."""
        X = np.ascontiguousarray(X, dtype=np.float64)
        Y = np.ascontiguousarray(Y, dtype=np.float64)
        if lib().oracle_set_refmap(self.h, int(solid), _dp(X), _dp(Y)) != 0:
            self._raise()

    def solid_stats(self, solid):
        """(area sum lambda, centroid x, y, mass, momentum x, y, max |det F - 1|,
        mean |det F - 1|, contact force x, y) of one solid."""
        out = np.empty(10)
        if lib().oracle_solid_stats(self.h, solid, _dp(out)) != 0:
            self._raise()
        return out

    def close(self):
        if self.h:
            lib().oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
