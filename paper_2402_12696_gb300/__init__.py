"""Thin Python binding of the GB300 LBRMT library (C ABI of include/lbrmt.h).

Every step of the time step runs in the CUDA kernels of ``liblbrmt.so``; this
module only marshals arguments.  PyTorch supplies device memory (through the
allocator callbacks of ``lbrmt_config``) and the CUDA stream.  There is no CPU
fallback: importing the library on a machine where ``liblbrmt.so`` is missing
or cannot be loaded raises.

The module-level functions carry the C names (``lbrmt_create``,
``lbrmt_add_solid``, ``lbrmt_step``, ``lbrmt_read_fields``, ...); the
``Simulation`` class builds one simulation from a scenario dict of the
``scenarios`` module.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbrmt.so")

LBRMT_OK = 0
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_NUMERIC", -4: "ERR_OVERFLOW",
          -5: "ERR_EXTRAP", -6: "ERR_TIMEOUT", -7: "ERR_PARAM_RANGE", -8: "ERR_STATE"}
PRECISION = {"fp32": 0, "fp64": 1, "fp16": 2, "bf16": 3}
FIELDS = {"rho": 0, "ux": 1, "uy": 2, "Fx": 3, "Fy": 4, "drho": 5,
          "xi_x": 10, "xi_y": 11, "phi": 12, "detF_dev": 14, "von_mises": 15}
SHAPES = {"disk": 0, "ellipse": 1, "rect": 2}
EXPORTS = ["lbrmt_default_config", "lbrmt_create", "lbrmt_add_solid", "lbrmt_add_solid_shape",
           "lbrmt_batch_add_solid_shape", "lbrmt_init", "lbrmt_step",
           "lbrmt_read_fields", "lbrmt_read_fields_host", "lbrmt_set_populations_host",
           "lbrmt_solid_stats", "lbrmt_solid_stats_async", "lbrmt_total_mass", "lbrmt_sync", "lbrmt_total_mass_noalloc", "lbrmt_active_tiles", "lbrmt_step_timed", "lbrmt_steps_done",
           "lbrmt_num_solids", "lbrmt_last_launch_count", "lbrmt_set_use_graphs", "lbrmt_set_use_tma",
           "lbrmt_uses_tma", "lbrmt_set_overlap", "lbrmt_uses_overlap", "lbrmt_set_rmt_threads", "lbrmt_rmt_threads", "lbrmt_save", "lbrmt_load", "lbrmt_check_bounded_wait",
           "lbrmt_last_error", "lbrmt_destroy", "lbrmt_set_body_force_field", "lbrmt_set_solid_params",
           "lbrmt_reset", "lbrmt_forward_checkpointed", "lbrmt_backward", "lbrmt_set_tile_x", "lbrmt_tile_x",
           "lbrmt_autotune_tile",
           "lbrmt_create_batch", "lbrmt_batch_add_solid", "lbrmt_batch_init", "lbrmt_batch_step",
           "lbrmt_batch_set_overlap", "lbrmt_batch_uses_overlap",
           "lbrmt_batch_step_timed", "lbrmt_batch_sync", "lbrmt_batch_member", "lbrmt_batch_size",
           "lbrmt_batch_tile_x", "lbrmt_batch_tune_log", "lbrmt_batch_steps_done",
           "lbrmt_batch_last_launch_count", "lbrmt_batch_last_error", "lbrmt_destroy_batch"]

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


# columns of lbrmt_solid_stats: area, centroid x, y, mass, momentum x, y, max and mean |det F - 1|, contact force x, y
STATS_COLS = 10


class lbrmt_config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("bc_x", C.c_int), ("bc_y", C.c_int),
                ("tau", C.c_double), ("rho_f", C.c_double), ("lid_u", C.c_double),
                ("eps", C.c_double), ("n_layers", C.c_int), ("eta", C.c_double),
                ("gravity", C.c_double), ("force_kind", C.c_int), ("force_a", C.c_double * 2),
                ("precision", C.c_int), ("max_solids_per_tile", C.c_int), ("rmax", C.c_int),
                ("tile_x", C.c_int), ("deform_margin", C.c_double), ("force_mode", C.c_int),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p)]


class LbrmtError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load():
    """Load liblbrmt.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"liblbrmt.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    p, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
    cfgp = C.POINTER(lbrmt_config)
    L.lbrmt_default_config.argtypes = [cfgp]
    L.lbrmt_default_config.restype = None
    L.lbrmt_create.argtypes = [cfgp, p, C.POINTER(p)]
    L.lbrmt_add_solid.argtypes = [p, i, d, d, d, d, d, C.POINTER(i)]
    L.lbrmt_add_solid_shape.argtypes = [p, i, d, d, d, d, d, d, C.POINTER(i)]
    L.lbrmt_batch_add_solid_shape.argtypes = [p, i, i, d, d, d, d, d, d, C.POINTER(i)]
    L.lbrmt_init.argtypes = [p]
    L.lbrmt_step.argtypes = [p, i]
    L.lbrmt_read_fields.argtypes = [p, i, i, i, p]
    L.lbrmt_read_fields_host.argtypes = [p, i, i, i, p]
    L.lbrmt_set_populations_host.argtypes = [p, p]
    L.lbrmt_solid_stats.argtypes = [p, i, p]
    L.lbrmt_solid_stats_async.argtypes = [p, i, p]
    L.lbrmt_total_mass.argtypes = [p, i, p]
    L.lbrmt_sync.argtypes = [p]
    L.lbrmt_active_tiles.argtypes = [p, i, C.POINTER(ll)]
    L.lbrmt_total_mass_noalloc.argtypes = [p, i, p]
    L.lbrmt_step_timed.argtypes = [p, i, C.POINTER(C.c_float)]
    L.lbrmt_steps_done.argtypes = [p]
    L.lbrmt_steps_done.restype = ll
    L.lbrmt_num_solids.argtypes = [p]
    L.lbrmt_last_launch_count.argtypes = [p]
    L.lbrmt_last_launch_count.restype = ll
    L.lbrmt_set_use_graphs.argtypes = [p, i]
    L.lbrmt_set_use_tma.argtypes = [p, i]
    L.lbrmt_uses_tma.argtypes = [p]
    L.lbrmt_set_overlap.argtypes = [p, i]
    L.lbrmt_uses_overlap.argtypes = [p]
    L.lbrmt_set_rmt_threads.argtypes = [p, i]
    L.lbrmt_rmt_threads.argtypes = [p]
    L.lbrmt_last_error.argtypes = [p]
    L.lbrmt_last_error.restype = C.c_char_p
    L.lbrmt_destroy.argtypes = [p]
    L.lbrmt_destroy.restype = None
    L.lbrmt_set_body_force_field.argtypes = [p, i, p]
    L.lbrmt_set_solid_params.argtypes = [p, i, d, d]
    L.lbrmt_reset.argtypes = [p]
    L.lbrmt_save.argtypes = [p, p, C.POINTER(C.c_size_t)]
    L.lbrmt_load.argtypes = [p, p, C.c_size_t]
    L.lbrmt_check_bounded_wait.argtypes = [p]
    L.lbrmt_set_tile_x.argtypes = [p, i]
    L.lbrmt_tile_x.argtypes = [p]
    L.lbrmt_autotune_tile.argtypes = [p, i, C.POINTER(i), C.POINTER(i), p]
    L.lbrmt_forward_checkpointed.argtypes = [p, i, i, p]
    L.lbrmt_backward.argtypes = [p, p, p, p, p, p]
    L.lbrmt_create_batch.argtypes = [cfgp, i, p, C.POINTER(p)]
    L.lbrmt_batch_add_solid.argtypes = [p, i, i, d, d, d, d, d, C.POINTER(i)]
    L.lbrmt_batch_init.argtypes = [p, i]
    L.lbrmt_batch_step.argtypes = [p, i]
    L.lbrmt_batch_step_timed.argtypes = [p, i, C.POINTER(C.c_float)]
    L.lbrmt_batch_sync.argtypes = [p]
    L.lbrmt_batch_member.argtypes = [p, i, C.POINTER(p)]
    L.lbrmt_batch_size.argtypes = [p]
    L.lbrmt_batch_tile_x.argtypes = [p, i]
    L.lbrmt_batch_tune_log.argtypes = [p, p, p, p, p, i]
    L.lbrmt_batch_steps_done.argtypes = [p]
    L.lbrmt_batch_set_overlap.argtypes = [p, i]
    L.lbrmt_batch_uses_overlap.argtypes = [p]
    L.lbrmt_batch_steps_done.restype = ll
    L.lbrmt_batch_last_launch_count.argtypes = [p]
    L.lbrmt_batch_last_launch_count.restype = ll
    L.lbrmt_batch_last_error.argtypes = [p]
    L.lbrmt_batch_last_error.restype = C.c_char_p
    L.lbrmt_destroy_batch.argtypes = [p]
    L.lbrmt_destroy_batch.restype = None
    _lib = L
    return L


def _check(h, st):
    if st != LBRMT_OK:
        msg = load().lbrmt_last_error(h).decode() if h else ""
        raise LbrmtError(st, msg)


# ---------------------------------------------------------------------------
# C-named wrappers (argument marshalling only)
# ---------------------------------------------------------------------------

def lbrmt_default_config():
    cfg = lbrmt_config()
    load().lbrmt_default_config(C.byref(cfg))
    return cfg


def lbrmt_create(cfg, stream_ptr):
    h = C.c_void_p()
    _check(None, load().lbrmt_create(C.byref(cfg), C.c_void_p(stream_ptr), C.byref(h)))
    return h


def lbrmt_add_solid(h, shape, cx, cy, radius, rho_s, G):
    sid = C.c_int()
    _check(h, load().lbrmt_add_solid(h, shape, cx, cy, radius, rho_s, G, C.byref(sid)))
    return sid.value


def lbrmt_add_solid_shape(h, shape, cx, cy, a, b, rho_s, G):
    sid = C.c_int()
    _check(h, load().lbrmt_add_solid_shape(h, shape, cx, cy, a, b, rho_s, G, C.byref(sid)))
    return sid.value


def _solid_geometry(s):
    """(shape id, a, b) of a scenario solid dict (disks: a = b = r)."""
    shape = SHAPES[s.get("shape", "disk")]
    return (shape, s["r"], s["r"]) if shape == 0 else (shape, s["a"], s["b"])


def lbrmt_init(h):
    _check(h, load().lbrmt_init(h))


def lbrmt_step(h, nsteps):
    _check(h, load().lbrmt_step(h, int(nsteps)))


def lbrmt_read_fields(h, sim_index, field, solid_id, dev_ptr):
    _check(h, load().lbrmt_read_fields(h, sim_index, field, solid_id, C.c_void_p(dev_ptr)))


def lbrmt_read_fields_host(h, sim_index, field, solid_id, host_ptr):
    _check(h, load().lbrmt_read_fields_host(h, sim_index, field, solid_id, C.c_void_p(host_ptr)))


def lbrmt_set_populations_host(h, host_ptr):
    _check(h, load().lbrmt_set_populations_host(h, C.c_void_p(host_ptr)))


def lbrmt_solid_stats(h, sim_index, host_ptr):
    _check(h, load().lbrmt_solid_stats(h, sim_index, C.c_void_p(host_ptr)))


def lbrmt_solid_stats_async(h, sim_index, host_ptr):
    _check(h, load().lbrmt_solid_stats_async(h, sim_index, C.c_void_p(host_ptr)))


def lbrmt_total_mass(h, sim_index, host_ptr):
    _check(h, load().lbrmt_total_mass(h, sim_index, C.c_void_p(host_ptr)))


def lbrmt_sync(h):
    _check(h, load().lbrmt_sync(h))


def lbrmt_total_mass_noalloc(h, sim_index, dev_ptr):
    _check(h, load().lbrmt_total_mass_noalloc(h, sim_index, C.c_void_p(dev_ptr)))


def lbrmt_active_tiles(h, sim_index):
    n = C.c_longlong()
    _check(h, load().lbrmt_active_tiles(h, sim_index, C.byref(n)))
    return n.value


def lbrmt_step_timed(h, nsteps):
    ms = (C.c_float * 3)()
    _check(h, load().lbrmt_step_timed(h, int(nsteps), ms))
    return [ms[0], ms[1], ms[2]]


def lbrmt_destroy(h):
    load().lbrmt_destroy(h)


def lbrmt_set_body_force_field(h, sim_index, dev_ptr):
    _check(h, load().lbrmt_set_body_force_field(h, sim_index, C.c_void_p(dev_ptr)))


def lbrmt_set_solid_params(h, solid_id, rho_s, G):
    _check(h, load().lbrmt_set_solid_params(h, solid_id, rho_s, G))


def lbrmt_reset(h):
    _check(h, load().lbrmt_reset(h))


def lbrmt_save(h, dev_ptr=None, nbytes=0):
    """Checkpoint size (dev_ptr None), or write the checkpoint into nbytes of device memory; the bytes."""
    n = C.c_size_t(nbytes)
    _check(h, load().lbrmt_save(h, dev_ptr, C.byref(n)))
    return n.value


def lbrmt_load(h, dev_ptr, nbytes):
    _check(h, load().lbrmt_load(h, dev_ptr, nbytes))


def lbrmt_forward_checkpointed(h, nsteps, checkpoint_every, host_ptr):
    _check(h, load().lbrmt_forward_checkpointed(h, int(nsteps), int(checkpoint_every), C.c_void_p(host_ptr)))


def lbrmt_backward(h, dLdc_ptr, dG_ptr, dratio_ptr, dbody_dev_ptr, df0_dev_ptr=0):
    _check(h, load().lbrmt_backward(h, C.c_void_p(dLdc_ptr), C.c_void_p(dG_ptr), C.c_void_p(dratio_ptr),
                                    C.c_void_p(dbody_dev_ptr), C.c_void_p(df0_dev_ptr)))


def _bcheck(b, st):
    if st != LBRMT_OK:
        msg = load().lbrmt_batch_last_error(b).decode() if b else ""
        raise LbrmtError(st, msg)


def lbrmt_create_batch(cfgs, stream_ptr):
    arr = (lbrmt_config * len(cfgs))(*cfgs)
    b = C.c_void_p()
    _bcheck(None, load().lbrmt_create_batch(arr, len(cfgs), C.c_void_p(stream_ptr), C.byref(b)))
    return b


def lbrmt_batch_add_solid(b, sim_index, shape, cx, cy, radius, rho_s, G):
    sid = C.c_int()
    _bcheck(b, load().lbrmt_batch_add_solid(b, sim_index, shape, cx, cy, radius, rho_s, G, C.byref(sid)))
    return sid.value


def lbrmt_batch_add_solid_shape(b, sim_index, shape, cx, cy, a, bb, rho_s, G):
    sid = C.c_int()
    _bcheck(b, load().lbrmt_batch_add_solid_shape(b, sim_index, shape, cx, cy, a, bb, rho_s, G, C.byref(sid)))
    return sid.value


def lbrmt_batch_init(b, autotune_steps):
    _bcheck(b, load().lbrmt_batch_init(b, int(autotune_steps)))


def lbrmt_batch_step(b, nsteps):
    _bcheck(b, load().lbrmt_batch_step(b, int(nsteps)))


def lbrmt_batch_step_timed(b, nsteps):
    ms = (C.c_float * 3)()
    _bcheck(b, load().lbrmt_batch_step_timed(b, int(nsteps), ms))
    return [ms[0], ms[1], ms[2]]


def lbrmt_batch_sync(b):
    _bcheck(b, load().lbrmt_batch_sync(b))


def lbrmt_batch_member(b, sim_index):
    h = C.c_void_p()
    _bcheck(b, load().lbrmt_batch_member(b, sim_index, C.byref(h)))
    return h


def lbrmt_batch_tune_log(b):
    L = load()
    n = L.lbrmt_batch_tune_log(b, None, None, None, None, 0)
    nx, ny, tx = (C.c_int * max(n, 1))(), (C.c_int * max(n, 1))(), (C.c_int * max(n, 1))()
    ms = (C.c_double * max(n, 1))()
    L.lbrmt_batch_tune_log(b, nx, ny, tx, ms, n)
    return [(nx[k], ny[k], tx[k], ms[k]) for k in range(n)]


def lbrmt_destroy_batch(b):
    load().lbrmt_destroy_batch(b)


# ---------------------------------------------------------------------------
# Convenience class
# ---------------------------------------------------------------------------

class _TorchAllocator:
    """Routes the library's device allocations to the PyTorch caching allocator."""

    def __init__(self, torch, device, stream):
        self.torch, self.device, self.stream = torch, device, stream
        self.live = {}
        self.n_alloc = 0
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            with self.torch.cuda.stream(self.stream):
                t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        ptr = t.data_ptr()
        self.live[ptr] = t
        self.n_alloc += 1
        return ptr

    def _free(self, ptr, ctx):
        self.live.pop(ptr, None)


def scenario_config(sc, precision="fp32", max_solids_per_tile=8, rmax=11, tile_x=32):
    """lbrmt_config of a scenario dict (without allocator callbacks)."""
    cfg = lbrmt_default_config()
    cfg.nx, cfg.ny = sc["nx"], sc["ny"]
    cfg.bc_x, cfg.bc_y = sc["wall_x"], sc["wall_y"]
    cfg.tau, cfg.rho_f, cfg.lid_u = sc["tau"], sc["rho_f"], sc["lid_u"]
    cfg.eps, cfg.n_layers, cfg.eta = sc["eps"], sc["n_layers"], sc["eta"]
    cfg.gravity, cfg.force_kind = sc["gravity"], sc["force_kind"]
    fa = sc.get("force_a", [0.0, 0.0])
    cfg.force_a[0], cfg.force_a[1] = fa[0], fa[1]
    cfg.precision = PRECISION[precision]
    cfg.max_solids_per_tile = max_solids_per_tile
    cfg.rmax = rmax
    cfg.tile_x = tile_x
    cfg.deform_margin = sc.get("deform_margin", 0.25)
    cfg.force_mode = sc.get("force_mode", 0)
    return cfg


class Simulation:
    """One LBRMT simulation on a CUDA device, built from a scenario dict."""

    def __init__(self, sc, precision="fp32", device="cuda:0", stream=None, use_graphs=True,
                 max_solids_per_tile=8, rmax=11, tile_x=32, use_tma=True, overlap=True,
                 rmt_threads=0):
        import torch
        self.torch = torch
        self.sc = sc
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.nx, self.ny = sc["nx"], sc["ny"]
        self.nsolids = len(sc["solids"])
        cfg = scenario_config(sc, precision, max_solids_per_tile, rmax, tile_x)
        self._alloc = _TorchAllocator(torch, self.device, self.stream)
        cfg.alloc = self._alloc.alloc_cb
        cfg.free = self._alloc.free_cb
        self._cfg = cfg
        with torch.cuda.device(self.device):
            self.h = lbrmt_create(cfg, self.stream.cuda_stream)
            load().lbrmt_set_use_graphs(self.h, int(bool(use_graphs)))
            load().lbrmt_set_use_tma(self.h, int(bool(use_tma)))
            _check(self.h, load().lbrmt_set_overlap(self.h, int(bool(overlap))))
            _check(self.h, load().lbrmt_set_rmt_threads(self.h, int(rmt_threads)))
            for s in sc["solids"]:
                shape, a, b = _solid_geometry(s)
                lbrmt_add_solid_shape(self.h, shape, s["x"], s["y"], a, b, s["rho_s"], s["G"])
            if sc["force_kind"] == 3:
                self.set_body_force_field(sc["body_field"])

    def set_body_force_field(self, field):
        """Body force field (2, ny, nx) of a force_kind 3 scenario (array or tensor)."""
        torch = self.torch
        t = torch.as_tensor(field, dtype=torch.float64).reshape(2, self.ny, self.nx)
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            t = t.to(self.device, non_blocking=False).contiguous()
            lbrmt_set_body_force_field(self.h, 0, t.data_ptr())
            self._bfield = t  # kept alive until the copy kernel has run

    def set_solid_params(self, solid, rho_s, G):
        """Change a solid's density and shear modulus (lbrmt_set_solid_params; back to the initial state)."""
        with self.torch.cuda.device(self.device):
            lbrmt_set_solid_params(self.h, solid, rho_s, G)

    def reset(self):
        """Return to the initial state with the current parameters (lbrmt_reset)."""
        with self.torch.cuda.device(self.device):
            lbrmt_reset(self.h)

    def save(self):
        """Checkpoint of the current state (lbrmt_save) in a new uint8 device tensor."""
        torch = self.torch
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            n = lbrmt_save(self.h)
            blob = torch.empty(n, dtype=torch.uint8, device=self.device)  # ordered on the sim's stream
            lbrmt_save(self.h, blob.data_ptr(), n)
        return blob

    def load(self, blob):
        """Restore a checkpoint made by save() (a uint8 tensor, moved to this device)."""
        torch = self.torch
        blob = blob.to(self.device).contiguous()
        with torch.cuda.device(self.device):
            torch.cuda.current_stream(self.device).synchronize()  # the blob's producers are done
            lbrmt_load(self.h, blob.data_ptr(), blob.numel())

    @property
    def tile_x(self):
        """Registry / lattice Boltzmann tile width in use (lbrmt_tile_x)."""
        return load().lbrmt_tile_x(self.h)

    def set_tile_x(self, tx):
        """Registry / lattice Boltzmann tile width 16, 32, 64 or 128 (lbrmt_set_tile_x; back to the initial state)."""
        with self.torch.cuda.device(self.device):
            _check(self.h, load().lbrmt_set_tile_x(self.h, int(tx)))

    def autotune_tile(self, steps=20):
        """Time each tile shape with staged and direct LB loads; keep the fastest
        (state back to initial).  Returns ((tile_x, staged), {(tile_x, staged): ms})."""
        best, tma = C.c_int(), C.c_int()
        ms = (C.c_double * 8)()
        with self.torch.cuda.device(self.device):
            _check(self.h, load().lbrmt_autotune_tile(self.h, int(steps), C.byref(best), C.byref(tma), ms))
        table = {(tx, st): ms[2 * k + (0 if st else 1)] for k, tx in enumerate((16, 32, 64, 128)) for st in (True, False)}
        return (best.value, bool(tma.value)), table

    # -- time stepping ------------------------------------------------------
    def init(self):
        """Initialise (Algorithm 1, initialisation; lbrmt_init)."""
        with self.torch.cuda.device(self.device):
            lbrmt_init(self.h)

    def step(self, n=1):
        """Advance n steps, asynchronously on the simulation's stream (lbrmt_step)."""
        with self.torch.cuda.device(self.device):
            lbrmt_step(self.h, n)

    def sync(self):
        """Wait for the stream and raise on a device error flag (lbrmt_sync)."""
        lbrmt_sync(self.h)

    def active_tiles(self):
        """Registry tiles the last step registered for the force kernel (lbrmt_active_tiles)."""
        return lbrmt_active_tiles(self.h, 0)

    def step_timed(self, n):
        """Run n steps with per-kernel CUDA events; mean ms of [K2, K3, K1]."""
        with self.torch.cuda.device(self.device):
            return lbrmt_step_timed(self.h, n)

    @property
    def steps_done(self):
        """Steps taken since the initial state (lbrmt_steps_done)."""
        return load().lbrmt_steps_done(self.h)

    @property
    def uses_tma(self):
        """Whether the lattice Boltzmann kernel stages tiles with tensor-memory copies (lbrmt_uses_tma)."""
        return bool(load().lbrmt_uses_tma(self.h))

    def set_overlap(self, enable):
        """Overlapped (True) or sequential (False) step schedule (lbrmt_set_overlap)."""
        _check(self.h, load().lbrmt_set_overlap(self.h, int(bool(enable))))

    @property
    def uses_overlap(self):
        """Whether steps run the overlapped schedule (lbrmt_uses_overlap)."""
        return bool(load().lbrmt_uses_overlap(self.h))

    def set_rmt_threads(self, threads):
        """CTA width of the reference-map kernel: 0 (chosen), 256 or 1024 (lbrmt_set_rmt_threads)."""
        _check(self.h, load().lbrmt_set_rmt_threads(self.h, int(threads)))

    @property
    def rmt_threads(self):
        """CTA width of the reference-map kernel in use (lbrmt_rmt_threads)."""
        return load().lbrmt_rmt_threads(self.h)

    @property
    def last_launch_count(self):
        """Kernel launches of the last step call (lbrmt_last_launch_count)."""
        return load().lbrmt_last_launch_count(self.h)

    # -- adjoint --------------------------------------------------------------
    def forward_checkpointed(self, nsteps, checkpoint_every):
        """Run from the initial state; the solids' final centroids (S, 2)."""
        out = np.zeros((max(self.nsolids, 1), 2))
        with self.torch.cuda.device(self.device):
            lbrmt_forward_checkpointed(self.h, nsteps, checkpoint_every, out.ctypes.data)
        return out[: self.nsolids]

    def backward(self, dLdc, body=False, f0=False):
        """Gradients through the last forward_checkpointed run for dL/dc (S, 2):
        (dL/dG (S,), dL/d(rho_s/rho_f) (S,), dL/df body field (2, ny, nx) device
        tensor or None), and with ``f0`` also dL/df_q(t=0) (9, ny, nx)."""
        torch = self.torch
        g = np.ascontiguousarray(dLdc, dtype=np.float64).reshape(self.nsolids, 2)
        dG = np.zeros(max(self.nsolids, 1))
        dr = np.zeros(max(self.nsolids, 1))
        db = None
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            if body:
                db = torch.zeros((2, self.ny, self.nx), dtype=torch.float64, device=self.device)
            d0 = torch.zeros((9, self.ny, self.nx), dtype=torch.float64, device=self.device) if f0 else None
            lbrmt_backward(self.h, g.ctypes.data, dG.ctypes.data, dr.ctypes.data, db.data_ptr() if body else 0,
                           d0.data_ptr() if f0 else 0)
        if f0:
            return dG[: self.nsolids], dr[: self.nsolids], db, d0
        return dG[: self.nsolids], dr[: self.nsolids], db

    # -- outputs ------------------------------------------------------------
    def field(self, name, solid=0):
        """Device tensor (float64, [ny, nx]) of one field."""
        torch = self.torch
        with torch.cuda.device(self.device), torch.cuda.stream(self.stream):
            out = torch.empty(self.ny * self.nx, dtype=torch.float64, device=self.device)
            fid = FIELDS[name] if isinstance(name, str) else int(name)
            lbrmt_read_fields(self.h, 0, fid, solid, out.data_ptr())
        return out.view(self.ny, self.nx)

    def field_host(self, name, solid=0):
        """One field (a FIELDS name or id; solid selects the solid for per-solid fields) as an (ny, nx) array."""
        out = np.empty(self.ny * self.nx, dtype=np.float64)
        fid = FIELDS[name] if isinstance(name, str) else int(name)
        with self.torch.cuda.device(self.device):
            lbrmt_read_fields_host(self.h, 0, fid, solid, out.ctypes.data)
        return out.reshape(self.ny, self.nx)

    def populations_host(self):
        """The nine populations f_q as a (9, ny, nx) array."""
        return np.stack([self.field_host(20 + q) for q in range(9)])

    def set_populations_host(self, f):
        """Overwrite the populations from a (9, ny, nx) array (lbrmt_set_populations_host)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        with self.torch.cuda.device(self.device):
            lbrmt_set_populations_host(self.h, f.ctypes.data)

    def solid_stats(self):
        """Per-solid FP64 statistics of the current state, (S, 10) (lbrmt_solid_stats)."""
        out = np.zeros((max(self.nsolids, 1), STATS_COLS))
        with self.torch.cuda.device(self.device):
            lbrmt_solid_stats(self.h, 0, out.ctypes.data)
        return out[: self.nsolids]

    def total_mass(self):
        """Total mass sum rho of the current state (lbrmt_total_mass)."""
        out = np.zeros(1)
        with self.torch.cuda.device(self.device):
            lbrmt_total_mass(self.h, 0, out.ctypes.data)
        return float(out[0])

    def close(self):
        """Free the simulation and its device memory (lbrmt_destroy)."""
        if getattr(self, "h", None):
            lbrmt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Member(Simulation):
    """Borrowed view of one member of a Batch (reads only; the batch steps it)."""

    def __init__(self, batch, k):  # noqa: D401  (no Simulation.__init__: the batch owns the handle)
        self.torch, self.device, self.stream = batch.torch, batch.device, batch.stream
        self.sc = batch.scs[k]
        self.nx, self.ny = self.sc["nx"], self.sc["ny"]
        self.nsolids = len(self.sc["solids"])
        self.h = lbrmt_batch_member(batch.b, k)
        self._batch = batch

    def close(self):
        """Members are freed with their batch."""
        self.h = None


class Batch:
    """Many independent LBRMT simulations advanced by one persistent launch per
    kernel of the step (lbrmt_create_batch).  ``tile_x`` is one value or one per
    member; ``autotune_steps`` > 0 lets the library choose each grid size's tile
    shape by timing batch steps."""

    def __init__(self, scs, precision="fp32", device="cuda:0", stream=None, tile_x=32, autotune_steps=0,
                 max_solids_per_tile=8, rmax=11, overlap=True):
        import torch
        self.torch = torch
        self.scs = list(scs)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        txs = list(tile_x) if isinstance(tile_x, (list, tuple)) else [tile_x] * len(self.scs)
        self._alloc = _TorchAllocator(torch, self.device, self.stream)
        cfgs = []
        for sc, tx in zip(self.scs, txs):
            cfg = scenario_config(sc, precision, max_solids_per_tile, rmax, tx)
            cfg.alloc = self._alloc.alloc_cb
            cfg.free = self._alloc.free_cb
            cfgs.append(cfg)
        self._cfgs = cfgs
        with torch.cuda.device(self.device):
            self.b = lbrmt_create_batch(cfgs, self.stream.cuda_stream)
            _bcheck(self.b, load().lbrmt_batch_set_overlap(self.b, int(bool(overlap))))
            for k, sc in enumerate(self.scs):
                for s in sc["solids"]:
                    shape, a, bb = _solid_geometry(s)
                    lbrmt_batch_add_solid_shape(self.b, k, shape, s["x"], s["y"], a, bb, s["rho_s"], s["G"])
            lbrmt_batch_init(self.b, autotune_steps)
        self.members = [_Member(self, k) for k in range(len(self.scs))]

    def __len__(self):
        return len(self.scs)

    def __getitem__(self, k):
        return self.members[k]

    def step(self, n=1):
        """Advance every member n steps, asynchronously (lbrmt_batch_step)."""
        with self.torch.cuda.device(self.device):
            lbrmt_batch_step(self.b, n)

    def step_timed(self, n):
        """Mean ms of the three batched kernels over n sequential steps (lbrmt_batch_step_timed)."""
        with self.torch.cuda.device(self.device):
            return lbrmt_batch_step_timed(self.b, n)

    def set_overlap(self, enable):
        """Overlapped (True) or sequential (False) batch step (lbrmt_batch_set_overlap)."""
        _bcheck(self.b, load().lbrmt_batch_set_overlap(self.b, int(bool(enable))))

    @property
    def uses_overlap(self):
        """Whether batch steps run the overlapped schedule (lbrmt_batch_uses_overlap)."""
        return bool(load().lbrmt_batch_uses_overlap(self.b))

    def sync(self):
        """Wait for the stream and raise on any member's device error flag (lbrmt_batch_sync)."""
        lbrmt_batch_sync(self.b)

    def tile_x(self, k):
        """Tile width in use by member k (lbrmt_batch_tile_x)."""
        return load().lbrmt_batch_tile_x(self.b, k)

    def tune_log(self):
        """The autotuner's trials as (nx, ny, tile_x, ms per batch step) tuples (lbrmt_batch_tune_log)."""
        return lbrmt_batch_tune_log(self.b)

    @property
    def steps_done(self):
        """Batch steps taken (lbrmt_batch_steps_done)."""
        return load().lbrmt_batch_steps_done(self.b)

    @property
    def last_launch_count(self):
        """Kernel launches of the last batch step call (lbrmt_batch_last_launch_count)."""
        return load().lbrmt_batch_last_launch_count(self.b)

    @property
    def nodes(self):
        """Total grid nodes over the members."""
        return sum(sc["nx"] * sc["ny"] for sc in self.scs)

    def close(self):
        """Free the batch, its members and their device memory (lbrmt_destroy_batch)."""
        if getattr(self, "b", None):
            for m in self.members:
                m.close()
            lbrmt_destroy_batch(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_function():
    import torch

    class LBRMTFunction(torch.autograd.Function):
        """Final solid centroids c (S, 2) of a Simulation as a differentiable
        function of the shear moduli G (S,), the density ratios rho_s / rho_f
        (S,) and the body force field (2, ny, nx) (force_kind 3 scenarios; may
        be None).  ``apply(G, ratio, body, sim, nsteps, checkpoint_every)``;
        the backward pass is the library's adjoint sweep (lbrmt_backward)."""

        @staticmethod
        def forward(ctx, G, ratio, body, sim, nsteps, checkpoint_every):
            """Checkpointed forward run (lbrmt_forward_checkpointed): the solids' final centroids."""
            rho_f = sim.sc["rho_f"]
            for k in range(sim.nsolids):
                sim.set_solid_params(k, float(ratio[k]) * rho_f, float(G[k]))
            if body is not None:
                sim.set_body_force_field(body.detach())
            c = sim.forward_checkpointed(nsteps, checkpoint_every)
            ctx.sim = sim
            ctx.has_body = body is not None
            ctx.body_device = body.device if body is not None else None
            return torch.as_tensor(c, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_c):
            """Reverse run (lbrmt_backward): gradients for G, the density ratio and the body-force field."""
            dG, dr, db = ctx.sim.backward(grad_c.detach().cpu().numpy(), body=ctx.has_body)
            gb = db.to(ctx.body_device) if ctx.has_body else None
            return (torch.as_tensor(dG, dtype=torch.float64), torch.as_tensor(dr, dtype=torch.float64), gb,
                    None, None, None)

    return LBRMTFunction


def __getattr__(name):
    if name == "LBRMTFunction":
        fn = _make_function()
        globals()["LBRMTFunction"] = fn
        return fn
    raise AttributeError(name)
