"""The C-ABI library builds, loads and exports every entry point that
include/lbrmt.h declares; argument checks that need no GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(lbrmt_[a-z_0-9]+)\s*\(", src)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def lib():
    from paper_2402_12696_gb300 import build
    build.build()
    import paper_2402_12696_gb300 as pkg
    return pkg.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    import paper_2402_12696_gb300 as pkg
    assert set(pkg.EXPORTS) <= set(names)


def test_config_struct_layout_matches_header(lib):
    import paper_2402_12696_gb300 as pkg
    cfg = pkg.lbrmt_default_config()
    assert cfg.eps == 1.5 and cfg.n_layers == 11 and cfg.rho_f == 1.0 and cfg.rmax == 11
    assert cfg.max_solids_per_tile == 8 and cfg.precision == 0


def test_create_rejects_bad_parameters_without_touching_the_gpu(lib):
    import paper_2402_12696_gb300 as pkg
    cfg = pkg.lbrmt_default_config()
    h = C.c_void_p()
    cfg.tau = 0.5          # Appendix A: 1/2 < tau <= 1
    assert lib.lbrmt_create(C.byref(cfg), None, C.byref(h)) == -7
    cfg.tau = 1.2
    assert lib.lbrmt_create(C.byref(cfg), None, C.byref(h)) == -7
    cfg.tau = 0.8
    cfg.nx = 4
    assert lib.lbrmt_create(C.byref(cfg), None, C.byref(h)) == -1
    cfg.nx = 64
    cfg.lid_u = 0.05       # a lid needs walls in y
    assert lib.lbrmt_create(C.byref(cfg), None, C.byref(h)) == -1
    cfg.bc_y = 1
    cfg.lid_u = 0.3        # Ma* = 0.52 > 0.3
    assert lib.lbrmt_create(C.byref(cfg), None, C.byref(h)) == -7
    cfg.lid_u = 0.0
    cfg.max_solids_per_tile = 9
    assert lib.lbrmt_create(C.byref(cfg), None, C.byref(h)) == -1
    assert not h.value


def test_knobs_reject_a_null_handle_without_touching_the_gpu(lib):
    assert lib.lbrmt_set_rmt_threads(None, 128) == -1
    assert lib.lbrmt_rmt_threads(None) == 0
    assert lib.lbrmt_set_overlap(None, 1) == -1
    assert lib.lbrmt_uses_overlap(None) == 0
    n = C.c_size_t(0)
    assert lib.lbrmt_save(None, None, C.byref(n)) == -1
    assert lib.lbrmt_load(None, None, 0) == -1


def test_product_path_does_not_reference_the_oracle():
    pkg_dir = os.path.join(ROOT, "paper_2402_12696_gb300")
    for dirpath, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.lower(), f
