"""Parity of the 16-bit storage variants (FP32 arithmetic, populations and
half-force stored as FP16 or BF16) with the FP64 oracle.

The stored values are small deviations (f_q - w_q rho_f, the rest population
relative to its SFC rest value, each plane scaled by its own power of two)
rounded to the storage unit roundoff u_s (2^-11 for FP16, 2^-8 for BF16) at
every step; everything else (Delta rho, the reference map, the stresses) is
held as in the FP32 variant.  The bound is relative L-infinity per field, as
for FP32, in units of u_s:
  rho - rho_f, u : 4 u_s      F : 16 u_s (the stresses follow the rounded
  xi - x (solid and first 4 layers): 2 u_s, whole band 4 u_s     velocity)
measured over 1, 10 and 100 steps (4 at 4096^2): u, rho ~1.5 u_s, F up to
~7 u_s, xi below 0.5 u_s.
"""
import json
import os

import numpy as np
import pytest

import scenarios
from parity_util import run_pair

pytestmark = pytest.mark.gpu

US = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
OUT = os.environ.get("LBRMT_PARITY_LOG", "")


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_12696_gb300 import build
    build.build()


CASES = {
    "ldc_disk_64": scenarios.ldc_disk_64,
    "settling_small_0": lambda: scenarios.settling_small(0),
    "mixing_small_1": lambda: scenarios.mixing_small(1),
    "contact_pair": lambda: scenarios.contact_pair(gap=0.8, nx=96, ny=64),
    # a per-node body force (the half-force term rebuilt from the stored density
    # with the field), the conservative force mode, and non-disk shapes
    "ldc_body_field_64": lambda: scenarios.adjoint_ldc(64, r=12, body=scenarios.smooth_body_field(0, 64, amp=1e-4)),
    "settling_small_0_conservative": lambda: dict(scenarios.settling_small(0), force_mode=1),
    "shapes_small_0": lambda: scenarios.shapes_small(0),
}


def _log(name, res):
    if OUT:
        with open(OUT, "a") as f:
            f.write(json.dumps({"case": name, "res": {str(k): v for k, v in res.items()}}) + "\n")


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("case", list(CASES))
def test_half_storage_parity(case, prec):
    sc = CASES[case]()
    res = run_pair(sc, prec, [1, 10, 100])
    _log(f"{case}/{prec}", res)
    _check_half(res, prec, sc)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_half_storage_full_size_mixing(prec):
    # The 4096^2 mixing workload (1024 disks, seed 0) with 16-bit storage in the
    # launch configuration of the benchmark (16x16 tiles, direct loads,
    # overlapped schedule), 4 steps against the FP64 oracle: every node of the
    # grid fields and xi on 16 sampled solids, to the bounds above.
    import oracle
    import paper_2402_12696_gb300 as pkg
    from parity_util import compare
    sc = scenarios.mixing_4096(0)
    sim = pkg.Simulation(sc, precision=prec, tile_x=16, use_tma=False)
    ref = oracle.Oracle(sc)
    sim.step(4)
    ref.step(4)
    sol = sc["solids"]
    picks = sorted(set(sorted(range(len(sol)), key=lambda k: -sol[k]["r"])[:8] +
                       list(np.random.default_rng(11).choice(len(sol), 8, replace=False))))
    res = {4: compare(sim, ref, sc, solids=picks)}
    _log(f"mixing_4096_full/{prec}", res)
    _check_half(res, prec, sc)
    sim.close()
    ref.close()


def _check_half(res, prec, sc):
    us = US[prec]
    # Density floor of the comparison: next to a moving lid three stored
    # populations carry the bounce-back term 6 w rho u_w = rho u_w / 6 (w = 1/36),
    # whose 16-bit rounding alone moves rho by up to rho_f u_w / 2 u_s; a density
    # deviation smaller than that (the first step of a driven cavity) is
    # compared against it, as FP32's floor of 1e-4 rho_f (the same effect).
    rf = sc["rho_f"]
    floor = max(1e-4 * rf, 0.5 * abs(sc.get("lid_u", 0.0)) * rf)
    for n, r in res.items():
        for k, c in (("u", 4), ("F", 16), ("xi", 2), ("xi_band", 4), ("drho", 4)):
            assert r[k] <= c * us, (n, k, r[k], c * us, r)
        rho = r["rho_abs"] / max(r["rho_max"], floor)
        assert rho <= 4 * us, (n, "rho", rho, 4 * us, r)
        assert r["label_mismatch"] == 0, (n, r)
