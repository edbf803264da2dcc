"""Parity of the 16-bit storage variants (FP32 arithmetic, populations and
half-force stored as FP16 or BF16) with the FP64 oracle.

The stored values are small deviations (f_q - w_q rho_f, the rest population
relative to its SFC rest value) rounded to 2^-11 (FP16) or 2^-8 (BF16)
relative each step; the error bounds below are the FP32 bound of
test_gpu_parity.py with u_32 replaced by the storage unit roundoff u_s and
the random walk of n roundings: fields rho, u and F must satisfy
|err| <= 1e-5 |field|_max + 4 u_s (max|rho_s - rho_f| + |u|_max sqrt(n)) (rho, u),
|err| <= 1e-5 |F|_max + 8 u_s max G + 4 u_s |F|_max (F, which feels the rounded velocity)
and xi - x on the solid and first four layers within 64 u_s |u|_max n.
"""
import json
import os

import numpy as np
import pytest

import scenarios
from parity_util import FLOORS, run_pair

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
    drho = max([abs(s["rho_s"] - sc["rho_f"]) for s in sc["solids"]] + [0.0])
    gmax = max([s["G"] for s in sc["solids"]] + [0.0])
    for n, r in res.items():
        walk = 4 * us * (drho + r["u_max"] * np.sqrt(n))
        for k in ("rho", "u"):
            scale = max(r[k + "_max"], FLOORS[k] * (sc["rho_f"] if k == "rho" else 1.0))
            assert r[k + "_abs"] <= 1e-5 * scale + walk, (n, k, r)
        assert r["F_abs"] <= 1e-5 * r["F_max"] + 8 * us * gmax + 4 * us * r["F_max"], (n, r)
        assert r["xi"] <= 64 * us * max(r["u_max"], 1e-6) * n + 1e-6, (n, r)
