"""Host logic of bench.py that runs without a GPU."""
import os
import sys

import pytest

import scenarios

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_oracle_timing_runs_in_segments_from_the_initial_state(monkeypatch):
    # The mixing workload leaves the method's stable range after ~450 steps,
    # so the oracle's timed steps run in segments of at most SEG_STEPS, each
    # from a fresh initial state after a few untimed steps.
    import bench
    import oracle
    made, stepped = [], []

    class Counting(oracle.Oracle):
        def __init__(self, sc):
            super().__init__(sc)
            made.append(self)

        def step(self, n=1):
            stepped.append((len(made), n))
            return super().step(n)

    monkeypatch.setattr(oracle, "Oracle", Counting)
    monkeypatch.setattr(bench, "SEG_STEPS", 397)  # 3 untimed + up to 397 timed = 400 per segment
    sc = scenarios.fluid_only(16, 16, 0, 0, 0.7)
    value, dt, cores = bench.time_oracle(sc, 900, 10)
    assert len(made) == 3
    assert stepped == [(1, 3), (1, 397), (2, 3), (2, 397), (3, 3), (3, 106)]
    assert value > 0 and dt > 0 and cores >= 1


def test_k1_source_hash_covers_only_the_lattice_boltzmann_kernel():
    import bench
    src = open(os.path.join(ROOT, "paper_2402_12696_gb300", "csrc", "lbrmt_kernels.cuh")).read()
    h = bench.k1_source_sha1(src)
    # an edit outside the K1 section leaves the hash, one inside changes it
    assert bench.k1_source_sha1(src.replace("// K2: reference-map advection", "// K2:  reference-map advection")) == h
    i = src.index("// K1: fused moments")
    j = src.index("lb_step_kernel", i)
    assert bench.k1_source_sha1(src[:j] + " " + src[j:]) != h


def test_precision_error_record_round_trip(tmp_path, monkeypatch):
    # The per-precision errors of the full-size parity run reach the bench line
    # through the committed record, and only while the kernels' source hash
    # still matches the one the record was taken on.
    import json
    import bench
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import record_precision_errors as rec
    log = tmp_path / "parity.jsonl"
    lines = [{"case": "mixing_4096_full/fp32", "res": {"4": {"rho": 3e-11, "u": 5e-7, "F": 1e-7, "xi": 7e-11,
                                                            "label_mismatch": 0, "u_abs": 1.0}}},
             {"case": "mixing_4096_full/fp16", "res": {"4": {"rho": 5e-8, "u": 5e-4, "F": 9e-5}}},
             {"case": "ldc_disk_64/fp32", "res": {"1": {"rho": 1.0}}}]
    log.write_text("\n".join(json.dumps(x) for x in lines) + "\n")
    out = tmp_path / "profiles" / "precision_errors_mixing4096.json"
    out.parent.mkdir()
    r = rec.main(str(log), str(out))
    assert sorted(r["errors"]) == ["fp16", "fp32"]
    assert r["errors"]["fp32"] == {"rho": 3e-11, "u": 5e-7, "F": 1e-7, "xi": 7e-11, "label_mismatch": 0}
    # bench reads the record relative to its root: point it at a copy of the tree's kernels
    csrc = tmp_path / "paper_2402_12696_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = open(os.path.join(ROOT, "paper_2402_12696_gb300", "csrc", "lbrmt_kernels.cuh")).read()
    (csrc / "lbrmt_kernels.cuh").write_text(src)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.precision_errors("fp16") == {"rho": 5e-8, "u": 5e-4, "F": 9e-5}
    assert bench.precision_errors("bf16") is None
    (csrc / "lbrmt_kernels.cuh").write_text(src + "\n// edited\n")
    assert bench.precision_errors("fp16") is None  # stale: taken on other kernels
