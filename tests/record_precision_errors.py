"""Write the per-field errors of the full-size 4096^2 mixing parity run into
profiles/precision_errors_mixing4096.json, keyed by the kernels' source hash.

Usage: python tests/record_precision_errors.py <parity log (JSON lines)> [output path]

The log is what tests/test_gpu_parity.py and tests/test_gpu_half.py append
when LBRMT_PARITY_LOG names a file: one line per case, with the relative L-inf
error of every field against the FP64 oracle after 4 steps.  bench.py reports
these errors beside each precision's throughput only while the kernels' hash
still matches, so a record taken on older kernels is never shown.
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASE = "mixing_4096_full/"
FIELDS = ("rho", "u", "F", "drho", "xi", "xi_band", "label_mismatch")


def main(log, path=None):
    errors = {}
    for line in open(log):
        rec = json.loads(line)
        if not rec["case"].startswith(CASE):
            continue
        prec = rec["case"][len(CASE):]
        res = rec["res"]["4"]
        errors[prec] = {k: res[k] for k in FIELDS if k in res}
    if not errors:
        sys.exit(f"no {CASE}* case in {log}")
    src = open(os.path.join(ROOT, "paper_2402_12696_gb300", "csrc", "lbrmt_kernels.cuh")).read()
    out = {"workload": "mixing suspension 4096x4096, 1024 disks (seed 0), 4 steps from the initial state",
           "reference": "FP64 oracle (oracle/lbrmt_oracle.c); relative L-inf per field over the whole grid "
                        "(xi, xi_band, label_mismatch over 24 sampled solids)",
           "kernels_sha1": hashlib.sha1(src.encode()).hexdigest()[:12],
           "errors": errors}
    path = path or os.path.join(ROOT, "profiles", "precision_errors_mixing4096.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path, sorted(errors))
    return out


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2] if len(sys.argv) > 2 else None)
