"""Multi-process paths on the CPU (gloo, world size 2).

The benchmark runs one independent replica per GPU (no collective on the data
path); its process group only times the job: barriers around the timed region
and the maximum over ranks of each rank's time.  These tests run that host
logic in two gloo processes, and the reference arm (the oracle, rank 0 only)
under torch.distributed.run.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(ws),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import scenarios
    r = bench.Ranks("gloo")
    r.barrier()
    slowest = r.max(0.5 + rank)  # each rank's "time"; the job takes the slowest
    sc = scenarios.mixing_4096(seed=r.rank, n=256, count=8)  # the rank's replica
    first = (sc["solids"][0]["x"], sc["solids"][0]["y"])
    r.barrier()
    r.close()
    q.put((rank, slowest, first))


def test_ranks_barrier_and_max_over_two_gloo_processes():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [1.5, 1.5]  # both ranks see the slowest time
    assert out[0][2] != out[1][2]  # independent seeded replicas


def test_aggregate_throughput_counts_every_replica():
    sys.path.insert(0, ROOT)
    import bench
    # two replicas of 1e6 nodes, 100 steps, the slowest rank took 50 ms
    assert bench.aggregate_mlups(1_000_000, 100, 2, 50.0) == pytest.approx(4000.0)
    assert bench.aggregate_mlups(1_000_000, 100, 1, 50.0) == pytest.approx(2000.0)


@pytest.mark.slow
def test_reference_arm_prints_one_line_from_rank_zero():
    # the oracle on a bounded sample, under torch.distributed.run with two ranks:
    # rank 0 alone times it and prints the JSON line, rank 1 exits without work
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
