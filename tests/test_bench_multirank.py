"""The multi-rank path of bench.py on CPU (gloo, world size 2): interval sharding without shared
data, whole-job reduction (elapsed time maxed, atom-steps summed over the ranks), and the
reference arm's rank-0-only output."""
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


WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
rank, ws = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
import bench
seed, id0 = bench._shard(rank)
# rank r pretends to have run (r + 1) * 10 ms over (r + 1) * 1000 atom-steps
rate, ms, steps = bench._job_rate(10.0 * (rank + 1), 1000.0 * (rank + 1), ws, "cpu")
print(json.dumps({{"rank": rank, "seed": seed, "id0": id0, "rate": rate, "ms": ms, "steps": steps}}))
dist.destroy_process_group()
"""


def test_two_rank_sharding_and_reduction():
    port = _free_port()
    code = WORKER.format(root=ROOT, port=port)
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(__import__("json").loads(o.strip().splitlines()[-1]))
    a, b = sorted(outs, key=lambda d: d["rank"])
    import bench
    # disjoint interval ranges (distinct noise keys) and distinct workload seeds
    assert a["id0"] == 0 and b["id0"] == bench.NSLAB
    assert a["seed"] != b["seed"]
    # whole job: slowest rank's time, all ranks' atom-steps; every rank reports the same
    for d in (a, b):
        assert d["ms"] == 20.0
        assert d["steps"] == 3000.0
        assert d["rate"] == pytest.approx(3000.0 / 0.020)


def test_single_rank_reduction_is_local():
    import bench
    rate, ms, steps = bench._job_rate(50.0, 1e6, 1, "cpu")
    assert (ms, steps) == (50.0, 1e6) and rate == pytest.approx(2e7)


def test_reference_arm_prints_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
