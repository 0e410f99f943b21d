"""Adaptive parareal with the fine batch split across ranks (paper_2212_10508_gb300.distributed),
on CPU: gloo ranks, propagators from the oracle (Finnis-Sinclair fine, a perturbed
Finnis-Sinclair coarse, the 55-atom W + SIA cell).  Two ranks must give, bit for bit, the states
and slab log of one rank, and the slabs of the oracle's Algorithm 2 with the same propagators;
the block split must tile every slab."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_blocks_tile_the_slab():
    from paper_2212_10508_gb300.distributed import block
    for a, b in [(0, 7), (3, 3), (5, 6), (10, 31)]:
        for world in (1, 2, 3, 4):
            spans = [block(a, b, r, world) for r in range(world)]
            assert spans[0][0] == a and spans[-1][1] == b
            assert all(s[1] == t[0] for s, t in zip(spans, spans[1:]))
            sizes = [h - l for l, h in spans]
            assert max(sizes) - min(sizes) <= 1


WORKER = r"""
import json, os, sys
sys.path.insert(0, {root!r})
sys.path.insert(0, os.path.join({root!r}, "tests"))
import numpy as np, torch, torch.distributed as dist
from dist_ops import OracleOps, setup
from paper_2212_10508_gb300.distributed import adaptive_parareal_dist
rank, ws = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
q0, v0, ops, N, dc, de = setup()
cur, st = adaptive_parareal_dist(ops, torch.as_tensor(q0), torch.as_tensor(v0), N, dc, de)
if rank == 0:
    np.save(os.path.join({out!r}, "cur_%d.npy" % ws), cur.numpy())
    json.dump(st.log(), open(os.path.join({out!r}, "log_%d.json" % ws), "w"))
dist.destroy_process_group()
"""


def _run(world, out):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    code = WORKER.format(root=ROOT, port=port, out=str(out))
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                   OMP_NUM_THREADS="2")
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    for p in procs:
        o, e = p.communicate(timeout=600)
        assert p.returncode == 0, e[-3000:]


def test_two_ranks_equal_one_rank_and_algorithm_2(tmp_path):
    _run(1, tmp_path)
    _run(2, tmp_path)
    c1, c2 = np.load(tmp_path / "cur_1.npy"), np.load(tmp_path / "cur_2.npy")
    assert np.array_equal(c1, c2)
    l1 = json.load(open(tmp_path / "log_1.json"))
    l2 = json.load(open(tmp_path / "log_2.json"))
    assert l1 == l2 and len({e[3] for e in l1}) > 1          # several slabs
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from dist_ops import setup
    from oracle import parareal as PR
    q0, v0, ops, N, dc, de = setup()
    ocur, olog = PR.adaptive(q0, v0, N, dc, de, ops.F, ops.C, metric="maxdisp")
    want = [[w["n_init"], e, k, i] for i, w in enumerate(olog.windows) for e, k in w["subs"]]
    assert [list(e) for e in l1] == want
    for n in range(N + 1):
        assert np.abs(c1[n, :3] - ocur[n][0]).max() < 1e-12
