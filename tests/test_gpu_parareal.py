"""GPU parareal against the oracle's Algorithm 2 transcription and the exactness property
(Sec. 2.1: q^k_n = q^ref_n for n <= k).  Engine: SNAP 2J = 8 fine, Finnis-Sinclair coarse,
the 55-atom W + SIA cell (3^3 cells), FP64."""
import numpy as np
import pytest

import oracle as O
from oracle import parareal as PR
import paper_2212_10508_gb300 as P
import workloads as W
from gpu_util import N, T, dev, rel_max, torch

pytestmark = pytest.mark.gpu

DT, GAMMA, TEMP, SEED = 2e-3, 1.0, 2000.0, 31


def _setup():
    pos, box = W.bcc_sia(3)
    q0 = W.displaced(pos, 0.05, W.rng(21, 1))
    v0 = W.velocities(pos.shape[1], TEMP, W.rng(21, 2))
    beta = W.snap_beta(55, W.rng(21, 3))
    eng = P.Engine(pos.shape[1], box, P.snap_params(), P.fs_params(), beta=T(beta))
    return q0, v0, box, beta, eng


def _oracle_props(box, beta, L):
    lp = O.langevin(dt=DT, gamma=GAMMA, T=TEMP, seed=SEED, schedule=O.SCHED_ROBUST)

    def make(pot):
        def prop(states, ns):
            q = np.ascontiguousarray(np.array([s[0] for s in states]))
            v = np.ascontiguousarray(np.array([s[1] for s in states]))
            O.propagate(pot, q, v, box, [L] * len(ns), ns, lp)
            return [(q[i], v[i]) for i in range(len(ns))]
        return prop
    return make(O.potential(O.POT_SNAP, beta=beta)), make(O.potential(O.POT_FS))


@pytest.mark.parametrize("metric,dc,de", [(P.METRIC_REL, 1e-13, 1.0), (P.METRIC_MAXDISP, 1e-10, 4e-4)])
def test_adaptive_parareal_matches_algorithm_2(metric, dc, de):
    q0, v0, box, beta, eng = _setup()
    Nint, L = 6, 2
    lp = P.langevin(dt=DT, gamma=GAMMA, T=TEMP, seed=SEED, schedule=P.SCHED_ROBUST)
    cur, st = P.adaptive_parareal(eng, T(q0), T(v0), Nint, L, dc, de, lp, metric=metric)
    eng.sync_status()
    F, C = _oracle_props(box, beta, L)
    ocur, olog = PR.adaptive(q0, v0, Nint, dc, de, F, C, metric="rel" if metric == P.METRIC_REL else "maxdisp")
    want = [(w["n_init"], e, k, i) for i, w in enumerate(olog.windows) for e, k in w["subs"]]
    assert st.log() == want
    g = N(cur)
    for n in range(Nint + 1):
        assert np.abs(g[n, :3] - ocur[n][0]).max() < 1e-8
        assert np.abs(g[n, 3:] - ocur[n][1]).max() < 1e-6


def test_exactness_k_ge_n_on_gpu():
    """After k parareal iterations the first k intervals equal the sequential fine trajectory."""
    q0, v0, box, beta, eng = _setup()
    n_at = q0.shape[1]
    Nint, L = 5, 3
    lp = P.langevin(dt=DT, gamma=GAMMA, T=TEMP, seed=SEED)
    ref = torch.empty(Nint + 1, 6, n_at, dtype=torch.float64, device=dev())
    ref[0, :3], ref[0, 3:] = T(q0), T(v0)
    for n in range(Nint):
        s = ref[n:n + 1].clone()
        eng.baoab_propagate_batch(P.FINE, s, None, T([L], torch.int32), T([n], torch.int64), lp)
        ref[n + 1] = s[0]
    cur = torch.zeros_like(ref)
    cur[0] = ref[0]
    cache = torch.zeros(Nint, 6, n_at, dtype=torch.float64, device=dev())
    eng.parareal_correct(0, Nint, None, cur, cur, cache, float("inf"), P.METRIC_REL, L, lp)
    ids = T(np.arange(Nint), torch.int64)
    for k in range(1, Nint + 2):            # E = 0 once k >= N + 1 (Sec. 2.1)
        prev = cur.clone()
        fine = prev[:Nint].clone()
        eng.baoab_propagate_batch(P.FINE, fine, None, T([L] * Nint, torch.int32), ids, lp)
        jumps = torch.empty_like(fine)
        eng.parareal_jumps(Nint, fine, cache, jumps)
        delta, n_stop = eng.parareal_correct(0, Nint, jumps, prev, cur, cache, float("inf"), P.METRIC_REL, L, lp)
        assert n_stop == Nint
        kk = min(k, Nint)
        d = (cur[:kk + 1] - ref[:kk + 1]).abs().max().item()
        assert d < 1e-12
    assert delta < 1e-14


def test_correct_reports_explosion_and_nonfinite():
    q0, v0, box, beta, eng = _setup()
    n_at = q0.shape[1]
    lp = P.langevin(dt=DT, gamma=GAMMA, T=TEMP, seed=SEED)
    cur = torch.zeros(4, 6, n_at, dtype=torch.float64, device=dev())
    cur[0, :3], cur[0, 3:] = T(q0), T(v0)
    prev = cur.clone()
    cache = torch.zeros(3, 6, n_at, dtype=torch.float64, device=dev())
    jumps = torch.zeros(3, 6, n_at, dtype=torch.float64, device=dev())
    jumps[1, 0, 0] = 0.5                    # a 0.5 Angstrom kick on atom 0 after interval 1
    prev[1:] = cur[0]                       # prev far from the coarse path: large REL error
    eng.parareal_correct(0, 3, None, prev, prev, torch.zeros_like(cache), float("inf"), P.METRIC_REL, 1, lp)
    d, ns = eng.parareal_correct(0, 3, jumps, prev, cur, cache, 0.3, P.METRIC_MAXDISP, 1, lp)
    assert ns == 1 and d > 0.3
    jumps[0, 0, 3] = float("nan")
    d, ns = eng.parareal_correct(0, 3, jumps, prev, cur, cache, 1e9, P.METRIC_REL, 1, lp)
    assert ns == 0 and d == float("inf")


DIST_WORKER = r"""
import os, sys
sys.path.insert(0, {root!r})
import numpy as np, torch, torch.distributed as dist
import paper_2212_10508_gb300 as P
import workloads as W
from paper_2212_10508_gb300.distributed import EngineOps, adaptive_parareal_dist
torch.cuda.set_device(0)
dist.init_process_group("nccl", init_method="tcp://127.0.0.1:{port}", rank=0, world_size=1)
pos, box = W.bcc_sia(3)
q0 = torch.as_tensor(W.displaced(pos, 0.05, W.rng(21, 1)), device="cuda")
v0 = torch.as_tensor(W.velocities(pos.shape[1], 2000.0, W.rng(21, 2)), device="cuda")
beta = torch.as_tensor(W.fitted_beta(), device="cuda")
lp = P.langevin(dt=2e-3, gamma=1.0, T=2000.0, seed=31, schedule=P.SCHED_ROBUST)
e1 = P.Engine(pos.shape[1], box, beta=beta)
c1, s1 = P.adaptive_parareal(e1, q0, v0, 12, 2, 1e-10, 2e-3, lp, metric=P.METRIC_MAXDISP)
e2 = P.Engine(pos.shape[1], box, beta=beta)
c2, s2 = adaptive_parareal_dist(EngineOps(e2, 2, lp, P.METRIC_MAXDISP), q0, v0, 12, 1e-10, 2e-3)
e1.sync_status(); e2.sync_status()
assert torch.equal(c1, c2), float((c1 - c2).abs().max())
assert s1.log() == s2.log() and len({{e[3] for e in s1.log()}}) > 1, s1.log()
dist.destroy_process_group()
print("ok")
"""


def test_distributed_driver_with_engine_equals_single_gpu_driver():
    """The multi-rank driver (EngineOps, NCCL process group of one rank) gives, bit for bit, the
    single-GPU adaptive_parareal's states and slab log (several slabs)."""
    import os
    import socket
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), NCCL_NVLS_ENABLE="0")
    r = subprocess.run([sys.executable, "-c", DIST_WORKER.format(root=root, port=port)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-3000:]


def _sweep_system(name):
    """Cells of the cluster sweep's range: K = min(8, ceil(n/32)) CTAs of m = ceil(n/K) own atoms,
    two threads per atom's pairs up to 256 atoms, one above."""
    if name == "first65":   # 65 atoms of the 129-atom cell: 3 CTAs of 22, 22, 21 atoms
        pos, box = W.bcc_sia(4)
        return np.ascontiguousarray(pos[:, :65]), box
    return W.bcc_sia({"129": 4, "251": 5, "433": 6}[name])


@pytest.mark.parametrize("system", ["first65", "129", "251", "433"])
@pytest.mark.parametrize("precision", [P.FP64, P.FP32_BULK])
@pytest.mark.parametrize("scheme,L", [(P.SCHEME_PAPER, 1), (P.SCHEME_PAPER, 3), (P.SCHEME_BAOAB, 2)])
@pytest.mark.parametrize("jumps", [False, True])
def test_cluster_sweep_equals_coarse_batch(system, precision, scheme, L, jumps):
    """The correction sweep of the Finnis-Sinclair coarse potential runs on a cluster of CTAs for
    systems of 64..512 atoms; the coarse states it caches, C(cur_n), must equal bit for bit those
    of the one-CTA coarse batch kernel applied to the same cur_n (the jumps J_n = F - C(prev_n) of
    the next iteration use the batch's values), with or without jumps (a jump moves every atom,
    so the sweep's Verlet lists and the batch's come from different position histories), and
    without jumps cur_{n+1} = C(cur_n).  The systems cover an uneven split over 3 CTAs, 5 and 8
    CTAs with two threads per atom, and 8 CTAs of 55 atoms with one thread per atom (own atoms in
    two blocks of 32)."""
    pos, box = _sweep_system(system)
    n = pos.shape[1]
    N = 7
    eng = P.Engine(n, box, P.snap_params(), P.fs_params(precision=precision))
    lp = P.langevin(dt=2e-3, gamma=1.0, T=2000.0, scheme=scheme, seed=23)
    cur = torch.zeros(N + 1, 6, n, dtype=torch.float64, device=dev())
    cur[0, :3] = T(W.displaced(pos, 0.05, W.rng(24, 1)))
    cur[0, 3:] = T(W.velocities(n, 2000.0, W.rng(24, 2)))
    J = None
    if jumps:
        g = W.rng(24, 3)
        J = T(np.concatenate([g.normal(0.0, 0.02, (N, 3, n)), g.normal(0.0, 0.5, (N, 3, n))], axis=1))
    prev = cur.clone()
    cache = torch.zeros(N, 6, n, dtype=torch.float64, device=dev())
    delta, n_stop = eng.parareal_correct(0, N, J, prev, cur, cache, float("inf"), P.METRIC_MAXDISP, L, lp)
    eng.sync_status()
    assert n_stop == N
    batch = cur[:N].clone()
    eng.baoab_propagate_batch(P.COARSE, batch, None, T(np.full(N, L, np.int32), torch.int32),
                              T(np.arange(N), torch.int64), lp)
    eng.sync_status()
    assert torch.equal(batch, cache)
    if jumps:
        assert torch.equal(cur[1:], cache + J)
    else:
        assert torch.equal(cur[1:], cache)


def test_cluster_sweep_adaptive_parareal_matches_algorithm_2_251_atoms():
    """Algorithm 2 on the 251-atom cell (cluster sweep) against the oracle's transcription:
    the same slabs and iteration counts, trajectories to 1e-8 Angstrom."""
    pos, box = W.bcc_sia(5)
    n = pos.shape[1]
    q0 = W.displaced(pos, 0.05, W.rng(25, 1))
    v0 = W.velocities(n, 1500.0, W.rng(25, 2))
    beta = W.fitted_beta()
    eng = P.Engine(n, box, P.snap_params(), P.fs_params(), beta=T(beta))
    Nint, L, dc, de = 6, 1, 1e-10, 2e-3
    lp = P.langevin(dt=DT, gamma=GAMMA, T=1500.0, seed=SEED, schedule=P.SCHED_ROBUST)
    cur, st = P.adaptive_parareal(eng, T(q0), T(v0), Nint, L, dc, de, lp, metric=P.METRIC_MAXDISP)
    eng.sync_status()
    olp = O.langevin(dt=DT, gamma=GAMMA, T=1500.0, seed=SEED, schedule=O.SCHED_ROBUST)

    def make(pot):
        def prop(states, ns):
            q = np.ascontiguousarray(np.array([s[0] for s in states]))
            v = np.ascontiguousarray(np.array([s[1] for s in states]))
            O.propagate(pot, q, v, box, [L] * len(ns), ns, olp)
            return [(q[i], v[i]) for i in range(len(ns))]
        return prop
    ocur, olog = PR.adaptive(q0, v0, Nint, dc, de, make(O.potential(O.POT_SNAP, beta=beta)), make(O.potential(O.POT_FS)),
                             metric="maxdisp")
    want = [(w["n_init"], e, k, i) for i, w in enumerate(olog.windows) for e, k in w["subs"]]
    assert st.log() == want
    g = N(cur)
    for k in range(Nint + 1):
        assert np.abs(g[k, :3] - ocur[k][0]).max() < 1e-8


def _host_delta(cur, prev, k, metric):
    """The sweep's error after interval k (states 0..k+1), from the definition in pmd.h."""
    c, p = N(cur[:k + 2, :3]), N(prev[:k + 2, :3])
    if metric == P.METRIC_MAXDISP:
        return float(np.sqrt(((c - p) ** 2).sum(axis=1)).max())
    num = sum(np.linalg.norm(c[m] - p[m]) for m in range(k + 2))
    den = sum(np.linalg.norm(p[m]) for m in range(k + 2))
    return num / den


@pytest.mark.parametrize("system", ["129", "433"])
@pytest.mark.parametrize("metric", [P.METRIC_MAXDISP, P.METRIC_REL])
def test_cluster_sweep_error_and_explosion_test(system, metric):
    """The cluster sweep's running error and explosion test (Algorithm 2, "N_final := n"): the
    returned delta equals the error recomputed on the host from the output states; a threshold
    between two intervals' errors stops the sweep at the first interval above it, with the states
    before the stop those of the full sweep; a threshold equal to the device's own error after
    interval k does not stop at k (the maximum metric compares squares with a precomputed
    threshold: exact at the boundary); a non-finite jump stops the sweep at its interval with
    delta = inf and no device error, and with delta_expl = inf the next intervals integrate the
    non-finite state and the call fails with ENONFINITE."""
    pos, box = _sweep_system(system)
    n = pos.shape[1]
    Nn = 6
    eng = P.Engine(n, box, P.snap_params(), P.fs_params(precision=P.FP32_BULK))
    lp = P.langevin(dt=2e-3, gamma=1.0, T=2000.0, seed=29)
    cur0 = torch.zeros(Nn + 1, 6, n, dtype=torch.float64, device=dev())
    cur0[0, :3] = T(W.displaced(pos, 0.05, W.rng(26, 1)))
    cur0[0, 3:] = T(W.velocities(n, 2000.0, W.rng(26, 2)))
    prev = cur0.clone()
    prev[1:] = cur0[0]                       # the error grows with the distance from the start
    g = W.rng(26, 3)
    J = T(np.concatenate([g.normal(0.0, 0.01, (Nn, 3, n)), g.normal(0.0, 0.2, (Nn, 3, n))], axis=1))

    def run(nfin, dexpl, jumps=J, check=True):
        cur = cur0.clone()
        cache = torch.zeros(Nn, 6, n, dtype=torch.float64, device=dev())
        d, ns = eng.parareal_correct(0, nfin, jumps, prev, cur, cache, dexpl, metric, 1, lp)
        if check:
            eng.sync_status()
        return cur, d, ns

    def first_above(thr):
        return next((k for k in range(Nn) if D[k] > thr), Nn)

    full, dA, nsA = run(Nn, float("inf"))
    assert nsA == Nn
    D = [_host_delta(full, prev, k, metric) for k in range(Nn)]
    assert abs(dA - D[-1]) <= 1e-12 * D[-1]
    k1 = next(k for k in range(1, Nn) if D[k] > D[k - 1] * (1 + 1e-6))   # an interval whose error rises
    stop = first_above(0.5 * (D[k1 - 1] + D[k1]))
    cut, dB, nsB = run(Nn, 0.5 * (D[k1 - 1] + D[k1]))
    assert nsB == stop <= k1 and abs(dB - D[stop]) <= 1e-12 * D[stop]
    assert torch.equal(cut[:stop + 1], full[:stop + 1])
    _, dk, _ = run(k1, float("inf"))            # the device's own error after interval k1 - 1
    assert abs(dk - D[k1 - 1]) <= 1e-12 * D[k1 - 1]
    _, dC, nsC = run(Nn, dk)
    assert nsC != k1 - 1 and nsC == first_above(dk * (1 + 1e-12))
    Jn = J.clone()
    Jn[1, 0, n // 2] = float("nan")
    _, d, ns = run(Nn, 1e9, Jn)                 # reported by delta = inf; nothing integrated it
    assert ns == 1 and d == float("inf")
    with pytest.raises(P.PmdError, match="ENONFINITE"):   # delta_expl = inf: the next intervals
        run(Nn, float("inf"), Jn, check=False)             # integrate it, and the call reports that
