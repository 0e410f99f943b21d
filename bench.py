#!/usr/bin/env python3
"""Throughput of the batched fine propagator (SNAP 2J = 8 Langevin steps for all parareal
intervals in one persistent launch) on GB300, with the plain-FP64 form, the larger 2001-atom
cell, the oracle on the host cores, the roofline of the dominant kernel against the measured FMA
throughput of the device, and an end-to-end number through the C ABI.

Workload (one "step"): 64 intervals of the 129-atom W + SIA cell (4^3 BCC cells + a <111>
dumbbell), SNAP coefficients fitted to Finnis-Sinclair tungsten (tests/golden/beta_fs_w_2j8.txt;
random coefficients collapse the cell), interval lengths L_b ~ U{100..2000}, 1500 K, dt = 1 fs,
gamma = 1/ps, paper scheme with the robust temperature schedule; the whole batch is advanced by
one baoab_propagate_batch(FINE) call (FP32-bulk SNAP: U/Z/Y in FP32, energy sums in FP64, force
sums in double-float; FP64 positions, velocities and noise).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line on rank 0.  Under torchrun each rank advances its own 64 intervals
(weak scaling, no data-path collective).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fine atom-steps/s (SNAP 2J=8, batched slabs) vs plain FP64; parareal speedup"
UNIT = "atom-steps/s"
NSLAB, NCELL, TEMP, DT, GAMMA = 64, 4, 1500.0, 1e-3, 1.0
WORKLOAD = ("batched fine propagation: 64 intervals x 129-atom W+SIA cell, SNAP 2J=8 (55 B, fitted to FS W), "
            "L_b ~ U{100..2000}, 1500 K, dt 1 fs, gamma 1/ps, one persistent launch")
SMALL = "profiling case: the same 64 intervals with L_b ~ U{5..20}"
WORKLOAD3 = ("2001-atom W+SIA cell (10^3 cells), SNAP 2J=8 fitted, 32 intervals x 500 steps, 1000 K, "
             "dt 1 fs, gamma 1/ps, one persistent launch")
# DRAM bytes (read + write) of one full-size launch of the persistent FP32 kernel, from one ncu
# capture of this workload (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the
# kernel sources it was taken on (fingerprint of the persistent kernel's translation unit and of
# the host code that builds its tables); reported as null otherwise.
TRAFFIC = {"bytes_per_launch": 3.30e6 + 19.80e6, "csrc_sha256_16": "e366a45a5738d27b"}
# CPU-baseline samples of the oracle: (intervals or members, steps each) of config 2 and config 3,
# on all host cores; the single-thread legs take one interval or member of the same sample (the
# oracle's per-atom-step cost on one thread does not depend on how many members a call holds)
CPU_SAMPLES = {"cfg2": (8, 100), "cfg3": (2, 20)}
CPU_SAMPLES_1T = {"cfg2": (1, 100), "cfg3": (1, 10)}


# the persistent kernel's translation unit (propagate.cu and every header it includes) and the host
# code that builds its tables (snap.cu)
KERNEL_SOURCES = ("propagate.cu", "snap.cu", "snap_kernels.cuh", "snap_batch.cuh", "snap_v2.cuh", "snap_device.cuh",
                  "device_common.cuh", "langevin_device.cuh", "eam_device.cuh", "snap_coarse.cuh", "sweep_cluster.cuh",
                  "pmd_internal.h", "status_bits.h")


def _csrc_fingerprint():
    import hashlib
    d = os.path.join(ROOT, "paper_2212_10508_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 comparison")
    ap.add_argument("--no-config3", action="store_true", help="skip the 2001-atom cell")
    ap.add_argument("--no-parareal", action="store_true", help="skip the single-system parareal leg")
    ap.add_argument("--case", default="full", choices=["full", "small"],
                    help="small: L_b ~ U{5..20} (a short launch for ncu captures)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the engine's default launch shape (profiling captures count launches)")
    ap.add_argument("--cpu-leg", default=None, choices=sorted(CPU_SAMPLES),
                    help=argparse.SUPPRESS)   # worker: one oracle sample, prints one JSON line
    return ap.parse_args()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _shard(rank):
    """Rank r owns the intervals [r*NSLAB, (r+1)*NSLAB) (their ids key the noise) and draws its own
    configurations and lengths from a rank-specific seed: the ranks share no data."""
    return 2212 + 7919 * rank, rank * NSLAB


def _job_rate(elapsed_ms, atom_steps, ws, device):
    """Whole-job throughput: atom-steps summed over the ranks / elapsed time maxed over the ranks.
    Returns (rate per s, job elapsed ms, job atom-steps)."""
    if ws > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
        a = torch.tensor([atom_steps], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(a, op=dist.ReduceOp.SUM)
        elapsed_ms, atom_steps = float(t.item()), float(a.item())
    return atom_steps / (elapsed_ms / 1e3), elapsed_ms, atom_steps


class Clocks:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _avg_neighbors(q, box, rc):
    """Mean neighbour count of the batch (measurement input for the flop model)."""
    tot = 0
    for m in range(q.shape[0]):
        X = q[m].T
        d = X[None, :, :] - X[:, None, :]
        d -= box * np.rint(d / box)
        r2 = np.sum(d * d, axis=2)
        tot += np.sum(r2 < rc * rc) - X.shape[0]
    return tot / (q.shape[0] * q.shape[2])


def _config3_inputs(nmem=32, steps=500):
    import workloads as W
    pos, box = W.bcc_sia(10)
    n = pos.shape[1]
    q = W.displaced(pos, 0.05, W.rng(61, 1), count=nmem)
    v = W.velocities(n, 1000.0, W.rng(61, 2), count=nmem)
    L = np.full(nmem, steps, np.int32)
    ids = np.arange(nmem, dtype=np.int64)
    return q, v, box, W.fitted_beta(), L, ids, 1000.0


def _cpu_sample(cfg, single=False):
    """The oracle sample of config 2 (first 8 intervals x 100 steps) or config 3 (2 members x 20
    steps), or its single-thread cut: returns its inputs (q, v, box, beta, L, ids, T) with L cut
    to the sample's steps."""
    import workloads as W
    nm, steps = (CPU_SAMPLES_1T if single else CPU_SAMPLES)[cfg]
    if cfg == "cfg2":
        q, v, box, beta, L, ids = W.batch_workload(nbatch=NSLAB, T=TEMP)
        T = TEMP
    else:
        q, v, box, beta, L, ids, T = _config3_inputs()
    return (q[:nm].copy(), v[:nm].copy(), box, beta, np.minimum(L[:nm], steps).astype(np.int32), ids[:nm].copy(), T)


def _oracle_run(cfg, single=False):
    """Runs the oracle on one CPU sample on as many threads as OpenMP gives it; returns
    (result dict, final q, final v, sample inputs)."""
    import oracle as O
    q, v, box, beta, L, ids, T = _cpu_sample(cfg, single)
    pot = O.potential(O.POT_SNAP, beta=beta)
    lp = O.langevin(dt=DT, gamma=GAMMA, T=T, seed=2212, schedule=O.SCHED_ROBUST)
    qq, vv = q.copy(), v.copy()
    t0 = time.perf_counter()
    O.propagate(pot, qq, vv, box, L, ids, lp)
    dt = time.perf_counter() - t0
    atom_steps = float(L.sum()) * q.shape[2]
    nm, steps = (CPU_SAMPLES_1T if single else CPU_SAMPLES)[cfg]
    what = ("config 2: %d of the 64 intervals x %d steps (129 atoms)" if cfg == "cfg2"
            else "config 3: %d of the 32 members x %d steps (2001 atoms)") % (nm, steps)
    res = {"value": atom_steps / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
           "sample": "%s, FP64 oracle, %.1f s" % (what, dt), "seconds": dt}
    return res, qq, vv, (q, v, box, beta, L, ids, T)


def _spawn_single_thread_legs():
    """Starts the single-thread oracle legs as child processes (fresh interpreters, one OpenMP
    thread each) so that they run while the GPU legs run; returns {cfg: Popen}."""
    procs = {}
    env = dict(os.environ, OMP_NUM_THREADS="1")
    for cfg in sorted(CPU_SAMPLES):
        procs[cfg] = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-leg", cfg], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
    return procs


def _collect(procs):
    out = {}
    for cfg, p in procs.items():
        so, se = p.communicate()
        try:
            out[cfg] = json.loads(so.strip().splitlines()[-1])
        except (ValueError, IndexError):
            out[cfg] = {"error": (se or so).strip().splitlines()[-1:] or ["no output"]}
    return out


def _parareal(P, W, dev, torch, Nh=300, window=300, ncell=5, T=1500.0, strategy=2):
    """Adaptive parareal (Algorithm 2) on a 251-atom cell vs the same N intervals run one after
    the other with the fine propagator (the paper's sequential cost N C_f), on this GPU.  The N
    intervals are cut into windows of `window` intervals; window w draws its noise with seed + w
    on both sides (interval ids 0 .. window - 1), and each trajectory starts a window from its own
    end state of the previous one.  strategy 2: Finnis-Sinclair coarse propagator (the correction
    sweep on a thread-block cluster); strategy 1: SNAP-6 (2J = 2) coarse propagator, coefficients
    fitted like the fine ones (the one-CTA sweep)."""
    pos, box = W.bcc_sia(ncell)
    n = pos.shape[1]
    beta = torch.as_tensor(W.fitted_beta(), device=dev)
    q0 = torch.as_tensor(W.displaced(pos, 0.05, W.rng(5, 1)), device=dev)
    v0 = torch.as_tensor(W.velocities(n, T, W.rng(5, 2)), device=dev)
    if strategy == 1:
        eng = P.Engine(n, box, P.snap_params(precision=P.FP32_BULK),
                       coarse_snap=P.snap_params(twojmax=2, precision=P.FP32_BULK), beta=beta,
                       coarse_beta=torch.as_tensor(W.fitted_beta(2), device=dev))
    else:
        eng = P.Engine(n, box, P.snap_params(precision=P.FP32_BULK), P.fs_params(precision=P.FP32_BULK), beta=beta)
    eng.reserve(window)
    L, dconv, dexpl = 1, 1e-3, 0.1
    nwin = Nh // window

    def lp_of(w):
        return P.langevin(dt=1e-3, gamma=1.0, T=T, scheme=P.SCHEME_PAPER, schedule=P.SCHED_L1_SYM, seed=77 + w)
    one = torch.ones(1, dtype=torch.int32, device=dev)
    ids = torch.arange(window, dtype=torch.int64, device=dev)

    def sequential():
        st = torch.empty(1, 6, n, dtype=torch.float64, device=dev)
        st[0, :3], st[0, 3:] = q0, v0
        for w in range(nwin):
            lp = lp_of(w)
            for k in range(window):
                eng.baoab_propagate_batch(P.FINE, st, None, one, ids[k:k + 1], lp)
        return st

    def parareal():
        q, v = q0, v0
        logs = []
        for w in range(nwin):
            cur, st = P.adaptive_parareal(eng, q, v, window, L, dconv, dexpl, lp_of(w), metric=P.METRIC_MAXDISP)
            q, v = cur[window, :3].contiguous(), cur[window, 3:].contiguous()
            logs.append(st)
        return q, logs

    sequential()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ref = sequential()
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    P.adaptive_parareal(eng, q0, v0, 20, L, dconv, dexpl, lp_of(0), metric=P.METRIC_MAXDISP)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qend, logs = parareal()
    torch.cuda.synchronize()
    t_par = time.perf_counter() - t0
    eng.sync_status()
    # coarse cost per interval: one sweep over a window
    cache = torch.empty(window, 6, n, dtype=torch.float64, device=dev)
    tmp = torch.empty(window + 1, 6, n, dtype=torch.float64, device=dev)
    tmp[0, :3], tmp[0, 3:] = q0, v0
    eng.parareal_correct(0, window, None, tmp, tmp, cache, float("inf"), P.METRIC_MAXDISP, L, lp_of(0))
    t0 = time.perf_counter()
    eng.parareal_correct(0, window, None, tmp, tmp, cache, float("inf"), P.METRIC_MAXDISP, L, lp_of(0))
    t_c = (time.perf_counter() - t0) / window
    t_f = t_seq / Nh
    # eqs. (7)-(9) summed over the windows (each window is its own Algorithm 2 horizon)
    costs = [st.cost(t_f, t_c) for st in logs]
    cost = sum(c[0] for c in costs)
    k_sum = sum(sum(e[2] for e in st.log()) for st in logs)
    # the fine batches alone: one launch of each slab width the run used, timed, times the number
    # of iterations on that width (the bound a free correction sweep would leave)
    width_ms = {}
    batch = tmp[:window].clone()
    for st in logs:
        for (a, b, k, _) in st.log():
            w = b - a
            if w not in width_ms:
                ns = torch.full((w,), L, dtype=torch.int32, device=dev)
                eng.baoab_propagate_batch(P.FINE, batch[:w], None, ns, ids[:w], lp_of(0))
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                eng.baoab_propagate_batch(P.FINE, batch[:w], None, ns, ids[:w], lp_of(0))
                torch.cuda.synchronize()
                width_ms[w] = (time.perf_counter() - t0) * 1e3
    t_fine_batches = sum(k * width_ms[b - a] for st in logs for (a, b, k, _) in st.log()) / 1e3
    coarse = "SNAP-6 (2J=2) fitted (FP32-bulk) coarse (Strategy I)" if strategy == 1 else \
        "FS EAM (FP32-bulk) coarse (Strategy II)"
    return {"workload": "251-atom W+SIA (5^3 cells), SNAP 2J=8 fitted (FP32-bulk) fine, %s, "
                        "dt 1 fs, L=1, 1500 K, gamma 1/ps, schedule C0=C1=2, N=%d intervals in windows of %d"
                        % (coarse, Nh, window),
            "delta_conv_A": dconv, "delta_expl_A": dexpl, "metric": "max per-atom displacement (A)",
            "wall_sequential_s": t_seq, "wall_parareal_s": t_par, "speedup": t_seq / t_par,
            "n_slab": int(sum((st.log()[-1][3] + 1) if st.log() else 0 for st in logs)), "iterations": int(k_sum),
            "C_f_ms": t_f * 1e3, "C_c_ms": t_c * 1e3, "gamma_adapt_eq8": Nh * t_f / cost, "gamma_ideal_eq9": Nh / k_sum,
            "fine_batches_s": t_fine_batches, "speedup_bound_free_sweeps": t_seq / t_fine_batches,
            "final_max_dq_vs_sequential_A": float((qend - ref[0, :3]).abs().max().item())}


def _energy_path(P, torch, tq, box, tbeta, snaps, reps=5):
    """SNAP energies and dE/dbeta without forces (U_tot pass, bispectrum B, energy sums: the path of
    the autograd forward and of the beta-fit design rows) on the batch's start states, per
    precision: CUDA-event time per call on the current stream after one warm-up call, and the
    bispectrum's algorithmic flops (34 946 Clebsch-Gordan terms x 8 flop per atom at 2J = 8) over
    that time, a lower bound of the path's flop rate (the U pass is not counted)."""
    nb, _, n = tq.shape
    out = {"workload": "%d x %d-atom W+SIA start states of the batch, 2J = 8, energies + dE/dbeta" % (nb, n)}
    for name, s in snaps:
        P.snap_energy_forces(s, tq, box, tbeta, energy=True, forces=False, sumB=True)
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            P.snap_energy_forces(s, tq, box, tbeta, energy=True, forces=False, sumB=True)
            b.record()
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        s.sync_status()
        t = float(np.median(ms))
        out[name] = {"ms_per_call": round(t, 3), "atoms_per_s": nb * n / (t / 1e3),
                     "bispectrum_tflops_lower_bound": round(nb * n * 34946 * 8 / (t / 1e3) / 1e12, 3)}
    return out


def _roofline(flops, k_ms, peak_tf, basis, kernel, measured=None, traffic=None):
    achieved = flops / (k_ms / 1e3) / 1e12
    r = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_tf, 2), "unit": "TFLOP/s",
         "frac": round(achieved / peak_tf, 4), "traffic": traffic, "kernel": kernel, "kernel_ms": round(k_ms, 3),
         "flops_per_launch": flops, "peak_basis": basis}
    if measured:
        r["peak_measured"] = round(measured[0], 2)
        r["frac_of_measured"] = round(achieved / measured[0], 4)
        r["peak_measured_basis"] = measured[1]
    return r


def _timed_launches(P, eng, torch, stream, flush, tq, tv, tL, tids, lp, runs):
    """Runs `runs` propagations of (tq, tv) from the same start, L2 flushed before each; returns
    (step ms, kernel ms) lists from CUDA events on the launching stream."""
    qw, vw = tq.clone(), tv.clone()
    steps, kern = [], []
    eng.profile(True)
    for _ in range(runs):
        qw.copy_(tq)
        vw.copy_(tv)
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        eng.baoab_propagate_batch(P.FINE, qw, vw, tL, tids, lp)
        b.record(stream)
        kern.append(eng.profile(True))
        torch.cuda.synchronize()
        steps.append(a.elapsed_time(b))
    eng.profile(False)
    eng.sync_status()
    return steps, kern, qw


def _config3(P, W, dev, torch, stream, flush, per_pair, per_atom, peak32, peak64, meas32, meas64):
    """Config 3: the 2001-atom cell, 32 intervals x 500 steps in FP32-bulk, and the plain-FP64 form
    on the same 32 members with 100 steps each (about 9 s)."""
    q, v, box, beta, L, ids, T = _config3_inputs()
    n = q.shape[2]
    tbeta = torch.as_tensor(beta, device=dev)
    tq, tv = torch.as_tensor(q, device=dev), torch.as_tensor(v, device=dev)
    tids = torch.as_tensor(ids, device=dev)
    lp = P.langevin(dt=DT, gamma=GAMMA, T=T, scheme=P.SCHEME_PAPER, schedule=P.SCHED_ROBUST, seed=61)
    nnb0 = _avg_neighbors(q[:4], box, 4.73)
    out = {"workload": WORKLOAD3}
    for name, prec, steps, runs in (("fp32_bulk", P.FP32_BULK, 500, 2), ("fp64", P.FP64, 100, 1)):
        eng = P.Engine(n, box, P.snap_params(precision=prec), P.fs_params(), beta=tbeta)
        eng.reserve(q.shape[0])
        Ls = np.full(q.shape[0], steps, np.int32)
        tL = torch.as_tensor(Ls, device=dev)
        shape = None
        if prec == P.FP32_BULK:
            shape, _ = eng.autotune(tq, tv, tL, tids, lp, max_steps=32)
        # warm-up with a few steps, then the timed runs
        _timed_launches(P, eng, torch, stream, flush, tq, tv, torch.full_like(tL, 3), tids, lp, 1)
        st_ms, k_ms, qf = _timed_launches(P, eng, torch, stream, flush, tq, tv, tL, tids, lp, runs)
        atom_steps = float(Ls.sum()) * n
        nnb = 0.5 * (nnb0 + _avg_neighbors(qf[:4].cpu().numpy(), box, 4.73))
        flops = float((Ls.astype(np.int64) + 1).sum()) * n * (nnb * per_pair + per_atom)
        km = float(np.mean(k_ms))
        pk, basis = (peak32 if prec == P.FP32_BULK else peak64)
        meas = meas32 if prec == P.FP32_BULK else meas64
        out[name] = {"value": atom_steps / (float(np.mean(st_ms)) / 1e3), "unit": UNIT,
                     "sample": "32 x %d steps (%d atom-steps)%s" % (steps, int(atom_steps),
                                                                    "" if steps == 500 else ", a sample of the 500"),
                     "ms_per_launch": round(float(np.mean(st_ms)), 2),
                     "roofline": _roofline(flops, km, pk, basis,
                                           "k_fine_persistent<%s,8>" % ("float" if prec == P.FP32_BULK else "double"),
                                           measured=meas)}
        if shape is not None:
            out[name]["autotuned_shape"] = shape
    return out


def run_cpu_leg(args):
    res, _, _, _ = _oracle_run(args.cpu_leg, single=True)
    print(json.dumps(res), flush=True)
    return 0


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle as O
    import workloads as W
    q, v, box, beta, L, ids = W.batch_workload(nbatch=NSLAB, T=TEMP)
    pot = O.potential(O.POT_SNAP, beta=beta)
    lp = O.langevin(dt=DT, gamma=GAMMA, T=TEMP, seed=2212, schedule=O.SCHED_ROBUST)
    vals, samples = [], []
    for it in range(args.warmup + args.steps):
        # one bounded sample per step: the first intervals of the batch, their first 20 steps each,
        # grown until the sample runs for a few seconds
        nm = 1
        budget = 2.0 if it < args.warmup else 6.0
        while True:
            qq, vv = q[:nm].copy(), v[:nm].copy()
            Ls = np.minimum(L[:nm], 20).astype(np.int32)
            t0 = time.perf_counter()
            O.propagate(pot, qq, vv, box, Ls, ids[:nm], lp)
            dt = time.perf_counter() - t0
            if dt >= budget / 3 or nm >= NSLAB:
                break
            nm = min(NSLAB, nm * 2)
        if it >= args.warmup:
            vals.append(float(Ls.sum()) * q.shape[2] / dt)
            samples.append("%d of the 64 intervals x 20 steps (%.1f s)" % (nm, dt))
    val = float(np.mean(vals))
    cb = {"value": val, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
          "sample": "; ".join(samples) + " (129 atoms, FP64 oracle, all host cores)"}
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD + " (bounded sample on the host cores)", "l2": "n/a (CPU)"},
           "cpu_baseline": cb, "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args):
    ws, rank, local = _dist()
    single = {}
    want_cpu = rank == 0 and ws == 1 and not args.no_cpu and args.case == "full"
    if want_cpu:
        # fresh interpreters (fork + exec), started before this process touches the GPU
        single = _spawn_single_thread_legs()
    import torch
    import __graft_entry__ as G
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    G.build()
    import paper_2212_10508_gb300 as P
    import workloads as W

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    # measured FMA throughput of this device (the ALU roofline's denominators)
    meas = {"ffma": P.alu_peak(P.PEAK_FFMA, 0.2), "ffma2": P.alu_peak(P.PEAK_FFMA2, 0.2),
            "dfma": P.alu_peak(P.PEAK_DFMA, 0.2)}
    lo, hi = (5, 20) if args.case == "small" else (100, 2000)
    master, id0 = _shard(rank)
    q, v, box, beta, L, ids = W.batch_workload(master=master, nbatch=NSLAB, T=TEMP, lo=lo, hi=hi)
    n = q.shape[2]
    ids = ids + id0
    total_atom_steps = float(L.astype(np.int64).sum()) * n
    lp = P.langevin(dt=DT, gamma=GAMMA, T=TEMP, scheme=P.SCHEME_PAPER, schedule=P.SCHED_ROBUST, seed=2212)
    tq, tv = torch.as_tensor(q, device=dev), torch.as_tensor(v, device=dev)
    tL = torch.as_tensor(L, device=dev)
    tids = torch.as_tensor(ids, device=dev)
    tbeta = torch.as_tensor(beta, device=dev)
    eng = P.Engine(n, box, P.snap_params(precision=P.FP32_BULK), P.fs_params(), beta=tbeta)
    eng.reserve(NSLAB)
    # launch shape of the batched kernel picked by the library's autotuner on this batch
    # (interval lengths scaled to at most 64 steps), before warm-up and graph capture
    t_tune = time.perf_counter()
    if args.no_autotune:
        tuned = eng.tuning()
    else:
        tuned, tuned_ms = eng.autotune(tq, tv, tL, tids, lp, max_steps=64)
    t_tune = time.perf_counter() - t_tune
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # 256 MB > 129 MB L2
    qw, vw = tq.clone(), tv.clone()

    graph = None

    def one(timed):
        qw.copy_(tq)
        vw.copy_(tv)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if graph is not None:
            graph.replay()
        else:
            eng.baoab_propagate_batch(P.FINE, qw, vw, tL, tids, lp)
        e1.record(stream)
        return e0, e1

    for _ in range(args.warmup):
        one(False)
    torch.cuda.synchronize()
    eng.sync_status()
    # capture the whole propagation call (status clear, prologue, position wrap, persistent kernel and
    # the kernel's own timing events) into one CUDA graph and replay it in the timed loop
    graph_note = "captured"
    try:
        eng.profile(True)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            eng.baoab_propagate_batch(P.FINE, qw, vw, tL, tids, lp)
        graph = g
        stream = torch.cuda.current_stream()
        one(False)
        torch.cuda.synchronize()
        eng.sync_status()
    except Exception as exc:   # fall back to direct launches, and say so in the JSON line
        graph = None
        graph_note = "not captured: %s" % (str(exc).splitlines()[0][:160],)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    eng.profile(True)
    evs, kern_ms = [], []
    for _ in range(args.steps):
        evs.append(one(True))
        kern_ms.append(eng.profile(True))
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    eng.profile(False)
    clk = clocks.stop()
    eng.sync_status()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    value, tot_ms, job_atom_steps = _job_rate(float(np.sum(step_ms)), total_atom_steps * args.steps, ws, dev)

    # ---- roofline of the persistent SNAP kernel (FP32 ALU bound): the device's FP32 lanes at the
    # clock sampled during the timed region, beside the measured FMA throughput
    per_pair, per_atom = P.Snap(P.snap_params(precision=P.FP32_BULK)).flop_model()
    qf = qw.cpu().numpy()
    nnb = 0.5 * (_avg_neighbors(q, box, 4.73) + _avg_neighbors(qf, box, 4.73))
    force_evals = float((L.astype(np.int64) + 1).sum()) * n
    flops = force_evals * (nnb * per_pair + per_atom)
    k_ms = float(np.mean(kern_ms))
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or 2070.0
    peak32 = (nsm * 128 * 2 * mhz * 1e6 / 1e12,
              "FP32 ALU: %d SMs x 128 lanes x 2 flop x %.0f MHz (median SM clock sampled in the timed region)"
              % (nsm, mhz))
    best32 = max(meas["ffma"], meas["ffma2"])
    meas32 = (best32, "pmd_alu_peak: FP32 FMA microbenchmark on this device (FFMA %.1f, FFMA2 %.1f TFLOP/s)"
              % (meas["ffma"], meas["ffma2"]))
    # the FP64 path's denominator: the measured DFMA throughput (the nominal 1.25 TFLOP/s of this
    # part is the datasheet's)
    peak64 = (meas["dfma"], "FP64: pmd_alu_peak DFMA microbenchmark on this device (datasheet 1.25 TFLOP/s)")
    meas64 = (meas["dfma"], "pmd_alu_peak DFMA")
    traffic = TRAFFIC["bytes_per_launch"] if (args.case == "full" and
                                             _csrc_fingerprint() == TRAFFIC["csrc_sha256_16"]) else None
    roof = _roofline(flops, k_ms, peak32[0], peak32[1], "k_fine_persistent<float,8>", measured=meas32,
                     traffic=traffic)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD if args.case == "full" else SMALL, "precision": "FP32-bulk SNAP (FP64 energy sums, double-float force sums; FP64 positions, velocities, noise)",
                      "slabs_per_gpu": NSLAB, "atoms": n, "atom_steps_per_step": job_atom_steps / args.steps,
                      "l2": "flushed (256 MB write) before every timed step",
                      "autotuned_shape": tuned, "autotune_s": round(t_tune, 2)},
           "roofline": roof, "clocks": clk, "gpu_launches": 3 * args.steps, "cuda_graph": graph_note,
           "alu_peaks_measured_tflops": {k: round(x, 2) for k, x in meas.items()}}
    if rank == 0 and not args.no_parareal:   # one-GPU extras run on rank 0 only
        out["parareal"] = _parareal(P, W, dev, torch)                              # one window of 300
        out["parareal_windows_100"] = _parareal(P, W, dev, torch, window=100)     # three windows of 100
        out["parareal_windows_1000"] = _parareal(P, W, dev, torch, Nh=1000, window=1000)   # one window of 1000
        out["parareal_strategy1_windows_100"] = _parareal(P, W, dev, torch, window=100, strategy=1)

    # ---- matched force error FP32-bulk vs FP64 and the plain-FP64 form on the same workload
    s64 = P.Snap(P.snap_params(precision=P.FP64))
    s32 = P.Snap(P.snap_params(precision=P.FP32_BULK))
    _, F64, _ = P.snap_energy_forces(s64, tq, box, tbeta)
    _, F32, _ = P.snap_energy_forces(s32, tq, box, tbeta)
    ferr = float(((F32 - F64).abs().max() / F64.abs().max()).item())
    out["fp32_force_rel_err_vs_fp64"] = ferr
    if rank == 0:
        out["energy_path"] = _energy_path(P, torch, tq, box, tbeta, (("fp32_bulk", s32), ("fp64", s64)))
    if rank == 0 and not args.no_fp64:
        e64 = P.Engine(n, box, P.snap_params(precision=P.FP64), P.fs_params(), beta=tbeta)
        e64.reserve(NSLAB)
        L64w = np.maximum(1, L // 100).astype(np.int32)
        _timed_launches(P, e64, torch, stream, flush, tq, tv, torch.as_tensor(L64w, device=dev), tids, lp, 1)
        ms64, k64, _ = _timed_launches(P, e64, torch, stream, flush, tq, tv, tL, tids, lp, 1)
        v64 = total_atom_steps / (np.mean(ms64) / 1e3)
        out["fp64"] = {"value": v64, "unit": UNIT,
                       "speedup_fp32_bulk": (total_atom_steps * args.steps / (float(np.sum(step_ms)) / 1e3)) / v64,
                       "sample": "the same 64 intervals with the same lengths L_b (%d atom-steps), one timed launch"
                                 % int(total_atom_steps),
                       "ms_per_launch": round(float(np.mean(ms64)), 1),
                       "roofline": _roofline(flops, float(np.mean(k64)), peak64[0], peak64[1],
                                             "k_fine_persistent<double,8>")}
    if rank == 0 and not args.no_config3 and args.case == "full":
        out["config3"] = _config3(P, W, dev, torch, stream, flush, per_pair, per_atom, peak32, peak64, meas32,
                                  meas64)

    # ---- end to end through the C ABI from pinned host buffers
    hq = torch.as_tensor(q).pin_memory()
    hv = torch.as_tensor(v).pin_memory()
    hL = torch.as_tensor(L).pin_memory()
    hids = torch.as_tensor(ids).pin_memory()
    oq, ov = torch.empty_like(hq).pin_memory(), torch.empty_like(hv).pin_memory()
    dq, dv = torch.empty_like(tq), torch.empty_like(tv)
    dL, dids = torch.empty_like(tL), torch.empty_like(tids)
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dq.copy_(hq, non_blocking=True)
        dv.copy_(hv, non_blocking=True)
        dL.copy_(hL, non_blocking=True)
        dids.copy_(hids, non_blocking=True)
        eng.baoab_propagate_batch(P.FINE, dq, dv, dL, dids, lp)
        oq.copy_(dq, non_blocking=True)
        ov.copy_(dv, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    eng.sync_status()
    h2d = hq.numel() * 8 + hv.numel() * 8 + hL.numel() * 4 + hids.numel() * 8
    d2h = oq.numel() * 8 + ov.numel() * 8
    if ws > 1:
        torch.distributed.barrier()
    e2e_value, _, _ = _job_rate(float(np.sum(e2e_ms)), total_atom_steps * len(e2e_ms), ws, dev)
    out["e2e"] = {"value": e2e_value, "unit": UNIT,
                  "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    if want_cpu:
        st = _collect(single)          # the single-thread legs ran alongside the GPU legs
        legs = {}
        for cfg in sorted(CPU_SAMPLES):   # then the all-core legs, alone on the host
            legs[cfg] = _oracle_run(cfg)
        res2, q1, v1, (q0, v0, box0, beta0, Ls, sids, T2) = legs["cfg2"]

        # GPU FP32-bulk and FP64 results on the oracle's config 2 sample: trajectory (max |dq| in A
        # after the sample's steps) and, on its first start configuration, energy and force errors
        import oracle as O
        err = {}
        dq0, dv0 = torch.as_tensor(q0, device=dev), torch.as_tensor(v0, device=dev)
        dLs, dids0 = torch.as_tensor(Ls, device=dev), torch.as_tensor(sids, device=dev)
        E_o, F_o, _ = O.snap_energy_forces(q0[:1], box0, beta0)
        for name, prec in (("fp32_bulk", P.FP32_BULK), ("fp64", P.FP64)):
            e = P.Engine(n, box0, P.snap_params(precision=prec), P.fs_params(), beta=tbeta)
            qq, vv = dq0.clone(), dv0.clone()
            e.baoab_propagate_batch(P.FINE, qq, vv, dLs, dids0, lp)
            e.sync_status()
            err[name + "_traj_max_dq_A"] = float(np.abs(qq.cpu().numpy() - q1).max())
            err[name + "_traj_max_dv_rel"] = float(np.abs(vv.cpu().numpy() - v1).max() / np.abs(v1).max())
            E_g, F_g, _ = P.snap_energy_forces(P.Snap(P.snap_params(precision=prec)), dq0[:1], box0, tbeta)
            err[name + "_energy_rel"] = float(abs(E_g.cpu().numpy()[0] - E_o[0]) / abs(E_o[0]))
            err[name + "_force_rel_max"] = float(np.abs(F_g.cpu().numpy() - F_o).max() / np.abs(F_o).max())
        err["steps"] = int(Ls.max())
        cb = dict(res2)
        cb["sample"] = res2["sample"] + " on %d threads" % res2["cores"]
        cb["errors_vs_oracle"] = err
        cb["single_thread"] = st.get("cfg2")
        cb["config3"] = {"all_cores": legs["cfg3"][0], "single_thread": st.get("cfg3")}
        out["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.cpu_leg:
        return run_cpu_leg(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
