#!/usr/bin/env python3
"""Throughput of the batched fine propagator (SNAP 2J = 8 Langevin steps for all parareal
intervals in one persistent launch) on GB300, with the plain-FP64 form, the oracle on the
host cores, the roofline of the dominant kernel and an end-to-end number through the C ABI.

Workload (one "step"): 64 intervals of the 129-atom W + SIA cell (4^3 BCC cells + a <111>
dumbbell), SNAP coefficients fitted to Finnis-Sinclair tungsten (tests/golden/beta_fs_w_2j8.txt;
random coefficients collapse the cell), interval lengths L_b ~ U{100..2000}, 1500 K, dt = 1 fs, gamma = 1/ps, paper scheme with the robust
temperature schedule; the whole batch is advanced by one baoab_propagate_batch(FINE) call
(FP32-bulk SNAP: U/Z/Y in FP32, energy sums in FP64, force sums in double-float; FP64 positions,
velocities and noise).

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
# DRAM bytes (read + write) of one full-size launch of the persistent FP32 kernel, from one ncu
# capture of this workload (profiles/fine_persistent_batch64_dram.md), valid only for the kernel
# sources it was taken on (fingerprint of the persistent kernel's translation unit and of the host
# code that builds its tables); reported as null otherwise.
TRAFFIC = {"bytes_per_launch": 3.47e6 + 45.87e6, "csrc_sha256_16": "cf52c70b9164b7bc"}


KERNEL_SOURCES = ("propagate.cu", "snap.cu", "snap_kernels.cuh", "snap_batch.cuh", "snap_v2.cuh", "snap_device.cuh",
                  "device_common.cuh", "langevin_device.cuh", "eam_device.cuh", "pmd_internal.h", "status_bits.h")


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
    ap.add_argument("--case", default="full", choices=["full", "small"],
                    help="small: L_b ~ U{5..20} (a short launch for ncu captures)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the engine's default launch shape (profiling captures count launches)")
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


def _cpu_baseline(q, v, box, beta, L, ids, budget_s=12.0, compare=None):
    """The oracle as it stands on the host cores: first members of the batch, first 20 steps each,
    growing the sample until it has run for about budget_s.  compare(q0, v0, Ls, ids, q1, v1, O), if
    given, receives the sample's inputs and the oracle's final states and returns the GPU results'
    errors against the oracle (reported with the baseline)."""
    import oracle as O
    pot = O.potential(O.POT_SNAP, beta=beta)
    lp = O.langevin(dt=DT, gamma=GAMMA, T=TEMP, seed=2212, schedule=O.SCHED_ROBUST)
    nm, steps = 1, 20
    while True:
        qq, vv = q[:nm].copy(), v[:nm].copy()
        Ls = np.minimum(L[:nm], steps).astype(np.int32)
        t0 = time.perf_counter()
        O.propagate(pot, qq, vv, box, Ls, ids[:nm], lp)
        dt = time.perf_counter() - t0
        if dt >= budget_s / 3 or nm >= q.shape[0]:
            atom_steps = float(Ls.sum()) * q.shape[2]
            res = {"value": atom_steps / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                   "sample": "%d of the 64 intervals x %d steps each (129 atoms, FP64 oracle, %.1f s)"
                             % (nm, steps, dt)}
            if compare is not None:
                res["errors_vs_oracle"] = compare(q[:nm], v[:nm], Ls, ids[:nm], qq, vv, O)
            return res
        nm = min(q.shape[0], nm * 2)


def _parareal(P, W, dev, torch, Nh=300, ncell=5, T=1500.0):
    """Adaptive parareal (Algorithm 2) on a 251-atom cell vs the same N intervals run one after
    the other with the fine propagator (the paper's sequential cost N C_f), on this GPU."""
    pos, box = W.bcc_sia(ncell)
    n = pos.shape[1]
    beta = torch.as_tensor(W.fitted_beta(), device=dev)
    q0 = torch.as_tensor(W.displaced(pos, 0.05, W.rng(5, 1)), device=dev)
    v0 = torch.as_tensor(W.velocities(n, T, W.rng(5, 2)), device=dev)
    eng = P.Engine(n, box, P.snap_params(precision=P.FP32_BULK), P.fs_params(precision=P.FP32_BULK), beta=beta)
    eng.reserve(Nh)
    lp = P.langevin(dt=1e-3, gamma=1.0, T=T, scheme=P.SCHEME_PAPER, schedule=P.SCHED_L1_SYM, seed=77)
    L, dconv, dexpl = 1, 1e-3, 0.1
    one = torch.ones(1, dtype=torch.int32, device=dev)
    ids = torch.arange(Nh, dtype=torch.int64, device=dev)

    def sequential():
        st = torch.empty(1, 6, n, dtype=torch.float64, device=dev)
        st[0, :3], st[0, 3:] = q0, v0
        for k in range(Nh):
            eng.baoab_propagate_batch(P.FINE, st, None, one, ids[k:k + 1], lp)
        return st

    sequential()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ref = sequential()
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    P.adaptive_parareal(eng, q0, v0, 20, L, dconv, dexpl, lp, metric=P.METRIC_MAXDISP)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cur, st = P.adaptive_parareal(eng, q0, v0, Nh, L, dconv, dexpl, lp, metric=P.METRIC_MAXDISP)
    torch.cuda.synchronize()
    t_par = time.perf_counter() - t0
    eng.sync_status()
    # coarse cost per interval: one sweep over the horizon
    cache = torch.empty(Nh, 6, n, dtype=torch.float64, device=dev)
    tmp = cur.clone()
    t0 = time.perf_counter()
    eng.parareal_correct(0, Nh, None, tmp, tmp, cache, float("inf"), P.METRIC_MAXDISP, L, lp)
    t_c = (time.perf_counter() - t0) / Nh
    t_f = t_seq / Nh
    cost, g_ad, g_id = st.cost(t_f, t_c)
    log = st.log()
    return {"workload": "251-atom W+SIA (5^3 cells), SNAP 2J=8 fitted (FP32-bulk) fine, FS EAM (FP32-bulk) coarse, "
                        "dt 1 fs, L=1, 1500 K, gamma 1/ps, schedule C0=C1=2, N=%d intervals" % Nh,
            "delta_conv_A": dconv, "delta_expl_A": dexpl, "metric": "max per-atom displacement (A)",
            "wall_sequential_s": t_seq, "wall_parareal_s": t_par, "speedup": t_seq / t_par,
            "n_slab": (log[-1][3] + 1) if log else 0, "iterations": int(sum(e[2] for e in log)),
            "C_f_ms": t_f * 1e3, "C_c_ms": t_c * 1e3, "gamma_adapt_eq8": g_ad, "gamma_ideal_eq9": g_id,
            "final_max_dq_vs_sequential_A": float((cur[Nh, :3] - ref[0, :3]).abs().max().item())}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import workloads as W
    q, v, box, beta, L, ids = W.batch_workload(nbatch=NSLAB, T=TEMP)
    times, atom_steps = [], 0.0
    cb = None
    for it in range(args.warmup + args.steps):
        cb = _cpu_baseline(q, v, box, beta, L, ids, budget_s=6.0 if it < args.warmup else 9.0)
        if it >= args.warmup:
            times.append(cb["value"])
    val = float(np.mean(times))
    cb["value"] = val
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD + " (bounded sample on the host cores)", "l2": "n/a (CPU)"},
           "cpu_baseline": cb, "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def run_ours(args):
    import torch
    import __graft_entry__ as G
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    G.build()
    import paper_2212_10508_gb300 as P
    import workloads as W

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
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
    stream = torch.cuda.current_stream()
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

    # ---- roofline of the persistent SNAP kernel (FP32 ALU bound)
    per_pair, per_atom = P.Snap(P.snap_params(precision=P.FP32_BULK)).flop_model()
    qf = qw.cpu().numpy()
    nnb = 0.5 * (_avg_neighbors(q, box, 4.73) + _avg_neighbors(qf, box, 4.73))
    force_evals = float((L.astype(np.int64) + 1).sum()) * n
    flops = force_evals * (nnb * per_pair + per_atom)
    k_ms = float(np.mean(kern_ms))
    achieved = flops / (k_ms / 1e3) / 1e12
    sm_clock = 2070.0
    peak = 152 * 128 * 2 * sm_clock * 1e6 / 1e12
    roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4),
            "traffic": TRAFFIC["bytes_per_launch"] if (args.case == "full" and
                                                       _csrc_fingerprint() == TRAFFIC["csrc_sha256_16"]) else None,
            "kernel": "k_fine_persistent<float,8>", "kernel_ms": round(k_ms, 3),
            "flops_per_launch": flops, "peak_basis": "FP32 ALU: 152 SMs x 128 lanes x 2 flop x 2070 MHz"}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD if args.case == "full" else SMALL, "precision": "FP32-bulk SNAP (FP64 energy sums, double-float force sums; FP64 positions, velocities, noise)",
                      "slabs_per_gpu": NSLAB, "atoms": n, "atom_steps_per_step": job_atom_steps / args.steps,
                      "l2": "flushed (256 MB write) before every timed step",
                      "autotuned_shape": tuned, "autotune_s": round(t_tune, 2)},
           "roofline": roof, "clocks": clk, "gpu_launches": 3 * args.steps, "cuda_graph": graph_note}
    if rank == 0:   # one-GPU extras (single-system parareal, FP64 form) run on rank 0 only
        out["parareal"] = _parareal(P, W, dev, torch)

    # ---- matched force error FP32-bulk vs FP64 and the plain-FP64 form
    s64 = P.Snap(P.snap_params(precision=P.FP64))
    s32 = P.Snap(P.snap_params(precision=P.FP32_BULK))
    _, F64, _ = P.snap_energy_forces(s64, tq, box, tbeta)
    _, F32, _ = P.snap_energy_forces(s32, tq, box, tbeta)
    ferr = float(((F32 - F64).abs().max() / F64.abs().max()).item())
    out["fp32_force_rel_err_vs_fp64"] = ferr
    if rank == 0 and not args.no_fp64:
        L64 = np.maximum(1, L // 20).astype(np.int32)
        e64 = P.Engine(n, box, P.snap_params(precision=P.FP64), P.fs_params(), beta=tbeta)
        e64.reserve(NSLAB)
        tL64 = torch.as_tensor(L64, device=dev)
        q6, v6 = tq.clone(), tv.clone()
        e64.baoab_propagate_batch(P.FINE, q6, v6, tL64, tids, lp)
        torch.cuda.synchronize()
        ms64 = []
        for _ in range(2):
            q6.copy_(tq)
            v6.copy_(tv)
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            e64.baoab_propagate_batch(P.FINE, q6, v6, tL64, tids, lp)
            b.record(stream)
            torch.cuda.synchronize()
            ms64.append(a.elapsed_time(b))
        e64.sync_status()
        v64 = float(L64.sum()) * n / (np.mean(ms64) / 1e3)
        out["fp64"] = {"value": v64, "unit": UNIT, "speedup_fp32_bulk": (total_atom_steps * args.steps / (
                           float(np.sum(step_ms)) / 1e3)) / v64,
                       "sample": "same 64 intervals with L_b/20 steps (%d atom-steps)" % int(L64.sum() * n)}

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

    if rank == 0 and ws == 1 and not args.no_cpu:
        def compare(q0, v0, Ls, sids, q1, v1, O):
            """GPU FP32-bulk and FP64 results on the oracle's sample: trajectory (max |dq| in A after the
            sample's steps) and, on member 0's start configuration, energy and force relative errors."""
            err = {}
            dq0 = torch.as_tensor(q0, device=dev)
            dv0 = torch.as_tensor(v0, device=dev)
            dL = torch.as_tensor(Ls, device=dev)
            dids = torch.as_tensor(sids, device=dev)
            E_o, F_o, _ = O.snap_energy_forces(q0[:1], box, beta)
            for name, prec in (("fp32_bulk", P.FP32_BULK), ("fp64", P.FP64)):
                e = P.Engine(n, box, P.snap_params(precision=prec), P.fs_params(), beta=tbeta)
                qq, vv = dq0.clone(), dv0.clone()
                e.baoab_propagate_batch(P.FINE, qq, vv, dL, dids, lp)
                e.sync_status()
                err[name + "_traj_max_dq_A"] = float(np.abs(qq.cpu().numpy() - q1).max())
                err[name + "_traj_max_dv_rel"] = float(np.abs(vv.cpu().numpy() - v1).max() / np.abs(v1).max())
                E_g, F_g, _ = P.snap_energy_forces(P.Snap(P.snap_params(precision=prec)), dq0[:1], box, tbeta)
                err[name + "_energy_rel"] = float(abs(E_g.cpu().numpy()[0] - E_o[0]) / abs(E_o[0]))
                err[name + "_force_rel_max"] = float(np.abs(F_g.cpu().numpy() - F_o).max() / np.abs(F_o).max())
            err["steps"] = int(Ls.max())
            return err
        out["cpu_baseline"] = _cpu_baseline(q, v, box, beta, L, ids, compare=compare)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
