"""Residence times of the self-interstitial along a sequential and an adaptive-parareal trajectory
(Sec. 3: the interstitial's wells, their residence times in units of the time step, the mean with
a 95 % confidence interval), on the GPU through the library.

    python -m paper_2212_10508_gb300.residence [--T 2000] [--steps 20000] [--window 1000] [--equil 2000]

The horizon is cut into windows of `window` intervals of one step (L = 1); each window is run by
Algorithm 2 from the parareal trajectory's state and, for the reference, by the fine propagator
alone from the sequential trajectory's state.  Window w draws its noise with seed + w and interval
ids 0 .. window - 1 on both sides, so the two trajectories share every Gaussian increment and
differ only through the parareal tolerance.  The interstitial's well in every
frame comes from sia_locate (Wigner-Seitz reading of the Voronoi analysis), the residence times
from sia_residence.  Prints one JSON line.  Run it from the repository root: the seeded inputs
(lattice, fitted coefficients, velocities) come from the `workloads` module there.
"""
import argparse
import json
import time

import numpy as np


def sequential(engine, q0, v0, nsteps, lp, id0=0):
    """The fine propagator applied interval by interval (L = 1, interval id = id0 + step): the
    states [nsteps + 1, 6, n] after every step."""
    import torch
    from . import FINE
    n = engine.natoms
    st = torch.empty(nsteps + 1, 6, n, dtype=torch.float64, device=q0.device)
    st[0, :3] = q0
    st[0, 3:] = v0
    one = torch.ones(1, dtype=torch.int32, device=q0.device)
    ids = torch.arange(id0, id0 + nsteps, dtype=torch.int64, device=q0.device)
    for k in range(nsteps):
        st[k + 1] = st[k]
        engine.baoab_propagate_batch(FINE, st[k + 1:k + 2], None, one, ids[k:k + 1], lp)
    engine.sync_status()
    return st


def mean_ci95(lengths):
    x = np.asarray(lengths, dtype=np.float64)
    if x.size == 0:
        return None, None
    s = x.std(ddof=1) if x.size > 1 else 0.0
    return float(x.mean()), float(1.96 * s / np.sqrt(x.size))


T975 = {1: 12.706, 2: 4.303, 3: 3.182, 4: 2.776, 5: 2.571, 6: 2.447, 7: 2.365, 8: 2.306, 9: 2.262, 19: 2.093}


def batch_means(lengths, nframes, blocks=10):
    """Mean residence time with a 95 % interval from batch means: the trajectory's frames are cut
    into `blocks` equal blocks, each residence time is assigned to the block where it ends, and
    the interval is mean +- t(0.975, blocks - 1) s / sqrt(blocks) over the block means.  Unlike
    mean +- 1.96 s / sqrt(m) over the m residence times, it stays valid when successive residence
    times are correlated (slow switches of the interstitial between states of different
    mobility).  Returns (mean of block means, half-width, block means)."""
    x = np.asarray(lengths, dtype=np.int64)
    ends = np.cumsum(x)
    blk = np.minimum(ends * blocks // max(int(nframes), 1), blocks - 1)
    means = np.array([x[blk == b].mean() if np.any(blk == b) else np.nan for b in range(blocks)])
    means = means[np.isfinite(means)]
    if means.size < 2:
        return (float(means.mean()) if means.size else None), None, means.tolist()
    t = T975.get(means.size - 1, 1.96)
    return float(means.mean()), float(t * means.std(ddof=1) / np.sqrt(means.size)), means.tolist()


def summary(states, sites, box, ref):
    """Wells, residence times (steps), mean and 95 % half-width, histogram (50-step bins)."""
    from . import sia_locate, sia_residence
    well, occ = sia_locate(states, ref, sites, box)
    lengths, _ = sia_residence(well)
    m, h = mean_ci95(lengths)
    bm, bh, blocks = batch_means(lengths, well.shape[0])
    hist, edges = np.histogram(lengths, bins=np.arange(0, max(int(lengths.max()) if lengths.size else 0, 50) + 50, 50))
    return {"exits": int(lengths.size), "mean_steps": m, "ci95_half_width": h,
            "batch_means_mean_steps": bm, "batch_means_ci95_half_width": bh, "block_means_steps": blocks,
            "histogram_50_step_bins": hist.tolist(), "max_occupancy": int(occ.max().item()),
            "frames_with_one_doubly_occupied_site": float((occ == 2).float().mean().item())}


def study(T=2000.0, steps=20000, window=1000, equil=2000, delta_conv=1e-3, delta_expl=0.1, ncell=5, seed=2212):
    import torch
    import workloads as W
    from . import (FP32_BULK, METRIC_MAXDISP, SCHED_L1_SYM, SCHEME_PAPER, Engine, adaptive_parareal, fs_params,
                   langevin, snap_params)
    dev = torch.device("cuda", 0)
    pos, box = W.bcc_sia(ncell)
    sites, _ = W.bcc(ncell)
    n = pos.shape[1]
    eng = Engine(n, box, snap_params(precision=FP32_BULK), fs_params(precision=FP32_BULK),
                 beta=torch.as_tensor(W.fitted_beta(), device=dev))

    def lp_of(w):
        return langevin(dt=1e-3, gamma=1.0, T=T, scheme=SCHEME_PAPER, schedule=SCHED_L1_SYM, seed=seed + w)

    q = torch.as_tensor(W.displaced(pos, 0.05, W.rng(seed, 1)), device=dev)
    v = torch.as_tensor(W.velocities(n, T, W.rng(seed, 2)), device=dev)
    eq = sequential(eng, q, v, equil, lp_of(-1))             # equilibration: its own noise
    q0, v0 = eq[-1, :3].contiguous(), eq[-1, 3:].contiguous()
    tsites = torch.as_tensor(sites, device=dev)
    nw = steps // window
    seq_parts, par_parts = [eq[-1:]], [eq[-1:]]
    t_seq = t_par = 0.0
    for w in range(nw):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = sequential(eng, seq_parts[-1][-1, :3].contiguous(), seq_parts[-1][-1, 3:].contiguous(), window, lp_of(w))
        torch.cuda.synchronize()
        t_seq += time.perf_counter() - t0
        t0 = time.perf_counter()
        p, _ = adaptive_parareal(eng, par_parts[-1][-1, :3].contiguous(), par_parts[-1][-1, 3:].contiguous(), window,
                                 1, delta_conv, delta_expl, lp_of(w), metric=METRIC_MAXDISP)
        torch.cuda.synchronize()
        t_par += time.perf_counter() - t0
        seq_parts.append(s[1:])
        par_parts.append(p[1:])
    seq = torch.cat(seq_parts)
    par = torch.cat(par_parts)
    dq = float((par[:, :3] - seq[:, :3]).abs().max().item())
    return {"workload": "%d-atom W+SIA, fitted SNAP 2J=8 (FP32-bulk) fine, FS EAM coarse, dt 1 fs, L=1, %.0f K, "
                        "gamma 1/ps, %d steps in windows of %d after %d equilibration steps"
                        % (n, T, nw * window, window, equil),
            "delta_conv_A": delta_conv, "delta_expl_A": delta_expl,
            "sequential": dict(summary(seq, tsites, box, q0), wall_s=t_seq),
            "parareal": dict(summary(par, tsites, box, q0), wall_s=t_par),
            "max_dq_parareal_vs_sequential_A": dq}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--T", type=float, default=2000.0)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--window", type=int, default=1000)
    ap.add_argument("--equil", type=int, default=2000)
    ap.add_argument("--delta-conv", type=float, default=1e-3)
    ap.add_argument("--delta-expl", type=float, default=0.1)
    ap.add_argument("--seed", type=int, default=2212, help="master seed (displacements, velocities, noise)")
    a = ap.parse_args()
    print(json.dumps(dict(study(a.T, a.steps, a.window, a.equil, a.delta_conv, a.delta_expl, seed=a.seed), seed=a.seed)))


if __name__ == "__main__":
    main()
