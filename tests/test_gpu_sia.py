"""Interstitial tracking on the GPU against the oracle: the well and its occupancy in every frame
bit for bit (integer results of FP64 nearest-site decisions taken in the same order on both
sides), on synthetic trajectories, on frames of the library's own Langevin dynamics (positions
rows of [nf, 6, n] states, frame stride 6n) and on the edge cases; residence runs of the C host
function against the oracle's."""
import numpy as np
import pytest
import torch

import oracle.sia as OS
import paper_2212_10508_gb300 as P
import workloads as W
from gpu_util import N, T, dev

pytestmark = pytest.mark.gpu


def _both(frames, ref, sites, box):
    gw, go = P.sia_locate(T(frames), T(ref), T(sites), box)
    torch.cuda.synchronize()
    ow, oo = OS.locate(frames, ref, sites, box)
    return N(gw), N(go), ow, oo


@pytest.mark.parametrize("seed,sigma", [(1, 0.03), (2, 0.08), (3, 0.15)])
def test_synthetic_trajectories(seed, sigma):
    frames, sites, box, wells = W.sia_frames(4, 400, W.rng(40, seed), sigma=sigma, hop=0.05)
    gw, go, ow, oo = _both(frames, frames[0], sites, box)
    assert np.array_equal(gw, ow) and np.array_equal(go, oo)
    if sigma <= 0.03:
        assert np.array_equal(gw, wells)
    gl, gs = P.sia_residence(gw)
    ol, osites = OS.residence(ow)
    assert np.array_equal(gl, ol) and np.array_equal(gs, osites)


def test_larger_cell_and_many_frames():
    frames, sites, box, _ = W.sia_frames(6, 1500, W.rng(41, 1), sigma=0.08, hop=0.02)   # 433 atoms, 432 sites
    gw, go, ow, oo = _both(frames, frames[0], sites, box)
    assert np.array_equal(gw, ow) and np.array_equal(go, oo)


def test_frames_of_langevin_dynamics_with_state_stride():
    """Frames from the library's fine propagator (129-atom cell, 2000 K, fitted SNAP), recorded
    every 5 steps as [nf, 6, n] states: positions are rows 0..2 of each frame."""
    pos, box = W.bcc_sia(4)
    n = pos.shape[1]
    eng = P.Engine(n, box, P.snap_params(precision=P.FP32_BULK), P.fs_params(), beta=T(W.fitted_beta()))
    lp = P.langevin(T=2000.0, seed=9)
    st = torch.empty(60, 6, n, dtype=torch.float64, device=dev())
    st[0, :3] = T(W.displaced(pos, 0.05, W.rng(42, 1)))
    st[0, 3:] = T(W.velocities(n, 2000.0, W.rng(42, 2)))
    for f in range(1, 60):
        s = st[f - 1:f].clone()
        eng.baoab_propagate_batch(P.FINE, s, None, T([5], torch.int32), T([f], torch.int64), lp)
        st[f] = s[0]
    eng.sync_status()
    sites, _ = W.bcc(4)
    gw, go = P.sia_locate(st, st[0, :3].contiguous(), T(sites), box)
    ow, oo = OS.locate(N(st), N(st[0, :3]), sites, box)
    assert np.array_equal(N(gw), ow) and np.array_equal(N(go), oo)
    assert np.all(oo >= 2)


def test_edge_cases():
    sites, box = W.bcc(2)
    q = W.displaced(sites, 0.05, W.rng(43, 1))
    # no frames
    gw, go = P.sia_locate(T(np.zeros((0, 3, q.shape[1]))), T(q), T(sites), box)
    assert gw.numel() == 0
    # one site: every atom on it
    one = sites[:, :1].copy()
    gw, go, ow, oo = _both(q[None], q, one, box)
    assert gw.tolist() == [0] and go.tolist() == [q.shape[1]] and np.array_equal(go, oo)
    # bad arguments are rejected before any launch
    with pytest.raises(P.PmdError):
        P.sia_locate(T(q[None]), T(q), T(np.zeros((3, 0))), box)
    with pytest.raises(P.PmdError):
        P.sia_locate(T(q[None]), T(q), T(sites), [box[0], -1.0, box[2]])
    with pytest.raises(TypeError):
        P.sia_locate(T(q[None]).float(), T(q), T(sites), box)


def test_residence_study_pipeline_tight_tolerance():
    """The windowed study on a short horizon: with a tight parareal tolerance the parareal
    trajectory is the sequential one (shared noise per window), so the wells and residence times
    agree exactly."""
    from paper_2212_10508_gb300 import residence as R
    out = R.study(T=2000.0, steps=200, window=100, equil=50, delta_conv=1e-10, delta_expl=0.1, ncell=4)
    assert out["max_dq_parareal_vs_sequential_A"] < 1e-8
    s, p = out["sequential"], out["parareal"]
    assert s["exits"] == p["exits"] and s["histogram_50_step_bins"] == p["histogram_50_step_bins"]
    assert s["max_occupancy"] >= 2
