"""Full-size launches, checked on sampled outputs and on properties that hold at any size.

1. The bench's workload in the bench's launch configuration: 64 intervals of the 129-atom cell,
   L_b ~ U{100..2000}, fitted SNAP, 1500 K, one persistent FP32-bulk launch.
2. The 2001-atom cell (10^3 cells + SIA), 32 intervals x 500 steps.

Checks: sampled members of the full launch equal, bit for bit, the same members propagated alone
(no atom's arithmetic depends on the rest of the batch); the SNAP forces at the final
configurations of sampled members match the FP64 oracle (FP32-bulk 1e-5, FP64 1e-10, relative
max-norm); the kinetic temperature of the batch stays physical (near the bath temperature once
the run is longer than the thermostat's relaxation time)."""
import numpy as np
import pytest

import oracle as O
import paper_2212_10508_gb300 as P
import workloads as W
from gpu_util import N, T, rel_max, torch
from test_gpu_propagate import fp32_trajectory_bounds

pytestmark = pytest.mark.gpu


def _kinetic_temperature(v):
    """Per-member kinetic temperature of velocities v [nb, 3, n] (Angstrom/ps)."""
    m = W.M_W / W.FTOA                                    # eV ps^2 / Angstrom^2
    return m * np.mean(v * v, axis=(1, 2)) / W.KB


def _full_and_alone(q, v, box, beta, L, ids, T_K, seed, members):
    n = q.shape[2]
    eng = P.Engine(n, box, P.snap_params(precision=P.FP32_BULK), P.fs_params(), beta=T(beta))
    eng.reserve(q.shape[0])
    lp = P.langevin(dt=1e-3, gamma=1.0, T=T_K, scheme=P.SCHEME_PAPER, schedule=P.SCHED_ROBUST, seed=seed)
    gq, gv = T(q), T(v)
    eng.baoab_propagate_batch(P.FINE, gq, gv, T(L, torch.int32), T(ids, torch.int64), lp)
    eng.sync_status()
    for m in members:
        q1, v1 = T(q[m:m + 1]), T(v[m:m + 1])
        eng.baoab_propagate_batch(P.FINE, q1, v1, T(L[m:m + 1], torch.int32), T(ids[m:m + 1], torch.int64), lp)
        eng.sync_status()
        assert torch.equal(q1[0], gq[m]) and torch.equal(v1[0], gv[m]), m
    return N(gq), N(gv)


def _forces_match_oracle(pos, box, beta):
    oE, oF, _ = O.snap_energy_forces(pos, box, beta)
    for prec, tol in ((P.FP64, 1e-10), (P.FP32_BULK, 1e-5)):
        s = P.Snap(P.snap_params(precision=prec))
        E, F, _ = P.snap_energy_forces(s, T(pos), box, T(beta))
        s.sync_status()
        assert rel_max(N(F), oF) <= tol and rel_max(N(E), oE) <= tol, prec


def test_bench_workload_full_size():
    q, v, box, beta, L, ids = W.batch_workload(master=2212, nbatch=64, T=1500.0, lo=100, hi=2000)
    members = [int(np.argmax(L)), int(np.argmin(L)), 31]
    gq, gv = _full_and_alone(q, v, box, beta, L, ids, 1500.0, 2212, members)
    assert np.all(np.isfinite(gq)) and np.all(np.isfinite(gv))
    Tk = _kinetic_temperature(gv)
    assert abs(Tk.mean() - 1500.0) < 0.1 * 1500.0, Tk.mean()
    _forces_match_oracle(gq[members[:2]], box, beta)


def test_2001_atom_cell_full_size():
    pos, box = W.bcc_sia(10)
    n = pos.shape[1]
    q = W.displaced(pos, 0.05, W.rng(61, 1), count=32)
    v = W.velocities(n, 1000.0, W.rng(61, 2), count=32)
    beta = W.fitted_beta()
    L = np.full(32, 500, np.int32)
    ids = np.arange(32, dtype=np.int64)
    gq, gv = _full_and_alone(q, v, box, beta, L, ids, 1000.0, 61, [0, 19])
    # 0.5 ps is half the thermostat's relaxation time 1/gamma: the kinetic energy that flowed into
    # the lattice's potential energy (equipartition) is not yet replaced, so T_kin lies between
    # half the bath temperature and the bath temperature
    Tk = _kinetic_temperature(gv)
    assert 500.0 < Tk.mean() < 1050.0, Tk.mean()
    _forces_match_oracle(gq[:1], box, beta)


@pytest.mark.parametrize("precision", [P.FP64, P.FP32_BULK])
def test_2001_atom_cell_trajectory_matches_oracle(precision):
    """Two members of the 2001-atom cell, 20 and 13 steps at 1000 K with the fitted SNAP, against
    the oracle's trajectory: FP64 to 1e-8 Angstrom; FP32-bulk within the bounds implied by the
    1e-5 force bar."""
    pos, box = W.bcc_sia(10)
    n = pos.shape[1]
    q = W.displaced(pos, 0.05, W.rng(62, 1), count=2)
    v = W.velocities(n, 1000.0, W.rng(62, 2), count=2)
    beta = W.fitted_beta()
    L = np.array([20, 13], np.int32)
    ids = np.array([5, 77], np.int64)
    eng = P.Engine(n, box, P.snap_params(precision=precision), P.fs_params(precision=precision), beta=T(beta))
    lp = P.langevin(dt=1e-3, gamma=1.0, T=1000.0, scheme=P.SCHEME_PAPER, schedule=P.SCHED_ROBUST, seed=62)
    gq, gv = T(q), T(v)
    eng.baoab_propagate_batch(P.FINE, gq, gv, T(L, torch.int32), T(ids, torch.int64), lp)
    eng.sync_status()
    oq, ov = q.copy(), v.copy()
    olp = O.langevin(dt=1e-3, gamma=1.0, T=1000.0, scheme=O.SCHEME_PAPER, schedule=O.SCHED_ROBUST, seed=62)
    O.propagate(O.potential(O.POT_SNAP, beta=beta), oq, ov, box, L, ids, olp)
    dq, dv = np.abs(N(gq) - oq).max(), np.abs(N(gv) - ov).max()
    if precision == P.FP64:
        assert dq < 1e-8 and dv < 1e-6
    else:
        bq, bv = fp32_trajectory_bounds(q[:1], box, beta, 20)
        assert dq < bq and dv < bv
