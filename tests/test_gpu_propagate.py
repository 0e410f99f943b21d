"""GPU parity of baoab_propagate_batch against the oracle: the Langevin schemes of Sec. 2
(eqs. (2)-(3), (11)-(14), and BAOAB) driven by SNAP (FINE) or EAM (COARSE), with uneven
numbers of steps per member in one call and the shared Philox noise keyed by interval.
Bar: FP64 trajectories agree to 1e-8 Angstrom (positions) after up to 100 steps."""
import numpy as np
import pytest

import oracle as O
import paper_2212_10508_gb300 as P
import workloads as W
from gpu_util import N, T, dev, rel_max, torch

pytestmark = pytest.mark.gpu

SCHEMES = {"paper": (P.SCHEME_PAPER, O.SCHEME_PAPER), "baoab": (P.SCHEME_BAOAB, O.SCHEME_BAOAB)}
SCHEDS = {P.SCHED_NONE: O.SCHED_NONE, P.SCHED_ROBUST: O.SCHED_ROBUST, P.SCHED_L1_SYM: O.SCHED_L1_SYM}


def _system(ncell, nb, T_K, master):
    pos, box = W.bcc_sia(ncell)
    q = W.displaced(pos, 0.05, W.rng(master, 1), count=nb)
    v = W.velocities(pos.shape[1], T_K, W.rng(master, 2), count=nb)
    beta = W.snap_beta(55, W.rng(master, 3))
    return q, v, box, beta


def _run_both(potential, q, v, box, beta, L, ids, T_K=1000.0, scheme="paper", schedule=P.SCHED_ROBUST,
              precision=P.FP64, seed=2024):
    n = q.shape[2]
    eng = P.Engine(n, box, P.snap_params(precision=precision), P.fs_params(precision=precision), beta=T(beta))
    lp = P.langevin(dt=1e-3, gamma=1.0, T=T_K, scheme=SCHEMES[scheme][0], schedule=schedule, seed=seed)
    gq, gv = T(q), T(v)
    eng.baoab_propagate_batch(potential, gq, gv, T(L, torch.int32), T(ids, torch.int64), lp)
    eng.sync_status()
    pot = O.potential(O.POT_SNAP, beta=beta) if potential == P.FINE else O.potential(O.POT_FS)
    olp = O.langevin(dt=1e-3, gamma=1.0, T=T_K, scheme=SCHEMES[scheme][1], schedule=SCHEDS[schedule], seed=seed)
    oq, ov = q.copy(), v.copy()
    O.propagate(pot, oq, ov, box, L, ids, olp)
    return N(gq), N(gv), oq, ov


@pytest.mark.parametrize("scheme", ["paper", "baoab"])
def test_coarse_uneven_lengths(scheme):
    q, v, box, beta = _system(4, 8, 1500.0, 11)
    L = np.array([0, 1, 2, 5, 13, 40, 3, 7], dtype=np.int32)
    ids = np.array([5, 0, 17, 3, 2**33 + 1, 9, 8, 1], dtype=np.int64)
    gq, gv, oq, ov = _run_both(P.COARSE, q, v, box, beta, L, ids, scheme=scheme)
    assert np.abs(gq - oq).max() < 1e-9
    assert np.abs(gv - ov).max() < 1e-7
    assert np.array_equal(gq[0], q[0]) and np.array_equal(gv[0], v[0])      # L = 0 is the identity


@pytest.mark.parametrize("scheme", ["paper", "baoab"])
def test_fine_uneven_lengths(scheme):
    q, v, box, beta = _system(4, 4, 1000.0, 12)
    L = np.array([0, 1, 9, 4], dtype=np.int32)
    ids = np.array([3, 1, 0, 7], dtype=np.int64)
    gq, gv, oq, ov = _run_both(P.FINE, q, v, box, beta, L, ids, scheme=scheme)
    assert np.abs(gq - oq).max() < 1e-9
    assert np.abs(gv - ov).max() < 1e-7
    assert np.array_equal(gq[0], q[0])


def test_fine_100_step_trajectory():
    """The 129-atom cell, 100 steps at 1000 K, dt = 1 fs, gamma = 1/ps: positions to 1e-8 Angstrom."""
    q, v, box, beta = _system(4, 1, 1000.0, 13)
    gq, gv, oq, ov = _run_both(P.FINE, q, v, box, beta, np.array([100], np.int32), np.array([42], np.int64))
    assert np.abs(gq - oq).max() < 1e-8
    assert np.abs(gv - ov).max() < 1e-6


@pytest.mark.parametrize("schedule", [P.SCHED_NONE, P.SCHED_L1_SYM])
def test_schedules(schedule):
    q, v, box, beta = _system(4, 3, 2000.0, 14)
    L = np.array([1, 1, 0], dtype=np.int32)
    ids = np.array([0, 1, 2], dtype=np.int64)
    for pot in (P.FINE, P.COARSE):
        gq, gv, oq, ov = _run_both(pot, q, v, box, beta, L, ids, T_K=2000.0, schedule=schedule)
        assert np.abs(gq - oq).max() < 1e-10 and np.abs(gv - ov).max() < 1e-8


def test_l1_sym_rejects_longer_intervals():
    q, v, box, beta = _system(4, 1, 1000.0, 15)
    eng = P.Engine(q.shape[2], box, beta=T(beta))
    lp = P.langevin(schedule=P.SCHED_L1_SYM)
    eng.baoab_propagate_batch(P.FINE, T(q), T(v), T([3], torch.int32), T([0], torch.int64), lp)
    with pytest.raises(P.PmdError) as e:
        eng.sync_status()
    assert e.value.code == P.PMD_EINVAL


def test_fine_fp32_bulk_tracks_fp64():
    q, v, box, beta = _system(4, 2, 1500.0, 16)
    L = np.array([10, 6], dtype=np.int32)
    ids = np.array([4, 5], dtype=np.int64)
    gq, gv, oq, ov = _run_both(P.FINE, q, v, box, beta, L, ids, precision=P.FP32_BULK)
    assert np.abs(gq - oq).max() < 1e-6


def fp32_trajectory_bounds(q0, box, beta, nsteps, dt=1e-3, tol_f=1e-5, growth=2.0):
    """Position and velocity bounds for an FP32-bulk trajectory against the FP64 oracle, from
    the force bar alone: a force error |dF| <= tol_f max|F| (the FP32-bulk force tolerance,
    max-norm relative), with max|F| allowed to grow by `growth` along the run, moves an atom by
    at most (1/2) |dF|/m t^2 and changes its velocity by at most |dF|/m t after t = nsteps dt."""
    _, F0, _ = O.snap_energy_forces(q0, box, beta)
    a = tol_f * growth * np.abs(F0).max() * W.FTOA / W.M_W          # Angstrom / ps^2
    t = nsteps * dt
    return 0.5 * a * t * t, a * t


def test_fine_fp32_bulk_100_step_trajectory():
    """The 129-atom cell with the fitted SNAP, 100 FP32-bulk steps at 1500 K: positions and
    velocities within the bounds that the 1e-5 force bar implies (1.2e-4 Angstrom here)."""
    q, v, box, _ = _system(4, 2, 1500.0, 19)
    beta = W.fitted_beta()
    L = np.array([100, 100], dtype=np.int32)
    ids = np.array([8, 9], dtype=np.int64)
    gq, gv, oq, ov = _run_both(P.FINE, q, v, box, beta, L, ids, T_K=1500.0, precision=P.FP32_BULK)
    bq, bv = fp32_trajectory_bounds(q[:1], box, beta, 100)
    assert bq < 2e-4                     # max|F| = 22 eV/A at the dumbbell: bq = 1.2e-4 A
    assert np.abs(gq - oq).max() < bq
    assert np.abs(gv - ov).max() < bv


def test_noise_is_shared_between_fine_and_coarse_zero_force():
    """With gamma > 0 and both potentials switched off (beta = 0 and FS A = pair = 0) the two
    propagators see the same G_{l,n}: their trajectories coincide exactly."""
    q, v, box, beta = _system(4, 3, 1000.0, 17)
    n = q.shape[2]
    beta0 = np.zeros_like(beta)
    eng = P.Engine(n, box, P.snap_params(), P.fs_params(A=0.0, c0=0.0, c1=0.0, c2=0.0), beta=T(beta0))
    lp = P.langevin(T=1000.0, seed=99)
    L = T([4, 2, 7], torch.int32)
    ids = T([10, 11, 12], torch.int64)
    q1, v1, q2, v2 = T(q), T(v), T(q), T(v)
    eng.baoab_propagate_batch(P.FINE, q1, v1, L, ids, lp)
    eng.baoab_propagate_batch(P.COARSE, q2, v2, L, ids, lp)
    eng.sync_status()
    assert torch.equal(q1, q2) and torch.equal(v1, v2)


def test_fine_propagation_replays_from_a_cuda_graph():
    """The whole baoab_propagate_batch(FINE) call (prologue, persistent cooperative kernel) is
    captured once into a CUDA graph; replays give the direct call's result bit for bit."""
    q, v, box, beta = _system(4, 6, 1500.0, 18)
    n = q.shape[2]
    eng = P.Engine(n, box, P.snap_params(precision=P.FP32_BULK), P.fs_params(), beta=T(W.fitted_beta()))
    eng.reserve(6)
    lp = P.langevin(T=1500.0, seed=5)
    L = T([7, 3, 0, 12, 5, 9], torch.int32)
    ids = T(np.arange(6), torch.int64)
    q1, v1 = T(q), T(v)
    eng.baoab_propagate_batch(P.FINE, q1, v1, L, ids, lp)
    eng.sync_status()
    qg, vg = T(q), T(v)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        eng.baoab_propagate_batch(P.FINE, qg, vg, L, ids, lp)
    for _ in range(2):
        qg.copy_(T(q))
        vg.copy_(T(v))
        g.replay()
        torch.cuda.synchronize()
        eng.sync_status()
        assert torch.equal(qg, q1) and torch.equal(vg, v1)


def test_bounded_waits_time_out_and_engine_stays_usable():
    """The cross-CTA waits give up after their poll limit with ETIMEOUT (a counter nothing
    increments, a grid barrier missing a CTA), and the engine then propagates as before."""
    q, v, box, beta = _system(4, 2, 1000.0, 16)
    L = np.array([3, 2], dtype=np.int32)
    ids = np.array([5, 6], dtype=np.int64)
    eng = P.Engine(q.shape[2], box, beta=T(beta))
    lp = P.langevin(T=1000.0)
    q1, v1 = T(q), T(v)
    eng.baoab_propagate_batch(P.FINE, q1, v1, T(L, torch.int32), T(ids, torch.int64), lp)
    eng.sync_status()
    eng.selftest_waits(polls=1000)
    with pytest.raises(P.PmdError) as e:
        eng.sync_status()
    assert e.value.code == P.PMD_ETIMEOUT
    eng.sync_status()   # cleared
    q2, v2 = T(q), T(v)
    eng.baoab_propagate_batch(P.FINE, q2, v2, T(L, torch.int32), T(ids, torch.int64), lp)
    eng.sync_status()
    assert torch.equal(q1, q2) and torch.equal(v1, v2)
    with pytest.raises(P.PmdError):
        eng.selftest_waits(polls=0)


def test_mistyped_step_counts_and_ids_are_rejected():
    """The binding checks element types before anything is launched (the C ABI reads the bytes
    as int32 step counts and int64 interval ids)."""
    q, v, box, beta = _system(4, 2, 1000.0, 17)
    eng = P.Engine(q.shape[2], box, beta=T(beta))
    lp = P.langevin(T=1000.0)
    gq, gv = T(q), T(v)
    for L, ids in ((T([3, 2]), T([5, 6], torch.int64)), (T([3, 2], torch.int32), T([5, 6], torch.int32))):
        with pytest.raises(TypeError):
            eng.baoab_propagate_batch(P.FINE, gq, gv, L, ids, lp)
    assert torch.equal(gq, T(q)) and torch.equal(gv, T(v))


def _cluster(natoms, box_len, gen, dmin=2.3, spread=5.0):
    pts = [np.full(3, box_len / 2)]
    while len(pts) < natoms:
        p = box_len / 2 + gen.uniform(-spread, spread, 3)
        if all(np.linalg.norm(p - q) > dmin for q in pts):
            pts.append(p)
    return np.array(pts).T


@pytest.mark.parametrize("natoms,nb", [(2, 2000), (17, 300)])
def test_fp32_batches_spanning_many_members(natoms, nb):
    """Tiny systems, many members: a batch of the FP32 kernel holds atoms of up to ~14 members and
    a phase-B group of more; every member still matches the oracle."""
    gen = W.rng(71, natoms)
    box = np.full(3, 20.0)
    base = _cluster(natoms, 20.0, gen)
    q = np.ascontiguousarray(base[None] + gen.normal(0.0, 0.05, size=(nb, 3, natoms)))
    v = W.velocities(natoms, 1000.0, W.rng(71, 100 + natoms), count=nb)
    beta = W.fitted_beta()
    L = W.rng(71, 200 + natoms).integers(0, 6, size=nb).astype(np.int32)
    ids = np.arange(nb, dtype=np.int64)
    gq, gv, oq, ov = _run_both(P.FINE, q, v, box, beta, L, ids, precision=P.FP32_BULK)
    assert np.abs(gq - oq).max() < 1e-6
    assert np.abs(gv - ov).max() < 1e-3
