"""Strategy I of the paper (Sec. 3): SNAP-6 (2J = 2) as the coarse propagator of a larger SNAP
fine potential, on the GPU against the oracle.

1. The coarse propagator alone (baoab_propagate_batch(COARSE) with the engine's SNAP coarse
   potential: one CTA per interval, thread per atom) against the oracle's propagation with the
   same SNAP-6, uneven lengths, both schemes: FP64 to 1e-9 Angstrom, FP32-bulk within the bound
   its 1e-5 force bar implies.
2. Adaptive parareal (Algorithm 2) with SNAP 2J = 8 fine and SNAP-6 coarse against the oracle's
   Algorithm 2 with the same two potentials: identical slabs and iteration counts, trajectories
   to 1e-8 Angstrom.
Coefficients: both potentials fitted to Finnis-Sinclair W by the oracle (tests/golden)."""
import numpy as np
import pytest

import oracle as O
from oracle import parareal as PR
import paper_2212_10508_gb300 as P
import workloads as W
from gpu_util import N, T, torch
from test_gpu_propagate import fp32_trajectory_bounds

pytestmark = pytest.mark.gpu

SCHEMES = {"paper": (P.SCHEME_PAPER, O.SCHEME_PAPER), "baoab": (P.SCHEME_BAOAB, O.SCHEME_BAOAB)}


def _engine(n, box, precision=P.FP64):
    return P.Engine(n, box, P.snap_params(precision=precision), coarse_snap=P.snap_params(twojmax=2, precision=precision),
                    beta=T(W.fitted_beta(8)), coarse_beta=T(W.fitted_beta(2)))


def _snap6():
    return O.potential(O.POT_SNAP, beta=W.fitted_beta(2), snap=O.snap_params(twojmax=2))


@pytest.mark.parametrize("scheme", ["paper", "baoab"])
@pytest.mark.parametrize("precision", [P.FP64, P.FP32_BULK])
def test_snap6_coarse_propagation_matches_oracle(scheme, precision):
    pos, box = W.bcc_sia(4)
    n = pos.shape[1]
    q = W.displaced(pos, 0.05, W.rng(71, 1), count=6)
    v = W.velocities(n, 1500.0, W.rng(71, 2), count=6)
    L = np.array([0, 1, 3, 17, 40, 8], np.int32)
    ids = np.array([4, 0, 9, 2**33 + 5, 11, 3], np.int64)
    eng = _engine(n, box, precision)
    lp = P.langevin(dt=1e-3, gamma=1.0, T=1500.0, scheme=SCHEMES[scheme][0], schedule=P.SCHED_ROBUST, seed=8)
    gq, gv = T(q), T(v)
    eng.baoab_propagate_batch(P.COARSE, gq, gv, T(L, torch.int32), T(ids, torch.int64), lp)
    eng.sync_status()
    oq, ov = q.copy(), v.copy()
    olp = O.langevin(dt=1e-3, gamma=1.0, T=1500.0, scheme=SCHEMES[scheme][1], schedule=O.SCHED_ROBUST, seed=8)
    O.propagate(_snap6(), oq, ov, box, L, ids, olp)
    dq, dv = np.abs(N(gq) - oq).max(), np.abs(N(gv) - ov).max()
    assert np.array_equal(N(gq)[0], q[0])                      # L = 0 is the identity
    if precision == P.FP64:
        assert dq < 1e-9 and dv < 1e-7
    else:
        bq, bv = fp32_trajectory_bounds(q[:1], box, W.fitted_beta(8), 40)   # the fine forces bound the coarse ones
        assert dq < bq and dv < bv


def test_snap6_coarse_energy_conservation_gamma0():
    """gamma = 0: the coarse SNAP-6 dynamics is velocity Verlet; the total energy of the FP64
    trajectory (kinetic + SNAP-6 energy from the oracle) drifts by far less than its
    fluctuations' scale, which checks that the coarse forces are the gradient of the energy."""
    pos, box = W.bcc_sia(4)
    n = pos.shape[1]
    q = W.displaced(pos, 0.05, W.rng(72, 1), count=1)
    v = W.velocities(n, 600.0, W.rng(72, 2), count=1)
    eng = _engine(n, box)
    lp = P.langevin(dt=5e-4, gamma=0.0, T=0.0, schedule=P.SCHED_NONE, seed=1)
    gq, gv = T(q), T(v)
    m = W.M_W / W.FTOA
    energies = []
    for k in range(8):
        E, _, _ = O.snap_energy_forces(N(gq), box, W.fitted_beta(2), params=O.snap_params(twojmax=2))
        energies.append(E[0] + 0.5 * m * float(np.sum(N(gv) ** 2)))
        eng.baoab_propagate_batch(P.COARSE, gq, gv, T([50], torch.int32), T([k], torch.int64), lp)
        eng.sync_status()
    energies = np.array(energies)
    assert np.ptp(energies) < 2e-3 * abs(np.mean(energies)) / n, energies   # < 2 meV per atom


@pytest.mark.parametrize("metric,dc,de", [(P.METRIC_REL, 1e-13, 1.0), (P.METRIC_MAXDISP, 1e-10, 2e-3)])
def test_strategy1_adaptive_parareal_matches_algorithm_2(metric, dc, de):
    pos, box = W.bcc_sia(3)
    n = pos.shape[1]
    q0 = W.displaced(pos, 0.05, W.rng(73, 1))
    v0 = W.velocities(n, 1500.0, W.rng(73, 2))
    eng = _engine(n, box)
    Nint, L, dt, seed = 6, 2, 2e-3, 41
    lp = P.langevin(dt=dt, gamma=1.0, T=1500.0, seed=seed, schedule=P.SCHED_ROBUST)
    cur, st = P.adaptive_parareal(eng, T(q0), T(v0), Nint, L, dc, de, lp, metric=metric)
    eng.sync_status()
    olp = O.langevin(dt=dt, gamma=1.0, T=1500.0, seed=seed, schedule=O.SCHED_ROBUST)

    def make(pot):
        def prop(states, ns):
            q = np.ascontiguousarray(np.array([s[0] for s in states]))
            v = np.ascontiguousarray(np.array([s[1] for s in states]))
            O.propagate(pot, q, v, box, [L] * len(ns), ns, olp)
            return [(q[i], v[i]) for i in range(len(ns))]
        return prop
    F = make(O.potential(O.POT_SNAP, beta=W.fitted_beta(8)))
    C = make(_snap6())
    ocur, olog = PR.adaptive(q0, v0, Nint, dc, de, F, C, metric="rel" if metric == P.METRIC_REL else "maxdisp")
    want = [(w["n_init"], e, k, i) for i, w in enumerate(olog.windows) for e, k in w["subs"]]
    assert st.log() == want
    g = N(cur)
    for k in range(Nint + 1):
        assert np.abs(g[k, :3] - ocur[k][0]).max() < 1e-8
        assert np.abs(g[k, 3:] - ocur[k][1]).max() < 1e-6
