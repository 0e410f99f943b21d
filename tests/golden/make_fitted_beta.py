"""Write tests/golden/beta_fs_w_2j8.txt, beta_fs_w_2j6.txt and beta_fs_w_2j2.txt: SNAP coefficients
(2J = 8, 1 + 55 values; 2J = 6, 1 + 30 values; 2J = 2, 1 + 5 values, the SNAP-6 coarse potential
of Strategy I) fitted by ridge regression (lambda = 1e-6) to Finnis-Sinclair
tungsten energies and forces, computed with the FP64 oracle only.

Why: random coefficients beta_t ~ N(0, 0.01^2) give a SNAP without a repulsive core; the
129-atom cell then collapses within ~150 steps at 1500 K.  The fitted coefficients give a stable
tungsten-like SNAP, the setting the paper's SNAP fine potentials are used in (Sec. 3.1).

Training set (seeded, synthetic): the 129-atom W + SIA cell, 0.02 Angstrom displacements, 4
members each at 300, 800, 1500, 2200 and 3000 K, Langevin EAM dynamics (paper scheme, robust
schedule, dt 2 fs, gamma 5/ps) sampled after 100, 200 and 300 steps: 60 configurations.
Rows: energy per atom (weight 1) and every force component (weight 1).

2J = 6 and 2J = 2 (config 4's recipe, small): workloads.fit_starts(master=6, groups=4, members=4) -- four
temperatures drawn in 500-3000 K, each with four cells whose <111> dumbbell sits at a random
site along a random <111> axis, 0.02 Angstrom displacements -- then the same Langevin EAM
dynamics (dt 2 fs, gamma 5/ps, seed 1000 + group, interval ids 4 k + m) sampled after 100, 200
and 300 steps: 48 configurations.

    python tests/golden/make_fitted_beta.py     (about 2-3 minutes on 8 cores)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "beta_fs_w_2j8.txt")
OUT6 = os.path.join(HERE, "beta_fs_w_2j6.txt")
OUT2 = os.path.join(HERE, "beta_fs_w_2j2.txt")


def training_set(master=4):
    pos0, box = W.bcc_sia(4)
    n = pos0.shape[1]
    fs = O.potential(O.POT_FS)
    confs = []
    for it, Tk in enumerate([300, 800, 1500, 2200, 3000]):
        q = W.displaced(pos0, 0.02, W.rng(master, 10 + it), count=4)
        v = W.velocities(n, Tk, W.rng(master, 20 + it), count=4)
        lp = O.langevin(dt=2e-3, gamma=5.0, T=float(Tk), seed=1000 + it, schedule=O.SCHED_ROBUST)
        for k in range(3):
            O.propagate(fs, q, v, box, [100] * 4, [4 * k + m for m in range(4)], lp)
            confs.extend(list(q.copy()))
    return np.ascontiguousarray(np.array(confs)), box


def training_set_cfg4(master=6, groups=4, members=4, snapshots=3):
    starts, temps, box = W.fit_starts(master, groups, members)
    fs = O.potential(O.POT_FS)
    confs = []
    for it, ((q0, v0), Tk) in enumerate(zip(starts, temps)):
        q, v = q0.copy(), v0.copy()
        lp = O.langevin(dt=2e-3, gamma=5.0, T=float(Tk), seed=1000 + it, schedule=O.SCHED_ROBUST)
        for k in range(snapshots):
            O.propagate(fs, q, v, box, [100] * members, [members * k + m for m in range(members)], lp)
            confs.extend(list(q.copy()))
    return np.ascontiguousarray(np.array(confs)), box


def fit(confs, box, lam=1e-6, twojmax=8):
    nt = len(O.snap_triples(twojmax))
    n = confs.shape[2]
    p = O.snap_params(twojmax=twojmax)
    Efs, Ffs = O.fs_energy_forces(confs, box)
    _, _, sB = O.snap_energy_forces(confs, box, np.zeros(1 + nt), params=p)
    AF = np.zeros((len(confs), 3, n, nt))
    for t in range(nt):
        b = np.zeros(1 + nt)
        b[1 + t] = 1.0
        AF[..., t] = O.snap_energy_forces(confs, box, b, params=p)[1]
    XE = np.concatenate([np.ones((len(confs), 1)), sB[:, 1:] / n], axis=1)
    XF = np.concatenate([np.zeros((AF.size // nt, 1)), AF.reshape(-1, nt)], axis=1)
    X = np.concatenate([XE, XF])
    y = np.concatenate([Efs / n, Ffs.reshape(-1)])
    return np.linalg.solve(X.T @ X + lam * np.eye(1 + nt), X.T @ y)


def write(path, beta, twojmax, nt):
    with open(path, "w") as fh:
        fh.write("# SNAP 2J=%d coefficients beta_0..beta_%d fitted to Finnis-Sinclair W with the FP64 oracle\n"
                 % (twojmax, nt))
        fh.write("# written by tests/golden/make_fitted_beta.py (ridge lambda 1e-6; see its docstring)\n")
        for b in beta:
            fh.write("%.17g\n" % b)
    print(path, beta[0], np.abs(beta[1:]).max())


if __name__ == "__main__":
    which = sys.argv[1:] or ["8", "6", "2"]
    if "8" in which:
        confs, box = training_set()
        write(OUT, fit(confs, box), 8, 55)
    if "6" in which:
        confs, box = training_set_cfg4()
        write(OUT6, fit(confs, box, twojmax=6), 6, 30)
    if "2" in which:   # SNAP-6: the coarse potential of Strategy I, same training set as 2J = 6
        confs, box = training_set_cfg4()
        write(OUT2, fit(confs, box, twojmax=2), 2, 5)
