"""Ridge fit of linear SNAP coefficients to reference energies and forces (config 4 of the
workloads: Finnis-Sinclair tungsten as the reference), on the GPU through the library.

The energy model is linear in beta: E = sum_t beta_t dE/dbeta_t with dE/dbeta from the bispectrum
stage, and the forces are F = sum_t beta_t F(e_t) where F(e_t) is the force field of the unit
coefficient vector e_t (one adjoint + force pass per component).  Rows: energy per atom (weight
w_E) and every force component (weight 1); the normal equations (X^T X + lambda I) beta = X^T y
are solved in FP64.
"""
import torch

from . import (COARSE, FP64, SCHED_ROBUST, SCHEME_PAPER, Engine, Snap, eam_energy_forces, fs_params, langevin,
               snap_energy_forces, snap_params)


def fs_training_set(starts, box, temps, snapshots=3, steps=100, dt=2e-3, gamma=5.0, seed0=1000, fs=None):
    """Langevin Finnis-Sinclair dynamics (paper scheme, robust schedule) of each start (q, v)
    [m,3,n] at its temperature, sampled every `steps` steps: [len(temps)*snapshots*m, 3, n]."""
    q0 = starts[0][0]
    n = q0.shape[2]
    dev = q0.device
    eng = Engine(n, box, snap_params(), fs or fs_params(precision=FP64))
    confs = []
    for it, ((qs, vs), T) in enumerate(zip(starts, temps)):
        q, v = qs.clone().contiguous(), vs.clone().contiguous()
        m = q.shape[0]
        lp = langevin(dt=dt, gamma=gamma, T=float(T), scheme=SCHEME_PAPER, schedule=SCHED_ROBUST, seed=seed0 + it)
        ns = torch.full((m,), steps, dtype=torch.int32, device=dev)
        for k in range(snapshots):
            ids = torch.arange(m * k, m * k + m, dtype=torch.int64, device=dev)
            eng.baoab_propagate_batch(COARSE, q, v, ns, ids, lp)
            confs.append(q.clone())
    eng.sync_status()
    return torch.cat(confs)


def design(confs, box, twojmax=8, precision=FP64):
    """Energy rows [nc, 1+nB] (per atom) and force rows [nc*3*n, 1+nB] of the linear SNAP model."""
    snap = Snap(snap_params(twojmax=twojmax, precision=precision))
    nc, _, n = confs.shape
    nb1 = snap.num_coeffs
    zero = torch.zeros(nb1, dtype=torch.float64, device=confs.device)
    _, _, S = snap_energy_forces(snap, confs, box, zero, energy=False, forces=False, sumB=True)
    XE = S / n
    XF = torch.zeros(nc * 3 * n, nb1, dtype=torch.float64, device=confs.device)
    for t in range(1, nb1):
        e = torch.zeros(nb1, dtype=torch.float64, device=confs.device)
        e[t] = 1.0
        _, F, _ = snap_energy_forces(snap, confs, box, e, energy=False, forces=True)
        XF[:, t] = F.reshape(-1)
    snap.sync_status()
    return XE, XF


def fit_beta_ridge(confs, box, E_ref, F_ref, lam=1e-6, w_energy=1.0, twojmax=8, precision=FP64):
    """beta [1+nB] minimising |w_E (X_E beta - E_ref/n)|^2 + |X_F beta - F_ref|^2 + lam |beta|^2."""
    XE, XF = design(confs, box, twojmax, precision)
    n = confs.shape[2]
    X = torch.cat([w_energy * XE, XF])
    y = torch.cat([w_energy * E_ref / n, F_ref.reshape(-1)])
    A = X.T @ X + lam * torch.eye(X.shape[1], dtype=X.dtype, device=X.device)
    return torch.linalg.solve(A, X.T @ y)


def fs_reference(confs, box, fs=None):
    E, F = eam_energy_forces(confs, box, fs or fs_params(precision=FP64))
    return E, F
