"""Ridge fit of linear SNAP coefficients to reference energies and forces (config 4 of the
workloads: Finnis-Sinclair tungsten as the reference), on the GPU through the library.

The energy model is linear in beta: E = sum_t beta_t dE/dbeta_t with dE/dbeta from the bispectrum
stage, and the forces are F = sum_t beta_t F(e_t) where F(e_t) is the force field of the unit
coefficient vector e_t (one adjoint + force pass per component).  Rows: energy per atom (weight
w_E) and every force component (weight 1); the normal equations (X^T X + lambda I) beta = X^T y
are solved in FP64.  The design rows come from the SNAP kernels in the requested precision
(FP64, or FP32-bulk: U/Z/Y in FP32 with FP64 sums), so an FP32 fit is the fit of the FP32-bulk
model.

    python -m paper_2212_10508_gb300.fit [--configs 4096] [--twojmax 8 6] [--precision fp64 fp32]

builds config 4's training set (thermal snapshots at 500-3000 K of cells with a randomly placed
<111> dumbbell, Langevin Finnis-Sinclair dynamics on the GPU), fits each (2J, precision), and
prints one JSON line per fit: energy and force RMSE against Finnis-Sinclair on the training set
and on a held-out set of the same recipe, and central differences of the fitted FP64 energy
(h = 1e-5 Angstrom) against its forces on sampled coordinates.
"""
import argparse
import json
import time

import torch

from . import (COARSE, FP32_BULK, FP64, SCHED_ROBUST, SCHEME_PAPER, Engine, Snap, eam_energy_forces, fs_params,
               langevin, snap_energy_forces, snap_params)


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


def config4_set(master, groups, members, snapshots, device):
    """Config 4's training configurations: workloads.fit_starts (random <111> dumbbell sites and
    axes, temperatures uniform in 500-3000 K) advanced by fs_training_set."""
    import workloads as W
    starts, temps, box = W.fit_starts(master, groups, members)
    tstarts = [(torch.as_tensor(q, device=device), torch.as_tensor(v, device=device)) for q, v in starts]
    return fs_training_set(tstarts, box, temps, snapshots=snapshots), box


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


def rmse(beta, confs, box, E_ref, F_ref, twojmax=8, precision=FP64):
    """(energy RMSE per atom in eV/atom, force RMSE per component in eV/Angstrom) of the SNAP with
    coefficients beta against the reference energies and forces."""
    snap = Snap(snap_params(twojmax=twojmax, precision=precision))
    E, F, _ = snap_energy_forces(snap, confs, box, beta)
    snap.sync_status()
    n = confs.shape[2]
    eE = float(torch.sqrt(torch.mean(((E - E_ref) / n) ** 2)))
    eF = float(torch.sqrt(torch.mean((F - F_ref) ** 2)))
    return eE, eF


def fd_check(beta, confs, box, coords, h=1e-5, twojmax=8):
    """Central differences of the FP64 SNAP energy, (E(q + h e) - E(q - h e)) / 2h, at the given
    (config, axis, atom) coordinates against -F there.  Returns (max |fd + F| / max |F|, rows)."""
    snap = Snap(snap_params(twojmax=twojmax, precision=FP64))
    sel = sorted({c for c, _, _ in coords})
    base = confs[sel].clone()
    _, F, _ = snap_energy_forces(snap, base, box, beta, energy=False)
    plus, minus = [], []
    for c, al, i in coords:
        k = sel.index(c)
        qp, qm = base[k].clone(), base[k].clone()
        qp[al, i] += h
        qm[al, i] -= h
        plus.append(qp)
        minus.append(qm)
    Ep, _, _ = snap_energy_forces(snap, torch.stack(plus), box, beta, forces=False)
    Em, _, _ = snap_energy_forces(snap, torch.stack(minus), box, beta, forces=False)
    snap.sync_status()
    fd = (Ep - Em) / (2 * h)
    f = torch.stack([F[sel.index(c), al, i] for c, al, i in coords])
    err = float((fd + f).abs().max() / f.abs().max())
    return err, [(int(c), int(al), int(i), float(a), float(b)) for (c, al, i), a, b in zip(coords, fd, -f)]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--configs", type=int, default=4096, help="training configurations (multiple of 128)")
    ap.add_argument("--heldout", type=int, default=512, help="held-out configurations of the same recipe")
    ap.add_argument("--twojmax", type=int, nargs="+", default=[8, 6])
    ap.add_argument("--precision", nargs="+", default=["fp64", "fp32"], choices=["fp64", "fp32"])
    ap.add_argument("--lam", type=float, default=1e-6)
    args = ap.parse_args(argv)
    dev = torch.device("cuda", torch.cuda.current_device())
    members, snaps = 16, 8                          # configurations per temperature group: 16 x 8
    t0 = time.perf_counter()
    train, box = config4_set(4, args.configs // (members * snaps), members, snaps, dev)
    test, _ = config4_set(40, max(1, args.heldout // (members * snaps)), members, snaps, dev)
    Etr, Ftr = fs_reference(train, box)
    Ete, Fte = fs_reference(test, box)
    torch.cuda.synchronize()
    t_set = time.perf_counter() - t0
    g = torch.Generator().manual_seed(7)
    coords = [(int(torch.randint(0, train.shape[0], (1,), generator=g)), int(torch.randint(0, 3, (1,), generator=g)),
               int(torch.randint(0, train.shape[2], (1,), generator=g))) for _ in range(12)]
    for tj in args.twojmax:
        for name in args.precision:
            prec = FP64 if name == "fp64" else FP32_BULK
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            beta = fit_beta_ridge(train, box, Etr, Ftr, lam=args.lam, twojmax=tj, precision=prec)
            torch.cuda.synchronize()
            t_fit = time.perf_counter() - t0
            eE, eF = rmse(beta, train, box, Etr, Ftr, tj, prec)
            hE, hF = rmse(beta, test, box, Ete, Fte, tj, prec)
            fd_err, _ = fd_check(beta, train, box, coords, h=1e-5, twojmax=tj)
            print(json.dumps({"twojmax": tj, "precision": name, "configs": int(train.shape[0]),
                              "heldout": int(test.shape[0]), "atoms": int(train.shape[2]), "lambda": args.lam,
                              "rmse_energy_meV_per_atom": 1e3 * eE, "rmse_force_eV_per_A": eF,
                              "heldout_rmse_energy_meV_per_atom": 1e3 * hE, "heldout_rmse_force_eV_per_A": hF,
                              "fd_h1e-5_max_rel_err": fd_err, "fit_s": round(t_fit, 2),
                              "training_set_s": round(t_set, 2), "beta0": float(beta[0])}), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
