"""Pins for the oracle's Finnis-Sinclair EAM (coarse potential V_C, Sec. 3.1)."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _fs_shell_energy(a, p=W.FS_W):
    """Perfect BCC energy per atom from the neighbour shells: 8 at a*sqrt(3)/2, 6 at a, 12 at
    a*sqrt(2) (> d and > c for tungsten), i.e. the closed form of the FS energy."""
    shells = [(8, a * np.sqrt(3) / 2), (6, a), (12, a * np.sqrt(2)), (24, a * np.sqrt(11) / 2)]
    rho = sum(n * (r - p["d"]) ** 2 for n, r in shells if r < p["d"])
    phi = sum(n * (r - p["c"]) ** 2 * (p["c0"] + p["c1"] * r + p["c2"] * r * r) for n, r in shells if r < p["c"])
    return -p["A"] * np.sqrt(rho) + 0.5 * phi


def test_perfect_bcc_energy_and_equilibrium():
    pos, box = W.bcc(4)
    E, F = O.fs_energy_forces(pos, box)
    e = E[0] / pos.shape[1]
    assert e == pytest.approx(_fs_shell_energy(W.A_W), rel=1e-13)
    # the Finnis-Sinclair tungsten set reproduces E_coh = 8.90 eV at a = 3.1652 Angstrom
    assert e == pytest.approx(-8.90, abs=1e-5)
    assert np.abs(F).max() < 1e-12
    h = 1e-5
    ep = O.fs_energy_forces(*W.bcc(4, W.A_W + h))[0][0] / pos.shape[1]
    em = O.fs_energy_forces(*W.bcc(4, W.A_W - h))[0][0] / pos.shape[1]
    assert abs((ep - em) / (2 * h)) < 1e-3          # a = 3.1652 is the equilibrium spacing


def test_fs_forces_are_minus_gradient():
    P, box, _ = W.small_system(nconf=1)
    E, F = O.fs_energy_forces(P, box)
    assert np.abs(F[0].sum(axis=1)).max() < 1e-11
    h = 1e-4    # energy ~1e3 eV: a smaller step is dominated by roundoff
    for al, i in [(0, 0), (1, 77), (2, 128), (0, 127)]:
        qp, qm = P.copy(), P.copy()
        qp[0, al, i] += h
        qm[0, al, i] -= h
        fd = -(O.fs_energy_forces(qp, box)[0][0] - O.fs_energy_forces(qm, box)[0][0]) / (2 * h)
        assert F[0, al, i] == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_isolated_atom_has_zero_density_branch():
    pos = np.ascontiguousarray(np.array([[1.0, 20.0], [1.0, 20.0], [1.0, 20.0]]))
    E, F = O.fs_energy_forces(pos, np.full(3, 40.0))
    assert E[0] == 0.0 and np.all(F == 0.0)
