"""GPU parity of snap_energy_forces and eam_energy_forces against the FP64 oracle (Sec. 3.1).

Bars: FP64 kernels 1e-10 relative (max-norm over the batch) on energies, forces and dE/dbeta;
FP32-bulk kernels 1e-5.  Inputs: the 129-atom W + SIA cell with 0.05 Angstrom displacements
(16 configurations), other SNAP sizes, the 2001-atom cell, ragged and degenerate systems."""
import numpy as np
import pytest

import oracle as O
import paper_2212_10508_gb300 as P
import workloads as W
from gpu_util import N, T, dev, rel_max, torch

pytestmark = pytest.mark.gpu


def _snap(twojmax=8, precision=P.FP64):
    return P.Snap(P.snap_params(twojmax=twojmax, precision=precision))


def _compare_snap(pos, box, beta, twojmax, precision, tol):
    s = _snap(twojmax, precision)
    E, F, S = P.snap_energy_forces(s, T(pos), box, T(beta), sumB=True)
    s.sync_status()
    oE, oF, oS = O.snap_energy_forces(pos, box, beta, params=O.snap_params(twojmax=twojmax))
    assert rel_max(N(E), oE) <= tol
    assert rel_max(N(F), oF) <= tol
    assert rel_max(N(S), oS) <= tol
    return N(F), oF


def test_snap_fp64_matches_oracle_129_atoms():
    P_, box, beta = W.small_system(nconf=16)
    _compare_snap(P_, box, beta, 8, P.FP64, 1e-10)


def test_snap_fp32_bulk_matches_oracle_129_atoms():
    P_, box, beta = W.small_system(nconf=16)
    _compare_snap(P_, box, beta, 8, P.FP32_BULK, 1e-5)


@pytest.mark.parametrize("twojmax", [2, 4, 6])
@pytest.mark.parametrize("precision,tol", [(P.FP64, 1e-10), (P.FP32_BULK, 1e-5)])
def test_snap_other_band_limits(twojmax, precision, tol):
    P_, box, _ = W.small_system(nconf=3)
    beta = W.snap_beta(W.n_bispectrum(twojmax), W.rng(5, twojmax))
    _compare_snap(P_, box, beta, twojmax, precision, tol)


@pytest.mark.parametrize("twojmax", [10, 12, 14])
def test_snap_large_band_limits_fp64(twojmax):
    """2J = 10, 12 and 14 (14: the paper's SNAP-205 size, 204 bispectrum components), FP64 warp
    per atom with the Clebsch-Gordan values in global memory: energies, forces and dE/dbeta of
    two 129-atom configurations against the oracle at 1e-10."""
    P_, box, _ = W.small_system(nconf=2)
    beta = W.snap_beta(W.n_bispectrum(twojmax), W.rng(6, twojmax))
    _compare_snap(P_, box, beta, twojmax, P.FP64, 1e-10)


def test_snap_2001_atoms():
    pos, box = W.bcc_sia(10)
    pos = W.displaced(pos, 0.05, W.rng(7, 1), count=1)
    beta = W.snap_beta(55, W.rng(7, 2))
    _compare_snap(pos, box, beta, 8, P.FP64, 1e-10)
    _compare_snap(pos, box, beta, 8, P.FP32_BULK, 1e-5)


def test_snap_ragged_cluster_and_isolated_atoms():
    rng = np.random.default_rng(3)
    L = 40.0
    pts = [np.full(3, L / 2)]
    while len(pts) < 37:                       # 37 atoms: not a multiple of a warp
        p = L / 2 + rng.uniform(-5, 5, 3)
        if all(np.linalg.norm(p - q) > 2.0 for q in pts):
            pts.append(p)
    pts.append(np.array([2.0, 2.0, 2.0]))      # an atom with no neighbour at all
    pos = np.ascontiguousarray(np.array(pts).T[None])
    box = np.full(3, L)
    beta = W.snap_beta(55, W.rng(9, 1))
    F, oF = _compare_snap(pos, box, beta, 8, P.FP64, 1e-10)
    assert np.all(F[0, :, -1] == 0.0)


def test_snap_empty_batch_and_overflow():
    s = _snap()
    box = np.full(3, 30.0)
    beta = T(W.snap_beta(55, W.rng(1, 1)))
    E, F, _ = P.snap_energy_forces(s, T(np.zeros((0, 3, 5))), box, beta)
    s.sync_status()
    # 80 atoms inside 2 Angstrom: more than PMD_MAX_NEIGHBORS neighbours -> ENEIGH, not silent
    rng = np.random.default_rng(0)
    pos = 15.0 + rng.uniform(-1.0, 1.0, size=(1, 3, 80))
    P.snap_energy_forces(s, T(pos), box, beta)
    with pytest.raises(P.PmdError) as e:
        s.sync_status()
    assert e.value.code == P.PMD_ENEIGH
    s.sync_status()                             # the status word is cleared


def _compare_eam(pos, box, precision, tol):
    E, F = P.eam_energy_forces(T(pos), box, P.fs_params(precision=precision))
    torch.cuda.synchronize()
    oE, oF = O.fs_energy_forces(pos, box)
    assert rel_max(N(E), oE) <= tol
    assert rel_max(N(F), oF) <= tol


@pytest.mark.parametrize("precision,tol", [(P.FP64, 1e-10), (P.FP32_BULK, 1e-5)])
def test_eam_matches_oracle(precision, tol):
    P_, box, _ = W.small_system(nconf=16)
    _compare_eam(P_, box, precision, tol)
    pos, box = W.bcc_sia(10)
    _compare_eam(W.displaced(pos, 0.05, W.rng(4, 1), count=2), box, precision, tol)
    pos, box = W.bcc_sia(5)
    _compare_eam(W.displaced(pos, 0.1, W.rng(4, 2), count=3), box, precision, tol)


def test_eam_perfect_lattice_energy():
    pos, box = W.bcc(4)
    E, F = P.eam_energy_forces(T(pos[None]), box)
    assert N(E)[0] / pos.shape[1] == pytest.approx(-8.900002, abs=1e-6)
    assert np.abs(N(F)).max() < 1e-10
