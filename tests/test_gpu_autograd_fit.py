"""The differentiable SNAP energy (forward = bispectrum stage, backward = adjoint force pass and
dE/dbeta) and the GPU ridge fit of beta to Finnis-Sinclair tungsten (config 4's recipe),
against the oracle and central finite differences."""
import numpy as np
import pytest

import oracle as O
import paper_2212_10508_gb300 as P
from paper_2212_10508_gb300.autograd import snap_energy
from paper_2212_10508_gb300 import fit as FIT
import workloads as W
from gpu_util import N, T, dev, rel_max, torch

pytestmark = pytest.mark.gpu


def test_autograd_gradients_match_oracle_and_fd():
    pos, box, beta = W.small_system(master=41, nconf=3)
    snap = P.Snap(P.snap_params())
    tp = T(pos).requires_grad_(True)
    tb = T(beta).requires_grad_(True)
    E = snap_energy(tp, tb, snap, box)
    w = torch.tensor([1.0, -0.5, 2.0], dtype=torch.float64, device=tp.device)
    (E * w).sum().backward()
    oE, oF, oS = O.snap_energy_forces(pos, box, beta)
    assert rel_max(N(E), oE) <= 1e-10
    assert rel_max(N(tp.grad), -N(w)[:, None, None] * oF) <= 1e-10          # d(sum w E)/dr = -w F
    assert rel_max(N(tb.grad), (N(w)[:, None] * oS).sum(0)) <= 1e-10      # d(sum w E)/dbeta = sum w sumB
    h = 1e-4
    with torch.no_grad():
        for (b, al, i) in [(0, 0, 3), (1, 2, 100), (2, 1, 128)]:
            pp, pm = tp.detach().clone(), tp.detach().clone()
            pp[b, al, i] += h
            pm[b, al, i] -= h
            fd = (snap_energy(pp, tb.detach(), snap, box)[b] - snap_energy(pm, tb.detach(), snap, box)[b]) / (2 * h)
            assert float(fd) == pytest.approx(float(tp.grad[b, al, i] / w[b]), rel=1e-6, abs=1e-7)


def test_gpu_fit_reproduces_oracle_fit():
    """Same training set and normal equations as tests/golden/make_fitted_beta.py, built with the
    library (coarse propagator for the dynamics, SNAP kernels for the design): the coefficients
    agree with the stored oracle fit."""
    pos0, box = W.bcc_sia(4)
    n = pos0.shape[1]
    temps = [300, 800, 1500, 2200, 3000]
    starts = [(T(W.displaced(pos0, 0.02, W.rng(4, 10 + it), count=4)), T(W.velocities(n, Tk, W.rng(4, 20 + it), count=4)))
              for it, Tk in enumerate(temps)]
    confs = FIT.fs_training_set(starts, box, temps)
    E, F = FIT.fs_reference(confs, box)
    beta = FIT.fit_beta_ridge(confs, box, E, F, lam=1e-6)
    gold = W.fitted_beta()
    assert rel_max(N(beta), gold) <= 1e-6


def _cfg4_small():
    """Config 4's recipe at the size of the oracle's 2J = 6 golden: 4 temperatures in 500-3000 K x 4
    cells with a randomly placed <111> dumbbell x 3 snapshots = 48 configurations."""
    confs, box = FIT.config4_set(6, groups=4, members=4, snapshots=3, device=dev())
    E, F = FIT.fs_reference(confs, box)
    return confs, box, E, F


def test_gpu_fit_2j6_reproduces_oracle_fit():
    """The FP64 ridge fit at 2J = 6 on config 4's recipe (random dumbbell placements, 500-3000 K),
    training set generated and design built with the library, against the oracle's fit
    (tests/golden/make_fitted_beta.py, beta_fs_w_2j6.txt)."""
    confs, box, E, F = _cfg4_small()
    beta = FIT.fit_beta_ridge(confs, box, E, F, lam=1e-6, twojmax=6)
    assert rel_max(N(beta), W.fitted_beta(6)) <= 1e-6


@pytest.mark.parametrize("twojmax", [6, 8])
def test_fitted_forces_equal_central_differences_h1e5(twojmax):
    """dE/dr of the fitted FP64 SNAP against central differences with h = 1e-5 Angstrom on 12
    sampled coordinates of config 4's configurations (truncation ~h^2 E''' and roundoff
    ~eps |E| / h are both ~1e-8 eV/Angstrom here)."""
    confs, box, _, _ = _cfg4_small()
    g = np.random.default_rng(twojmax)
    coords = [(int(g.integers(confs.shape[0])), int(g.integers(3)), int(g.integers(confs.shape[2]))) for _ in range(12)]
    err, rows = FIT.fd_check(T(W.fitted_beta(twojmax)), confs, box, coords, h=1e-5, twojmax=twojmax)
    assert err < 1e-6, rows


def test_fp32_bulk_fit_matches_fp64_fit():
    """The same fit built from FP32-bulk design rows: its force and energy errors against
    Finnis-Sinclair stay within 1 % of the FP64 fit's (the FP32-bulk rows differ from the FP64
    rows by ~1e-6 relative)."""
    confs, box, E, F = _cfg4_small()
    out = {}
    for prec in (P.FP64, P.FP32_BULK):
        beta = FIT.fit_beta_ridge(confs, box, E, F, lam=1e-6, twojmax=6, precision=prec)
        out[prec] = FIT.rmse(beta, confs, box, E, F, twojmax=6, precision=prec)
    (e64, f64), (e32, f32) = out[P.FP64], out[P.FP32_BULK]
    assert f32 <= 1.01 * f64 and e32 <= 1.01 * e64 + 1e-5
    assert f64 < 0.5                                   # a usable fit: force RMSE well below typical forces
