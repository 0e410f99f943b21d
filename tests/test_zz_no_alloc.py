"""snap_energy_forces_noalloc through the C ABI: the allocation-free variant of
snap_energy_forces for callers that may not allocate device memory while they run (an
application that owns device memory through its own allocator, a loop where cudaMalloc would
stall the device, a fixed memory budget).  It must return what the regular entry point returns,
call after call, although every call reuses the same static scratch array.

This file is collected last on purpose; it must pass on its own in a fresh process as well."""
import ctypes

import numpy as np
import pytest

import paper_2212_10508_gb300 as P
import workloads as W
from gpu_util import N, T, rel_max, torch

pytestmark = pytest.mark.gpu


def _noalloc(lib, snap, pos, box, beta, energy=True):
    nb, _, n = pos.shape
    E = torch.full((nb,), float("nan"), dtype=torch.float64, device=pos.device)
    F = torch.full_like(pos, float("nan"))
    S = torch.full((nb, snap.num_coeffs), float("nan"), dtype=torch.float64, device=pos.device)
    rc = lib.snap_energy_forces_noalloc(snap.h, nb, n, P._box(box), P._ptr(pos), P._ptr(beta),
                                        P._ptr(E) if energy else None, P._ptr(F), P._ptr(S) if energy else None,
                                        P._stream())
    assert rc == P.PMD_OK, lib.pmd_last_error()
    return E, F, S


@pytest.mark.parametrize("precision,tol", [(P.FP64, 1e-10), (P.FP32_BULK, 1e-5)])
def test_noalloc_matches_snap_energy_forces_twice(precision, tol):
    lib = P.lib()
    snap = P.Snap(P.snap_params(precision=precision))
    beta = T(W.fitted_beta())
    cases = []
    for master in (31, 32):                        # two different inputs, one call after the other
        pos, box, _ = W.small_system(master=master, nconf=6)
        cases.append((T(pos), box))
    outs = [_noalloc(lib, snap, p, b, beta) for p, b in cases]
    snap.sync_status()
    for (p, b), (E, F, S) in zip(cases, outs):
        E0, F0, S0 = P.snap_energy_forces(snap, p, b, beta, sumB=True)
        snap.sync_status()
        assert rel_max(N(E), N(E0)) <= tol
        assert rel_max(N(F), N(F0)) <= tol
        assert rel_max(N(S), N(S0)) <= tol
    # forces only, again on the first input, after the energy path used more of the array
    _, F, _ = _noalloc(lib, snap, cases[0][0], cases[0][1], beta, energy=False)
    snap.sync_status()
    _, F0, _ = P.snap_energy_forces(snap, cases[0][0], cases[0][1], beta, energy=False)
    assert rel_max(N(F), N(F0)) <= tol


def test_noalloc_rejects_requests_larger_than_its_array():
    lib = P.lib()
    snap = P.Snap(P.snap_params(precision=P.FP64))
    pos, box = W.bcc_sia(10)                       # 2001 atoms
    big = T(np.repeat(pos[None], 4, axis=0))       # 8004 atoms with energies: > 16 MiB of scratch
    E = torch.empty(4, dtype=torch.float64, device=big.device)
    F = torch.empty_like(big)
    rc = lib.snap_energy_forces_noalloc(snap.h, 4, pos.shape[1], P._box(box), P._ptr(big), P._ptr(T(W.fitted_beta())),
                                        P._ptr(E), P._ptr(F), None, P._stream())
    assert rc == P.PMD_EUNSUPPORTED
    assert b"bytes of scratch" in lib.pmd_last_error()
