"""snap_energy_forces_noalloc through the C ABI: the allocation-free variant of
snap_energy_forces for callers that may not allocate device memory while they run (an
application that owns device memory through its own allocator, a loop where cudaMalloc would
stall the device, a fixed memory budget).  Both entry points run the same kernels on the same
inputs, so the new one must return the regular one's results bit for bit, call after call,
although every call reuses the same static scratch array -- and it must leave the device's
free memory unchanged.

This file is collected last on purpose; it must pass on its own in a fresh process as well."""
import numpy as np
import pytest

import paper_2212_10508_gb300 as P
import workloads as W
from gpu_util import N, T, torch

pytestmark = pytest.mark.gpu


def _outputs(pos, snap):
    nb = pos.shape[0]
    E = torch.full((nb,), float("nan"), dtype=torch.float64, device=pos.device)
    F = torch.full_like(pos, float("nan"))
    S = torch.full((nb, snap.num_coeffs), float("nan"), dtype=torch.float64, device=pos.device)
    return E, F, S


def _noalloc(lib, snap, pos, box, beta, out, energy=True):
    E, F, S = out
    nb, _, n = pos.shape
    rc = lib.snap_energy_forces_noalloc(snap.h, nb, n, P._box(box), P._ptr(pos), P._ptr(beta),
                                        P._ptr(E) if energy else None, P._ptr(F), P._ptr(S) if energy else None,
                                        P._stream())
    assert rc == P.PMD_OK, lib.pmd_last_error()
    return E, F, S


@pytest.mark.parametrize("precision", [P.FP64, P.FP32_BULK])
def test_noalloc_matches_snap_energy_forces_twice(precision):
    lib = P.lib()
    snap = P.Snap(P.snap_params(precision=precision))
    beta = T(W.fitted_beta())
    cases = []
    for master in (31, 32):                        # two different inputs, one call after the other
        pos, box, _ = W.small_system(master=master, nconf=6)
        cases.append((T(pos), box))
    outs = [_outputs(p, snap) for p, _ in cases]
    outs.append(_outputs(cases[0][0], snap))
    # warm-up calls (with and without energies): load the kernels' code and size the launch's
    # local memory before free memory is recorded
    _noalloc(lib, snap, cases[1][0], cases[1][1], beta, _outputs(cases[1][0], snap))
    _noalloc(lib, snap, cases[1][0], cases[1][1], beta, _outputs(cases[1][0], snap), energy=False)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    res = [_noalloc(lib, snap, p, b, beta, o) for (p, b), o in zip(cases, outs)]
    # forces only, again on the first input, after the energy path used more of the array
    _, F_only, _ = _noalloc(lib, snap, cases[0][0], cases[0][1], beta, outs[2], energy=False)
    snap.sync_status()
    assert torch.cuda.mem_get_info()[0] == free_before   # no device memory was allocated
    for (p, b), (E, F, S) in zip(cases, res):
        E0, F0, S0 = P.snap_energy_forces(snap, p, b, beta, sumB=True)
        snap.sync_status()
        assert np.array_equal(N(E), N(E0))
        assert np.array_equal(N(F), N(F0))
        assert np.array_equal(N(S), N(S0))
    _, F0, _ = P.snap_energy_forces(snap, cases[0][0], cases[0][1], beta, energy=False)
    assert np.array_equal(N(F_only), N(F0))


def test_noalloc_rejects_what_snap_energy_forces_rejects():
    lib = P.lib()
    snap = P.Snap(P.snap_params(precision=P.FP64))
    pos, box = W.bcc_sia(10)                       # 2001 atoms
    big = T(np.repeat(pos[None], 4, axis=0))       # 8004 atoms with energies: > 16 MiB of scratch
    beta = T(W.fitted_beta())
    E = torch.empty(4, dtype=torch.float64, device=big.device)
    F = torch.empty_like(big)
    rc = lib.snap_energy_forces_noalloc(snap.h, 4, pos.shape[1], P._box(box), P._ptr(big), P._ptr(beta),
                                        P._ptr(E), P._ptr(F), None, P._stream())
    assert rc == P.PMD_EUNSUPPORTED
    assert b"bytes of scratch" in lib.pmd_last_error()
    for bad in ([float("inf"), box[1], box[2]], [box[0], 2.0, box[2]]):   # same box checks as the regular call
        for fn in (lib.snap_energy_forces_noalloc, lib.snap_energy_forces):
            rc = fn(snap.h, 1, pos.shape[1], P._box(bad), P._ptr(big), P._ptr(beta), None, P._ptr(F), None,
                    P._stream())
            assert rc == P.PMD_EINVAL
