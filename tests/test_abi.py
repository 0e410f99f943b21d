"""The C-ABI boundary without a GPU: the library builds and loads, exports every function that
include/pmd.h declares, rejects bad arguments before touching the device, and its host-only
Algorithm 2 state machine (adaptive_restart) replays the oracle's transcription exactly."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import paper_2212_10508_gb300 as P
from paper_2212_10508_gb300 import build as B
from oracle import parareal as PR


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.lib()


def _declared():
    src = open(P.HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                                 src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", P.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)                      # resolvable through ctypes
    assert sorted(P.EXPORTS) == names        # the binding wraps exactly the declared calls


def test_bad_arguments_are_rejected_on_the_host(lib):
    h = ctypes.c_void_p()
    bad = P.snap_params(twojmax=3)
    assert lib.pmd_snap_create(ctypes.byref(bad), ctypes.byref(h)) == P.PMD_EUNSUPPORTED
    big32 = P.snap_params(twojmax=14, precision=P.FP32_BULK)      # 2J > 8: FP64 only
    assert lib.pmd_snap_create(ctypes.byref(big32), ctypes.byref(h)) == P.PMD_EUNSUPPORTED
    big = P.snap_params(twojmax=16)
    assert lib.pmd_snap_create(ctypes.byref(big), ctypes.byref(h)) == P.PMD_EUNSUPPORTED
    ep14 = P.EngineParams(P.snap_params(twojmax=14), P.fs_params(), (ctypes.c_double * 3)(20.0, 20.0, 20.0), 129,
                          P.COARSE_FS, P.snap_params(twojmax=2))
    assert lib.pmd_engine_create(ctypes.byref(ep14), ctypes.byref(h)) == P.PMD_EUNSUPPORTED
    bad = P.snap_params()
    bad.rmin0 = 0.5
    assert lib.pmd_snap_create(ctypes.byref(bad), ctypes.byref(h)) == P.PMD_EINVAL
    assert b"rmin0" in lib.pmd_last_error()
    fs = P.fs_params()
    box = (ctypes.c_double * 3)(20.0, 20.0, 20.0)
    assert lib.eam_energy_forces(ctypes.byref(fs), 1, 5000, box, None, None, None, None) == P.PMD_EUNSUPPORTED
    small = (ctypes.c_double * 3)(5.0, 20.0, 20.0)
    assert lib.eam_energy_forces(ctypes.byref(fs), 1, 10, small, None, None, None, None) == P.PMD_EINVAL
    assert lib.pmd_adaptive_create(10, 0.5, 0.1, ctypes.byref(h)) == P.PMD_EINVAL
    assert lib.adaptive_restart(None, 0.0, 0, None) == P.PMD_EINVAL
    t = P.FineTuning(16, 8, 8, -1, 16)
    assert lib.pmd_engine_set_tuning(None, ctypes.byref(t)) == P.PMD_EINVAL
    assert lib.pmd_engine_get_tuning(None, ctypes.byref(t)) == P.PMD_EINVAL
    assert lib.pmd_engine_autotune(None, 1, 1, None, None, 3, None, None, None, 1, None, None, None) == P.PMD_EINVAL
    assert lib.pmd_engine_selftest_waits(None, 100, None) == P.PMD_EINVAL
    # a SNAP coarse potential must have 2J = 2 (SNAP-6, Strategy I): rejected before any device work
    ep = P.EngineParams(P.snap_params(), P.fs_params(), (ctypes.c_double * 3)(20.0, 20.0, 20.0), 129,
                        P.COARSE_SNAP, P.snap_params(twojmax=4))
    assert lib.pmd_engine_create(ctypes.byref(ep), ctypes.byref(h)) == P.PMD_EUNSUPPORTED
    ep.coarse_kind = 7
    assert lib.pmd_engine_create(ctypes.byref(ep), ctypes.byref(h)) == P.PMD_EINVAL
    assert lib.pmd_engine_set_coarse_beta(None, None, None) == P.PMD_EINVAL
    box3 = (ctypes.c_double * 3)(10.0, 10.0, 10.0)
    assert lib.sia_locate(1, 0, 4, box3, None, 3, None, None, None, None, None) == P.PMD_EINVAL
    assert lib.sia_locate(1, 4, 0, box3, None, 12, None, None, None, None, None) == P.PMD_EINVAL
    assert lib.sia_locate(1, 4, 4097, box3, None, 12, None, None, None, None, None) == P.PMD_EINVAL
    assert lib.sia_locate(1, 4, 4, box3, None, 12, None, None, None, None, None) == P.PMD_EINVAL
    assert lib.sia_locate(0, 4, 4, box3, None, 12, None, None, None, None, None) == P.PMD_OK
    bad = (ctypes.c_double * 3)(10.0, 0.0, 10.0)
    assert lib.sia_locate(0, 4, 4, bad, None, 12, None, None, None, None, None) == P.PMD_EINVAL
    k = ctypes.c_int()
    assert lib.sia_residence(None, 3, 3, None, None, ctypes.byref(k)) == P.PMD_EINVAL
    w = (ctypes.c_int32 * 5)(1, 1, 2, 2, 3)
    L = (ctypes.c_int32 * 1)()
    assert lib.sia_residence(w, 5, 1, L, None, ctypes.byref(k)) == P.PMD_ENOMEM
    L2 = (ctypes.c_int32 * 5)()
    assert lib.sia_residence(w, 5, 5, L2, None, ctypes.byref(k)) == P.PMD_OK and k.value == 2
    assert list(L2)[:2] == [2, 2]


def _replay(N, dc, de, trace):
    st = P.Adaptive(N, dc, de)
    act = st.adaptive_restart()
    for (n_init, n_fin, delta, n_stop, _) in trace:
        assert act.kind == P.ACT_ITERATE and (act.n_in, act.n_fin) == (n_init, n_fin)
        act = st.adaptive_restart(delta, n_stop)
    assert act.kind == P.ACT_DONE
    return st


@pytest.mark.parametrize("f,c,N,dc,de", [(1.05, 0.5, 40, 1e-9, 0.3), (1.0, 0.8, 25, 1e-6, 1e9),
                                         (1.2, 0.3, 30, 1e-10, 0.05), (1.0, 1.0, 10, 1e-8, 0.2)])
def test_adaptive_restart_replays_algorithm_2(lib, f, c, N, dc, de):
    prop = lambda k: (lambda states, ns: [(k * s[0], k * s[1]) for s in states])
    trace = []
    _, log = PR.adaptive(np.array([1.0]), np.array([0.0]), N, dc, de, prop(f), prop(c), trace=trace)
    st = _replay(N, dc, de, trace)
    want = [(w["n_init"], e, k, i) for i, w in enumerate(log.windows) for e, k in w["subs"]]
    assert st.log() == want
    for Cf, Cc in [(1.0, 0.01), (1787.0, 0.6923)]:
        cost, g, gi = st.cost(Cf, Cc)
        ocost, og, ogi = PR.cost_and_gains(log, N, Cf, Cc)
        assert cost == pytest.approx(ocost, rel=1e-15) and g == pytest.approx(og) and gi == pytest.approx(ogi)


def test_adaptive_restart_degenerate_explosion_at_slab_start(lib):
    st = P.Adaptive(5, 1e-6, 0.1)
    a = st.adaptive_restart()
    assert (a.n_in, a.n_fin, a.open_slab) == (0, 5, 1)
    a = st.adaptive_restart(0.9, 0)          # explosion at n = N_init -> [0, 1], not empty
    assert (a.kind, a.n_in, a.n_fin, a.open_slab) == (P.ACT_ITERATE, 0, 1, 0)
    a = st.adaptive_restart(0.0, 1)          # converged -> next slab [1, 5]
    assert (a.n_in, a.n_fin, a.open_slab) == (1, 5, 1)
    a = st.adaptive_restart(float("nan"), 3)  # non-finite counts as an explosion
    assert (a.n_in, a.n_fin) == (1, 3)
    with pytest.raises(P.PmdError):
        st.adaptive_restart(1.0, 9)          # n_stop outside the slab


def test_adaptive_restart_follows_the_hand_worked_trace(lib):
    """The library's Algorithm 2 state machine fed the errors of the linear problem F x = x,
    C x = 0.7 x (N = 8, delta_expl = 0.35, delta_conv = 0.05; errors from the closed form,
    worked out by hand in tests/test_oracle_parareal.py) produces the hand-derived slabs and
    the eq. (7) cost 8 C_f + 56 C_c."""
    st = P.Adaptive(8, 0.05, 0.35)
    act = st.adaptive_restart()
    steps = [((0, 8), 0.4583, 2), ((0, 2), 0.0309, 2), ((2, 8), 0.4583, 4), ((2, 4), 0.0309, 4),
             ((4, 8), 0.4583, 6), ((4, 6), 0.0309, 6), ((6, 8), 0.3288, 8), ((6, 8), 0.0309, 8)]
    for (rng, delta, n_stop) in steps:
        assert act.kind == P.ACT_ITERATE and (act.n_in, act.n_fin) == rng
        act = st.adaptive_restart(delta, n_stop)
    assert act.kind == P.ACT_DONE
    assert st.log() == [(0, 8, 1, 0), (0, 2, 1, 0), (2, 8, 1, 1), (2, 4, 1, 1), (4, 8, 1, 2), (4, 6, 1, 2),
                        (6, 8, 2, 3)]
    cost, g, gi = st.cost(1.0, 0.01)
    assert cost == pytest.approx(8.56, rel=1e-14) and gi == 1.0
