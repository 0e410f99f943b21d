"""Python binding of ``libpmd.so``: the GB300 (sm_103a) hot path of adaptive parareal Langevin
dynamics with a SNAP fine and a Finnis-Sinclair EAM coarse potential (arXiv 2212.10508).

This module only marshals arguments: every step of the path runs in the library's CUDA
kernels.  Tensors are torch CUDA tensors (float64, contiguous); PyTorch provides device
memory and streams.  The C functions keep their names: :func:`snap_energy_forces`,
:func:`eam_energy_forces`, :meth:`Engine.baoab_propagate_batch`, :meth:`Engine.parareal_jumps`,
:meth:`Engine.parareal_correct` and :meth:`Adaptive.adaptive_restart`.

If ``libpmd.so`` has not been built the import of the library fails loudly (there is no
CPU fallback); build it with ``python -m paper_2212_10508_gb300.build``.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpmd.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pmd.h")

PMD_OK, PMD_EINVAL, PMD_ENOMEM, PMD_ECUDA = 0, -1, -2, -3
PMD_ENEIGH, PMD_ENONFINITE, PMD_ETIMEOUT, PMD_ELOSTATOM, PMD_EUNSUPPORTED = -4, -5, -6, -7, -8
FP64, FP32_BULK = 0, 1
FINE, COARSE = 0, 1
SCHEME_PAPER, SCHEME_BAOAB = 0, 1
SCHED_NONE, SCHED_ROBUST, SCHED_L1_SYM = 0, 1, 2
METRIC_REL, METRIC_MAXDISP = 0, 1
ACT_ITERATE, ACT_DONE = 0, 1
MAX_NEIGHBORS = 64

_ERRNAMES = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENEIGH", -5: "ENONFINITE", -6: "ETIMEOUT",
             -7: "ELOSTATOM", -8: "EUNSUPPORTED"}


class PmdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "?"), code, msg))
        self.code = code


class SnapParams(ctypes.Structure):
    _fields_ = [("twojmax", ctypes.c_int), ("rcut", ctypes.c_double), ("rfac0", ctypes.c_double),
                ("rmin0", ctypes.c_double), ("switchflag", ctypes.c_int), ("precision", ctypes.c_int)]


class FSParams(ctypes.Structure):
    _fields_ = [("d", ctypes.c_double), ("A", ctypes.c_double), ("c", ctypes.c_double),
                ("c0", ctypes.c_double), ("c1", ctypes.c_double), ("c2", ctypes.c_double),
                ("precision", ctypes.c_int)]


class Langevin(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("gamma", ctypes.c_double), ("T", ctypes.c_double),
                ("mass", ctypes.c_double), ("scheme", ctypes.c_int), ("schedule", ctypes.c_int),
                ("seed", ctypes.c_uint64)]


COARSE_FS, COARSE_SNAP = 0, 1


class EngineParams(ctypes.Structure):
    _fields_ = [("fine", SnapParams), ("coarse", FSParams), ("box", ctypes.c_double * 3),
                ("natoms", ctypes.c_int), ("coarse_kind", ctypes.c_int), ("coarse_snap", SnapParams)]


class FineTuning(ctypes.Structure):
    """Run-time shape of the batched FP32 fine kernel (pmd_fine_tuning)."""
    _fields_ = [("rows2_atoms", ctypes.c_int), ("rows4_atoms", ctypes.c_int), ("b_group", ctypes.c_int),
                ("noise_stage", ctypes.c_int), ("warps", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Action(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n_in", ctypes.c_int), ("n_fin", ctypes.c_int),
                ("open_slab", ctypes.c_int), ("k", ctypes.c_int)]


EXPORTS = ["pmd_last_error", "pmd_snap_create", "pmd_snap_destroy", "pmd_snap_num_coeffs", "pmd_snap_flop_model",
           "pmd_snap_reserve",
           "snap_energy_forces", "pmd_snap_sync_status", "snap_energy_forces_noalloc", "eam_energy_forces", "pmd_engine_create",
           "pmd_engine_destroy", "pmd_engine_set_beta", "pmd_engine_reserve", "pmd_engine_profile", "pmd_sync_status",
           "pmd_engine_selftest_waits", "pmd_engine_get_tuning", "pmd_engine_set_tuning", "pmd_engine_autotune",
           "baoab_propagate_batch", "parareal_jumps", "parareal_correct", "pmd_adaptive_create",
           "pmd_adaptive_destroy", "adaptive_restart", "pmd_adaptive_cost", "pmd_adaptive_log", "sia_locate",
           "sia_residence", "pmd_alu_peak", "pmd_engine_set_coarse_beta"]

_lib = None


def lib():
    """Load ``libpmd.so`` (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libpmd.so is not built; run `python -m paper_2212_10508_gb300.build` "
                          "(the CUDA library is required, there is no CPU path)")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    i32, i64 = ctypes.c_int, ctypes.c_int64
    L.pmd_last_error.restype = ctypes.c_char_p
    L.pmd_snap_create.argtypes = [ctypes.POINTER(SnapParams), ctypes.POINTER(vp)]
    L.pmd_snap_destroy.argtypes = [vp]
    L.pmd_snap_num_coeffs.argtypes = [vp]
    L.pmd_snap_reserve.argtypes = [vp, i32, i32]
    L.pmd_snap_flop_model.argtypes = [vp, dp, dp]
    L.snap_energy_forces.argtypes = [vp, i32, i32, dp, vp, vp, vp, vp, vp, vp]
    L.pmd_snap_sync_status.argtypes = [vp, vp]
    L.snap_energy_forces_noalloc.argtypes = [vp, i32, i32, dp, vp, vp, vp, vp, vp, vp]
    L.eam_energy_forces.argtypes = [ctypes.POINTER(FSParams), i32, i32, dp, vp, vp, vp, vp]
    L.pmd_engine_create.argtypes = [ctypes.POINTER(EngineParams), ctypes.POINTER(vp)]
    L.pmd_engine_destroy.argtypes = [vp]
    L.pmd_engine_set_beta.argtypes = [vp, vp, vp]
    L.pmd_engine_reserve.argtypes = [vp, i32]
    L.pmd_engine_profile.argtypes = [vp, i32, dp]
    L.pmd_engine_selftest_waits.argtypes = [vp, i64, vp]
    L.pmd_sync_status.argtypes = [vp, vp]
    L.pmd_engine_get_tuning.argtypes = [vp, ctypes.POINTER(FineTuning)]
    L.pmd_engine_set_tuning.argtypes = [vp, ctypes.POINTER(FineTuning)]
    L.pmd_engine_autotune.argtypes = [vp, i32, i32, vp, vp, i64, vp, vp, ctypes.POINTER(Langevin), i32, vp,
                                      ctypes.POINTER(FineTuning), dp]
    L.baoab_propagate_batch.argtypes = [vp, i32, i32, i32, vp, vp, i64, vp, vp, ctypes.POINTER(Langevin), vp]
    L.parareal_jumps.argtypes = [vp, i32, vp, vp, vp, vp]
    L.parareal_correct.argtypes = [vp, i32, i32, vp, vp, vp, vp, ctypes.c_double, i32, i32,
                                   ctypes.POINTER(Langevin), dp, ip, vp]
    L.pmd_adaptive_create.argtypes = [i32, ctypes.c_double, ctypes.c_double, ctypes.POINTER(vp)]
    L.pmd_adaptive_destroy.argtypes = [vp]
    L.adaptive_restart.argtypes = [vp, ctypes.c_double, i32, ctypes.POINTER(Action)]
    L.pmd_adaptive_cost.argtypes = [vp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
    L.pmd_adaptive_log.argtypes = [vp, i32, ip, ip, ip, ip]
    L.sia_locate.argtypes = [i32, i32, i32, dp, vp, i64, vp, vp, vp, vp, vp]
    L.sia_residence.argtypes = [vp, i32, i32, vp, vp, ip]
    L.pmd_alu_peak.argtypes = [i32, ctypes.c_double, vp, dp, dp]
    L.pmd_engine_set_coarse_beta.argtypes = [vp, vp, vp]
    _lib = L
    return L


def _check(rc):
    if rc != PMD_OK:
        raise PmdError(rc, lib().pmd_last_error().decode())


def _ptr(t, dtype="f64"):
    """Device pointer of a contiguous CUDA tensor of the given element type ("f64", "i32" or
    "i64"; the C ABI reads the bytes as that type), or None."""
    if t is None:
        return None
    import torch
    want = {"f64": torch.float64, "i32": torch.int32, "i64": torch.int64}[dtype]
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if t.dtype != want:
        raise TypeError("expected a %s tensor, got %s" % (want, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _box(box):
    return (ctypes.c_double * 3)(*[float(x) for x in box])


def snap_params(twojmax=8, rcut=4.73, rfac0=0.99363, switchflag=1, precision=FP64):
    return SnapParams(twojmax, rcut, rfac0, 0.0, switchflag, precision)


def fs_params(d=4.400224, A=1.896373, c=3.25, c0=47.1346499, c1=-33.7665655, c2=6.2541999, precision=FP64):
    return FSParams(d, A, c, c0, c1, c2, precision)


def langevin(dt=1e-3, gamma=1.0, T=1000.0, mass=183.84, scheme=SCHEME_PAPER, schedule=SCHED_ROBUST, seed=12345):
    return Langevin(dt, gamma, T, mass, scheme, schedule, seed & 0xFFFFFFFFFFFFFFFF)


PEAK_FFMA, PEAK_FFMA2, PEAK_DFMA = 0, 1, 2


def alu_peak(kind, seconds=0.2, stream=None):
    """Measured FMA throughput of the current device in TFLOP/s (pmd_alu_peak)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().pmd_alu_peak(kind, seconds, _stream(stream), ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value


class Snap:
    """SNAP context (tables and scratch on the current device)."""

    def __init__(self, params: SnapParams = None, **kw):
        self.params = params or snap_params(**kw)
        h = ctypes.c_void_p()
        _check(lib().pmd_snap_create(ctypes.byref(self.params), ctypes.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.pmd_snap_destroy(self.h)
            self.h = None

    @property
    def num_coeffs(self):
        return lib().pmd_snap_num_coeffs(self.h)

    def reserve(self, nbatch, natoms):
        _check(lib().pmd_snap_reserve(self.h, nbatch, natoms))

    def flop_model(self):
        """(operations per neighbour pair, operations per atom) of the force kernels."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(lib().pmd_snap_flop_model(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def sync_status(self, stream=None):
        _check(lib().pmd_snap_sync_status(self.h, _stream(stream)))


def snap_energy_forces(snap: Snap, pos, box, beta, energy=True, forces=True, sumB=False, stream=None):
    """SNAP energies [nb], forces [nb,3,n], dE/dbeta [nb,1+nB] for positions pos [nb,3,n]."""
    import torch
    nb, _, n = pos.shape
    E = torch.empty(nb, dtype=torch.float64, device=pos.device) if energy else None
    F = torch.empty_like(pos) if forces else None
    S = torch.empty(nb, snap.num_coeffs, dtype=torch.float64, device=pos.device) if sumB else None
    _check(lib().snap_energy_forces(snap.h, nb, n, _box(box), _ptr(pos), _ptr(beta), _ptr(E), _ptr(F), _ptr(S),
                                    _stream(stream)))
    return E, F, S


def sia_locate(frames, ref, sites, box, stream=None):
    """Well of the self-interstitial in every frame (Wigner-Seitz: most occupied site of the
    reference lattice `sites` [3,nsites] shifted by the frame's centre-of-mass displacement from
    `ref` [3,n]).  frames [nf, rows, n] float64 with the positions in rows 0..2 (rows = 3, or 6
    for the states of a parareal run).  Returns (well, occupancy), int32 [nf] CUDA tensors."""
    import torch
    nf, rows, n = frames.shape
    if rows < 3:
        raise ValueError("frames need at least 3 rows (positions)")
    well = torch.empty(nf, dtype=torch.int32, device=frames.device)
    occ = torch.empty(nf, dtype=torch.int32, device=frames.device)
    _check(lib().sia_locate(nf, n, sites.shape[1], _box(box), _ptr(frames), rows * n, _ptr(ref), _ptr(sites),
                            _ptr(well, "i32"), _ptr(occ, "i32"), _stream(stream)))
    return well, occ


def sia_residence(well):
    """Completed residence times (frames) of a well sequence and the well of each residence
    (the last, still open, run is left out): (lengths, sites) as int32 numpy arrays."""
    w = well.detach().cpu().numpy() if hasattr(well, "detach") else well
    w = np.ascontiguousarray(w, dtype=np.int32)
    nf = int(w.shape[0])
    lengths = np.empty(max(nf, 1), np.int32)
    sites = np.empty(max(nf, 1), np.int32)
    k = ctypes.c_int()
    _check(lib().sia_residence(w.ctypes.data_as(ctypes.c_void_p), nf, nf, lengths.ctypes.data_as(ctypes.c_void_p),
                               sites.ctypes.data_as(ctypes.c_void_p), ctypes.byref(k)))
    return lengths[:k.value].copy(), sites[:k.value].copy()


def eam_energy_forces(pos, box, params: FSParams = None, energy=True, forces=True, stream=None):
    """Finnis-Sinclair energies [nb] and forces [nb,3,n]."""
    import torch
    params = params or fs_params()
    nb, _, n = pos.shape
    E = torch.empty(nb, dtype=torch.float64, device=pos.device) if energy else None
    F = torch.empty_like(pos) if forces else None
    _check(lib().eam_energy_forces(ctypes.byref(params), nb, n, _box(box), _ptr(pos), _ptr(E), _ptr(F),
                                   _stream(stream)))
    return E, F


class Engine:
    """Fine (SNAP) + coarse potentials on one periodic cell of ``natoms`` atoms.  The coarse
    potential is Finnis-Sinclair EAM (``coarse``), or SNAP with 2J = 2 when ``coarse_snap``
    (SnapParams) is given, with coefficients ``coarse_beta`` (Strategy I of the paper)."""

    def __init__(self, natoms, box, fine: SnapParams = None, coarse: FSParams = None, beta=None,
                 coarse_snap: SnapParams = None, coarse_beta=None):
        kind = COARSE_SNAP if coarse_snap is not None else COARSE_FS
        self.params = EngineParams(fine or snap_params(), coarse or fs_params(), (ctypes.c_double * 3)(*box),
                                   natoms, kind, coarse_snap or snap_params(twojmax=2))
        h = ctypes.c_void_p()
        _check(lib().pmd_engine_create(ctypes.byref(self.params), ctypes.byref(h)))
        self.h = h
        self.natoms = natoms
        self.box = tuple(float(x) for x in box)
        if beta is not None:
            self.set_beta(beta)
        if coarse_beta is not None:
            self.set_coarse_beta(coarse_beta)

    def set_coarse_beta(self, beta, stream=None):
        _check(lib().pmd_engine_set_coarse_beta(self.h, _ptr(beta), _stream(stream)))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.pmd_engine_destroy(self.h)
            self.h = None

    def set_beta(self, beta, stream=None):
        _check(lib().pmd_engine_set_beta(self.h, _ptr(beta), _stream(stream)))

    def reserve(self, nbatch):
        _check(lib().pmd_engine_reserve(self.h, nbatch))

    def sync_status(self, stream=None):
        _check(lib().pmd_sync_status(self.h, _stream(stream)))

    def selftest_waits(self, polls=1000, stream=None):
        """Run the bounded-wait self-test; the next sync_status raises PmdError(ETIMEOUT)."""
        _check(lib().pmd_engine_selftest_waits(self.h, int(polls), _stream(stream)))

    def profile(self, enable=True):
        """Enable/disable kernel timing; returns the last persistent-kernel duration in ms (or -1)."""
        ms = ctypes.c_double()
        _check(lib().pmd_engine_profile(self.h, 1 if enable else 0, ctypes.byref(ms)))
        return ms.value

    def tuning(self):
        """The engine's run-time shape of the batched FP32 fine kernel, as a dict."""
        t = FineTuning()
        _check(lib().pmd_engine_get_tuning(self.h, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, **kw):
        t = FineTuning(**{**self.tuning(), **kw})
        _check(lib().pmd_engine_set_tuning(self.h, ctypes.byref(t)))

    def autotune(self, q, v, nsteps, interval_id, lp: Langevin, max_steps=64, stream=None):
        """Time candidate shapes on a copy of this batch (lengths scaled to at most max_steps) and
        keep the fastest; returns (shape dict, best ms).  q, v as in baoab_propagate_batch."""
        nb = q.shape[0]
        if v is None:
            qp = _ptr(q)
            vp = ctypes.c_void_p(qp.value + 3 * self.natoms * 8)
            stride = 6 * self.natoms
        else:
            qp, vp, stride = _ptr(q), _ptr(v), 3 * self.natoms
        t, ms = FineTuning(), ctypes.c_double()
        _check(lib().pmd_engine_autotune(self.h, nb, self.natoms, qp, vp, stride, _ptr(nsteps, "i32"), _ptr(interval_id, "i64"),
                                         ctypes.byref(lp), int(max_steps), _stream(stream), ctypes.byref(t),
                                         ctypes.byref(ms)))
        return t.as_dict(), ms.value

    def baoab_propagate_batch(self, potential, q, v, nsteps, interval_id, lp: Langevin, stream=None):
        """Propagate members in place.  q, v: [nb,3,n]; or v=None and q packed states [nb,6,n]
        (positions then velocities of each member)."""
        nb = q.shape[0]
        if v is None:
            assert q.shape[1] == 6
            qp = _ptr(q)
            vp = ctypes.c_void_p(qp.value + 3 * self.natoms * 8)
            stride = 6 * self.natoms
        else:
            qp, vp, stride = _ptr(q), _ptr(v), 3 * self.natoms
        _check(lib().baoab_propagate_batch(self.h, potential, nb, self.natoms, qp, vp, stride,
                                           _ptr(nsteps, "i32"), _ptr(interval_id, "i64"), ctypes.byref(lp), _stream(stream)))

    def parareal_jumps(self, count, fine_out, coarse_prev, jumps, stream=None):
        _check(lib().parareal_jumps(self.h, count, _ptr(fine_out), _ptr(coarse_prev), _ptr(jumps), _stream(stream)))

    def parareal_correct(self, n_in, n_fin, jumps, prev, cur, coarse_out, delta_expl, metric, L, lp: Langevin,
                         stream=None):
        """Sequential correction sweep; returns (delta, n_stop).  Synchronises the stream."""
        d = ctypes.c_double()
        ns = ctypes.c_int()
        _check(lib().parareal_correct(self.h, n_in, n_fin, _ptr(jumps), _ptr(prev), _ptr(cur), _ptr(coarse_out),
                                      float(delta_expl), metric, L, ctypes.byref(lp), ctypes.byref(d),
                                      ctypes.byref(ns), _stream(stream)))
        return d.value, ns.value


class Adaptive:
    """Host state machine of Algorithm 2 (adaptive_restart) and the cost model of eqs. (7)-(9)."""

    def __init__(self, N, delta_conv, delta_expl):
        h = ctypes.c_void_p()
        _check(lib().pmd_adaptive_create(N, delta_conv, delta_expl, ctypes.byref(h)))
        self.h = h
        self.N = N

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.pmd_adaptive_destroy(self.h)
            self.h = None

    def adaptive_restart(self, delta=0.0, n_stop=-1):
        a = Action()
        _check(lib().adaptive_restart(self.h, float(delta), int(n_stop), ctypes.byref(a)))
        return a

    def cost(self, C_f, C_c):
        c, g, gi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib().pmd_adaptive_cost(self.h, C_f, C_c, ctypes.byref(c), ctypes.byref(g), ctypes.byref(gi)))
        return c.value, g.value, gi.value

    def log(self):
        n = lib().pmd_adaptive_log(self.h, 0, None, None, None, None)
        arrs = [(ctypes.c_int * max(n, 1))() for _ in range(4)]
        lib().pmd_adaptive_log(self.h, n, *arrs)
        return [tuple(a[i] for a in arrs) for i in range(n)]   # (n_init, n_final, k, slab)


def adaptive_parareal(engine: Engine, q0, v0, N, L, delta_conv, delta_expl, lp: Langevin, metric=METRIC_REL,
                      max_iter=100000, stream=None):
    """Algorithm 2 on the GPU: returns (states [N+1,6,n], Adaptive).

    Per iteration: prev := cur on the slab, the fine batch F(prev_n) for all intervals of the
    slab in one launch, J_n = F(prev_n) - C(prev_n) with C(prev_n) cached from the previous
    sweep, then the sequential sweep (two host scalars come back)."""
    import torch
    n = engine.natoms
    dev = q0.device
    cur = torch.empty(N + 1, 6, n, dtype=torch.float64, device=dev)
    cur[0, :3] = q0
    cur[0, 3:] = v0
    cache = torch.zeros(max(N, 1), 6, n, dtype=torch.float64, device=dev)   # C(cur_n) of the last sweep
    st = Adaptive(N, delta_conv, delta_expl)
    act = st.adaptive_restart()
    ids_all = torch.arange(N, dtype=torch.int64, device=dev)
    iters = 0
    while act.kind == ACT_ITERATE:
        a, b = act.n_in, act.n_fin
        cnt = b - a
        if act.open_slab:      # coarse initialisation of the slab: cur_{n+1} = C(cur_n)
            engine.parareal_correct(a, b, None, cur[a:b + 1], cur[a:b + 1], cache[a:b], float("inf"), metric, L, lp,
                                    stream)
        prev = cur[a:b + 1].clone()
        fine = prev[:cnt].clone()
        nsteps = torch.full((cnt,), L, dtype=torch.int32, device=dev)
        engine.baoab_propagate_batch(FINE, fine, None, nsteps, ids_all[a:b], lp, stream=stream)
        jumps = torch.empty_like(fine)
        engine.parareal_jumps(cnt, fine, cache[a:b], jumps, stream)
        delta, n_stop = engine.parareal_correct(a, b, jumps, prev, cur[a:b + 1], cache[a:b], delta_expl, metric, L,
                                                lp, stream)
        act = st.adaptive_restart(delta, n_stop)
        iters += 1
        if iters > max_iter:
            raise RuntimeError("adaptive parareal did not terminate")
    return cur, st
