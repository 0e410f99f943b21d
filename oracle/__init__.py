"""FP64 CPU oracle for the adaptive-parareal Langevin hot path (arXiv 2212.10508).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
It shares no code with the CUDA library in ``paper_2212_10508_gb300/`` and never
imports it.

Contents:
  * ``liboracle.so`` (``pmd_oracle.c``): Philox4x32-10 + Box-Muller noise, brute-force
    neighbours, Finnis-Sinclair EAM, SNAP by the explicit Wigner formula and a direct
    product-rule gradient, the Langevin schemes of eqs. (2)-(3)/(11)-(12) and BAOAB.
  * ``oracle.parareal``: Alg. 1 (classical parareal), Alg. 2 (adaptive parareal) and
    the cost / gain model of eqs. (7)-(9), written in the paper's order and notation.
  * ``oracle.sia``: the interstitial's well in each frame (Wigner-Seitz reading of the
    Voronoi analysis of Sec. 3) and its residence times.

Parity status of each function is listed in the module docstrings.  The Philox bit
stream has no published known-answer vectors here; it is pinned bitwise against cuRAND's
device Philox4_32_10, an independent implementation of the same published generator
(tests/test_gpu_philox_curand.py, which runs on a GPU), and statistically on the CPU.
"""
import ctypes
import os

import numpy as np

from . import build as _build

KB = 8.617333262e-5          # eV/K
FTOA = 9648.533215665        # 1 eV/(Angstrom u) in Angstrom/ps^2

POT_SNAP, POT_FS, POT_ZERO = 0, 1, 2
SCHEME_PAPER, SCHEME_BAOAB = 0, 1
SCHED_NONE, SCHED_ROBUST, SCHED_L1_SYM = 0, 1, 2


class SnapParams(ctypes.Structure):
    _fields_ = [("twojmax", ctypes.c_int), ("rcut", ctypes.c_double), ("rfac0", ctypes.c_double),
                ("rmin0", ctypes.c_double), ("switchflag", ctypes.c_int)]


class FSParams(ctypes.Structure):
    _fields_ = [("d", ctypes.c_double), ("A", ctypes.c_double), ("c", ctypes.c_double),
                ("c0", ctypes.c_double), ("c1", ctypes.c_double), ("c2", ctypes.c_double)]


class Potential(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("snap", SnapParams),
                ("beta", ctypes.POINTER(ctypes.c_double)), ("fs", FSParams)]


class Langevin(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("gamma", ctypes.c_double), ("T", ctypes.c_double),
                ("mass", ctypes.c_double), ("scheme", ctypes.c_int), ("schedule", ctypes.c_int),
                ("seed", ctypes.c_uint64)]


_lib = None


def lib():
    """Load (building first if needed) ``liboracle.so``."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        L.or_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
        L.or_normals3.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, dp]
        L.or_cg.restype = ctypes.c_double
        L.or_cg.argtypes = [ctypes.c_int] * 6
        L.or_wigner_u.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [dp]
        L.or_snap_triples.argtypes = [ctypes.c_int, ip]
        L.or_snap_energy_forces.argtypes = [ctypes.POINTER(SnapParams), ctypes.c_int, ctypes.c_int, dp,
                                            dp, dp, dp, dp, dp, dp]
        L.or_fs_energy_forces.argtypes = [ctypes.POINTER(FSParams), ctypes.c_int, ctypes.c_int, dp, dp,
                                          dp, dp]
        L.or_neighbors.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int, ip, ip]
        L.or_propagate.argtypes = [ctypes.POINTER(Potential), ctypes.c_int, ctypes.c_int, dp, dp, dp,
                                   ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(Langevin)]
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    return lib().or_num_threads()


def philox4x32_10(ctr, key):
    """Raw Philox4x32-10 block (4 x uint32) for counter ``ctr`` (4) and key ``key`` (2)."""
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def normals3(seed: int, n: int, ell: int, atom: int) -> np.ndarray:
    """G_{ell,n} for one atom (x, y, z)."""
    g = np.zeros(3)
    lib().or_normals3(seed & 0xFFFFFFFFFFFFFFFF, n, ell, atom, _dp(g))
    return g


def cg(tj1, tm1, tj2, tm2, tJ, tM) -> float:
    """Clebsch-Gordan <j1 m1 j2 m2 | J M>, doubled arguments (Racah formula)."""
    return lib().or_cg(tj1, tm1, tj2, tm2, tJ, tM)


def wigner_u(tj: int, a: complex, b: complex) -> np.ndarray:
    """U^j(a,b) as a (2j+1)x(2j+1) complex matrix, rows m' = -j..j, columns m = -j..j."""
    n = tj + 1
    out = np.zeros(2 * n * n)
    lib().or_wigner_u(tj, a.real, a.imag, b.real, b.imag, _dp(out))
    return (out[0::2] + 1j * out[1::2]).reshape(n, n)


def snap_triples(twojmax: int) -> np.ndarray:
    """Bispectrum triples (2j1, 2j2, 2j) with j2 <= j1 <= j, in the order of beta[1:]."""
    n = lib().or_snap_triples(twojmax, None)
    out = (ctypes.c_int * (3 * n))()
    lib().or_snap_triples(twojmax, out)
    return np.array(list(out), dtype=np.int64).reshape(n, 3)


def snap_params(twojmax=8, rcut=4.73, rfac0=0.99363, rmin0=0.0, switchflag=1) -> SnapParams:
    return SnapParams(twojmax, rcut, rfac0, rmin0, switchflag)


def fs_params(d=4.400224, A=1.896373, c=3.25, c0=47.1346499, c1=-33.7665655, c2=6.2541999) -> FSParams:
    return FSParams(d, A, c, c0, c1, c2)


def snap_energy_forces(pos, box, beta, params: SnapParams = None, want_B=False):
    """SNAP energies [nb], forces [nb,3,n], sumB [nb,1+nB] (and per-atom B [nb,n,nB])."""
    params = params or snap_params()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    if pos.ndim == 2:
        pos = pos[None]
    nb, _, n = pos.shape
    nt = len(snap_triples(params.twojmax))
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    assert beta.shape == (1 + nt,)
    E = np.zeros(nb)
    F = np.zeros((nb, 3, n))
    sB = np.zeros((nb, 1 + nt))
    Bat = np.zeros((nb, n, nt)) if want_B else None
    boxa = np.ascontiguousarray(box, dtype=np.float64)
    rc = lib().or_snap_energy_forces(ctypes.byref(params), nb, n, _dp(boxa), _dp(pos), _dp(beta), _dp(E),
                                     _dp(F), _dp(sB), _dp(Bat))
    if rc != 0:
        raise ValueError("or_snap_energy_forces failed")
    return (E, F, sB, Bat) if want_B else (E, F, sB)


def fs_energy_forces(pos, box, params: FSParams = None):
    """Finnis-Sinclair energies [nb] and forces [nb,3,n]."""
    params = params or fs_params()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    if pos.ndim == 2:
        pos = pos[None]
    nb, _, n = pos.shape
    E = np.zeros(nb)
    F = np.zeros((nb, 3, n))
    boxa = np.ascontiguousarray(box, dtype=np.float64)
    rc = lib().or_fs_energy_forces(ctypes.byref(params), nb, n, _dp(boxa), _dp(pos), _dp(E), _dp(F))
    if rc != 0:
        raise ValueError("or_fs_energy_forces failed")
    return E, F


def neighbors(pos, box, rc, nmax=64):
    """Brute-force minimum-image neighbour lists (sorted), for one system [3,n]."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[1]
    cnt = (ctypes.c_int * n)()
    lst = (ctypes.c_int * (n * nmax))()
    boxa = np.ascontiguousarray(box, dtype=np.float64)
    m = lib().or_neighbors(n, _dp(pos), _dp(boxa), rc, nmax, cnt, lst)
    if m < 0:
        raise OverflowError("neighbour capacity exceeded")
    c = np.array(list(cnt))
    L = np.array(list(lst)).reshape(n, nmax)
    return [L[i, :c[i]].copy() for i in range(n)]


def potential(kind, beta=None, snap: SnapParams = None, fs: FSParams = None):
    """Build a ``Potential``; keeps a reference to ``beta`` on the returned object."""
    p = Potential()
    p.kind = kind
    p.snap = snap or snap_params()
    p.fs = fs or fs_params()
    if beta is not None:
        b = np.ascontiguousarray(beta, dtype=np.float64)
        p.beta = _dp(b)
        p._beta_keep = b
    return p


def langevin(dt=1e-3, gamma=1.0, T=1000.0, mass=183.84, scheme=SCHEME_PAPER, schedule=SCHED_ROBUST,
             seed=12345) -> Langevin:
    return Langevin(dt, gamma, T, mass, scheme, schedule, seed & 0xFFFFFFFFFFFFFFFF)


def propagate(pot: Potential, q, v, box, nsteps, interval_id, lp: Langevin):
    """Propagate members in place: q, v arrays [nb,3,n] (float64, C-contiguous)."""
    assert q.dtype == np.float64 and v.dtype == np.float64 and q.flags["C_CONTIGUOUS"] and v.flags["C_CONTIGUOUS"]
    nb, _, n = q.shape
    ns = np.ascontiguousarray(nsteps, dtype=np.int32)
    ids = np.ascontiguousarray(interval_id, dtype=np.int64)
    assert ns.shape == (nb,) and ids.shape == (nb,)
    boxa = np.ascontiguousarray(box, dtype=np.float64)
    rc = lib().or_propagate(ctypes.byref(pot), nb, n, _dp(boxa), _dp(q), _dp(v),
                            ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                            ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ctypes.byref(lp))
    if rc != 0:
        raise ValueError("or_propagate failed")
