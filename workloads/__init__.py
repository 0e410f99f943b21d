"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds none of the method's arithmetic: only geometry (a BCC tungsten
supercell with a <111> dumbbell self-interstitial, the system of Sec. 3.1), seeded
random draws (thermal displacements, Maxwell-Boltzmann velocities, random SNAP
coefficients, uneven interval lengths) and the workload definitions.

Recipe:
  * lattice: n x n x n conventional BCC cells, a = 3.1652 Angstrom, periodic box n*a;
  * SIA: the atom at the site nearest the box centre is replaced by two atoms at
    s +- 1.1 Angstrom * (1,1,1)/sqrt(3)  (2 n^3 + 1 atoms);
  * displacements: i.i.d. N(0, sigma^2) per coordinate (sigma = 0.05 Angstrom);
  * velocities: i.i.d. N(0, k_B T / m) per coordinate, centre-of-mass velocity removed;
  * SNAP coefficients: beta_0 = -8.9 eV, beta_t ~ N(0, 0.01^2) (parity inputs), or the
    coefficients fitted to Finnis-Sinclair tungsten stored in tests/golden/beta_fs_w_2j8.txt
    (long trajectories: random coefficients have no repulsive core and the cell collapses);
  * interval lengths: L_b ~ U{100, ..., 2000}.
Every draw comes from numpy's PCG64 seeded by a SplitMix64-derived sub-seed of one
master seed, so each stream is reproducible on its own.
"""
import os

import numpy as np

A_W = 3.1652             # BCC tungsten lattice constant, Angstrom
M_W = 183.84             # u
KB = 8.617333262e-5      # eV/K
FTOA = 9648.533215665    # eV/(Angstrom u) -> Angstrom/ps^2

SNAP = dict(twojmax=8, rcut=4.73, rfac0=0.99363, rmin0=0.0, switchflag=1)
FS_W = dict(d=4.400224, A=1.896373, c=3.25, c0=47.1346499, c1=-33.7665655, c2=6.2541999)
BETA0 = -8.9


def splitmix64(x: int) -> int:
    """One SplitMix64 output for state x (used only to derive independent sub-seeds)."""
    z = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


def subseed(master: int, stream: int) -> int:
    return splitmix64((master * 0x100000001B3 + stream) & 0xFFFFFFFFFFFFFFFF)


def rng(master: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(subseed(master, stream)))


def bcc(ncell: int, a: float = A_W):
    """Perfect BCC positions [3, 2 ncell^3] and the orthorhombic box [3]."""
    g = np.arange(ncell, dtype=np.float64)
    cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
    corner = np.stack([cx.ravel(), cy.ravel(), cz.ravel()])
    pos = np.concatenate([corner, corner + 0.5], axis=1) * a
    box = np.full(3, ncell * a)
    return np.ascontiguousarray(pos), box


def bcc_sia(ncell: int, a: float = A_W, split: float = 1.1):
    """BCC supercell with one <111> dumbbell interstitial: [3, 2 ncell^3 + 1] and box."""
    pos, box = bcc(ncell, a)
    centre = box / 2
    s = int(np.argmin(np.sum((pos - centre[:, None]) ** 2, axis=0)))
    site = pos[:, s].copy()
    u = np.ones(3) / np.sqrt(3.0)
    rest = np.delete(pos, s, axis=1)
    out = np.concatenate([rest, (site + split * u)[:, None], (site - split * u)[:, None]], axis=1)
    return np.ascontiguousarray(out), box


def bcc_sia_at(ncell: int, site: int, axis, a: float = A_W, split: float = 1.1):
    """BCC supercell with the <111> dumbbell at lattice site `site` (an index of bcc()) along
    axis (+-1, +-1, +-1): the site's atom is replaced by two atoms at s +- split * axis/sqrt(3)."""
    pos, box = bcc(ncell, a)
    u = np.asarray(axis, dtype=np.float64) / np.sqrt(3.0)
    x = pos[:, site].copy()
    rest = np.delete(pos, site, axis=1)
    out = np.concatenate([rest, (x + split * u)[:, None], (x - split * u)[:, None]], axis=1)
    return np.ascontiguousarray(out), box


def fit_starts(master: int, groups: int, members: int, ncell: int = 4, tmin: float = 500.0,
               tmax: float = 3000.0, sigma: float = 0.02):
    """Starting states of the beta-fitting training set (config 4): `groups` temperatures drawn
    uniformly in [tmin, tmax] K, each with `members` cells whose <111> dumbbell sits at a random
    lattice site along a random one of the four <111> axes (random sign), with N(0, sigma^2)
    displacements and Maxwell-Boltzmann velocities at the group's temperature.
    Returns (list of (q [members,3,n], v [members,3,n]) per group, temperatures [groups], box)."""
    g = rng(master, 31)
    temps = g.uniform(tmin, tmax, size=groups)
    nsite = 2 * ncell ** 3
    starts = []
    box = None
    for k in range(groups):
        qs = []
        for m in range(members):
            axis = g.choice([-1.0, 1.0], size=3)
            cell, box = bcc_sia_at(ncell, int(g.integers(nsite)), axis)
            qs.append(cell)
        q = np.ascontiguousarray(np.array(qs) + rng(master, 1000 + k).normal(0.0, sigma, size=(members,) + qs[0].shape))
        v = velocities(qs[0].shape[1], temps[k], rng(master, 2000 + k), count=members)
        starts.append((q, v))
    return starts, temps, box


def displaced(pos, sigma, gen: np.random.Generator, count=None):
    """count copies (or one if None) of pos with i.i.d. Gaussian displacements."""
    if count is None:
        return np.ascontiguousarray(pos + gen.normal(0.0, sigma, size=pos.shape))
    return np.ascontiguousarray(pos[None] + gen.normal(0.0, sigma, size=(count,) + pos.shape))


def velocities(natoms, T, gen: np.random.Generator, count=None, mass=M_W):
    """Maxwell-Boltzmann velocities in Angstrom/ps, centre-of-mass motion removed."""
    s = np.sqrt(KB * T / mass * FTOA)
    shape = (3, natoms) if count is None else (count, 3, natoms)
    v = gen.normal(0.0, s, size=shape)
    v -= v.mean(axis=-1, keepdims=True)
    return np.ascontiguousarray(v)


def snap_beta(nB, gen: np.random.Generator, std=0.01, beta0=BETA0):
    b = np.empty(1 + nB)
    b[0] = beta0
    b[1:] = gen.normal(0.0, std, size=nB)
    return b


GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")


def fitted_beta(twojmax: int = 8):
    """SNAP coefficients (1 + nB) fitted to Finnis-Sinclair W by the oracle: 2J = 8 (the bench's
    potential), 2J = 6 (config 4's recipe) or 2J = 2 (SNAP-6, the coarse potential of Strategy I);
    see tests/golden/make_fitted_beta.py."""
    name = {8: "beta_fs_w_2j8.txt", 6: "beta_fs_w_2j6.txt", 2: "beta_fs_w_2j2.txt"}[twojmax]
    vals = [float(ln) for ln in open(os.path.join(GOLDEN, name)) if ln.strip() and ln[0] != "#"]
    return np.array(vals)


def n_bispectrum(twojmax: int) -> int:
    """Number of triples j2 <= j1 <= j <= J/2 with j <= j1 + j2 and integer j1+j2+j."""
    c = 0
    for tj1 in range(twojmax + 1):
        for tj2 in range(tj1 + 1):
            for tj in range(tj1, twojmax + 1):
                if tj <= tj1 + tj2 and (tj1 + tj2 + tj) % 2 == 0:
                    c += 1
    return c


def interval_lengths(count, gen: np.random.Generator, lo=100, hi=2000):
    return gen.integers(lo, hi + 1, size=count).astype(np.int32)


# ---- the workloads ------------------------------------------------------------------

def small_system(master=2212, nconf=16, sigma=0.05, twojmax=8):
    """129 atoms (4^3 cells + SIA), nconf displaced copies, random beta."""
    pos, box = bcc_sia(4)
    P = displaced(pos, sigma, rng(master, 1), count=nconf)
    beta = snap_beta(n_bispectrum(twojmax), rng(master, 2))
    return P, box, beta


def batch_workload(master=2212, nbatch=64, T=1500.0, lo=100, hi=2000, ncell=4, sigma=0.05, twojmax=8,
                   fitted=True):
    """nbatch members of the (ncell^3 + SIA) system with uneven lengths L_b ~ U{lo..hi};
    fitted=True uses the coefficients fitted to Finnis-Sinclair W, else random ones."""
    pos, box = bcc_sia(ncell)
    n = pos.shape[1]
    q = displaced(pos, sigma, rng(master, 11), count=nbatch)
    v = velocities(n, T, rng(master, 12), count=nbatch)
    beta = fitted_beta() if (fitted and twojmax == 8) else snap_beta(n_bispectrum(twojmax), rng(master, 2))
    L = interval_lengths(nbatch, rng(master, 13), lo, hi)
    ids = np.arange(nbatch, dtype=np.int64)
    return q, v, box, beta, L, ids


def sia_frames(ncell, nframes, gen: np.random.Generator, sigma=0.08, hop=0.05, drift=0.05, images=True,
               a: float = A_W, split: float = 1.1):
    """Synthetic interstitial trajectory for the tracking tests: atoms keep their identity; the
    doubly occupied site (a <111> dumbbell, orientation sign drawn per frame) hops with
    probability `hop` per frame by moving one of its two atoms to one of the 8 nearest-neighbour
    sites (which then holds the new dumbbell); every frame adds i.i.d. N(0, sigma^2) displacements and a common drift
    (a Gaussian random walk with step `drift` per coordinate); if `images`, every atom's
    coordinates carry fixed box-vector offsets (-1, 0, +1), as unwrapped coordinates do.  Returns (frames [nf, 3, n], sites [3, ns],
    box, intended wells [nf])."""
    sites, box = bcc(ncell, a)
    ns = sites.shape[1]
    s0 = int(gen.integers(ns))
    home = np.concatenate([np.arange(ns), [s0]])          # atom i sits on site home[i]
    n = ns + 1
    u = np.ones(3) / np.sqrt(3.0)
    frames = np.empty((nframes, 3, n))
    wells = np.empty(nframes, np.int32)
    shift = np.zeros(3)
    offs = box[:, None] * gen.integers(-1, 2, size=(3, n)) if images else np.zeros((3, n))
    for f in range(nframes):
        if f > 0 and gen.random() < hop:
            w0 = wells[f - 1]
            pair = np.flatnonzero(home == w0)
            dd = sites - sites[:, w0:w0 + 1]
            dd -= box[:, None] * np.rint(dd / box[:, None])
            near = np.flatnonzero(np.abs(np.sqrt(np.sum(dd * dd, axis=0)) - a * np.sqrt(3.0) / 2) < 1e-6)
            home[pair[int(gen.integers(2))]] = int(near[int(gen.integers(near.size))])
        cnt = np.bincount(home, minlength=ns)
        w = int(np.flatnonzero(cnt == 2)[0])
        wells[f] = w
        q = sites[:, home].copy()
        pair = np.flatnonzero(home == w)
        sign = 1.0 if gen.random() < 0.5 else -1.0
        q[:, pair[0]] += sign * split * u
        q[:, pair[1]] -= sign * split * u
        if f > 0:
            shift = shift + gen.normal(0.0, drift, size=3)
        frames[f] = q + shift[:, None] + gen.normal(0.0, sigma, size=q.shape) + offs
    return frames, sites, box, wells
