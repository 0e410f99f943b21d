"""Oracle of the interstitial tracking (TEST INFRASTRUCTURE ONLY: see the package docstring).

The paper locates the self-interstitial atom in each frame by a Voronoi analysis and counts the
time steps the system spends in each well (Sec. 3: the table of residence times and the
statistical study of the mean residence time with a 95 % confidence interval).  Reading used
(Wigner-Seitz): every atom belongs to the nearest site of the reference lattice shifted by the
frame's centre-of-mass displacement; the interstitial's well is the most occupied site (the
smallest index on ties); a residence time is the length of a run of frames with the same well,
the last (still open) run excluded.

The arithmetic is the definition written out in FP64 in a fixed order (sequential centre-of-mass
sums, unfused products), the order the C ABI documents, so that nearest-site decisions can be
compared bit for bit.  Pinned in tests/test_oracle_sia.py against a periodic k-d tree query
(scipy), lattice symmetries and hand-made sequences.
"""
import numpy as np


def com_shift(q, ref):
    """Centre-of-mass displacement of positions q [3,n] from ref [3,n]: per axis, the sum over
    atoms in index order of (q - ref), divided by n."""
    n = q.shape[1]
    c = np.zeros(3)
    for a in range(3):
        s = 0.0
        for i in range(n):
            s = s + (float(q[a, i]) - float(ref[a, i]))
        c[a] = s / n
    return c


def nearest_sites(q, c, sites, box):
    """Index of the nearest site (minimum image, smallest index on ties) of every atom of q [3,n]
    after the shift c [3]; sites [3,ns]."""
    p = q - c[:, None]                                   # [3, n]
    d = p[:, :, None] - sites[:, None, :]                # [3, n, ns]
    L = np.asarray(box, dtype=np.float64)[:, None, None]
    d = d - L * np.rint(d / L)
    r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]       # unfused, left to right
    return np.argmin(r2, axis=1)                          # first minimum = smallest index


def locate(frames, ref, sites, box):
    """(well, occupancy) int arrays [nf] of frames [nf, >=3, n] (positions in rows 0..2)."""
    nf = frames.shape[0]
    well = np.zeros(nf, np.int32)
    occ = np.zeros(nf, np.int32)
    for f in range(nf):
        q = np.asarray(frames[f, :3], dtype=np.float64)
        s = nearest_sites(q, com_shift(q, ref), sites, box)
        cnt = np.bincount(s, minlength=sites.shape[1])
        well[f] = int(np.argmax(cnt))                     # first maximum = smallest index
        occ[f] = int(cnt[well[f]])
    return well, occ


def residence(well):
    """Completed runs of equal consecutive wells: (lengths, sites); the last run is open."""
    lengths, sites = [], []
    start = 0
    for f in range(1, len(well)):
        if well[f] != well[f - 1]:
            lengths.append(f - start)
            sites.append(int(well[f - 1]))
            start = f
    return np.array(lengths, np.int32), np.array(sites, np.int32)


def mean_ci95(lengths):
    """Mean residence time and its 95 % confidence half-width 1.96 s / sqrt(m) (s: sample
    standard deviation of the m residence times)."""
    x = np.asarray(lengths, dtype=np.float64)
    m = x.size
    if m == 0:
        return float("nan"), float("nan")
    s = x.std(ddof=1) if m > 1 else 0.0
    return float(x.mean()), float(1.96 * s / np.sqrt(m))
