"""Pins for the oracle's noise G_{l,n} (Sec. 2.1: independent standard Gaussians, the same
for F, C and every parareal iteration).

The Philox bit stream is not compared with published known-answer vectors (none are
available here: "parity unpinned" for the raw stream); what the paper fixes -- i.i.d.
N(0,1) increments keyed by interval n and sub-step l -- is pinned statistically.
"""
import numpy as np
import pytest
from scipy import stats

import oracle as O


def _draw(seed, ns, ells, atoms):
    return np.array([O.normals3(seed, n, l, a) for n in ns for l in ells for a in atoms])


def test_philox_bits_are_balanced_and_key_sensitive():
    outs = np.array([O.philox4x32_10([i, 0, 0, 0], [1, 2]) for i in range(4000)], dtype=np.uint64)
    bits = np.unpackbits(outs.astype(np.uint32).view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.005
    # flipping one key bit or one counter bit changes about half of the 128 output bits
    base = O.philox4x32_10([7, 8, 9, 10], [11, 12])
    flips = []
    for b in range(32):
        o1 = O.philox4x32_10([7 ^ (1 << b), 8, 9, 10], [11, 12])
        o2 = O.philox4x32_10([7, 8, 9, 10], [11 ^ (1 << b), 12])
        for o in (o1, o2):
            flips.append(np.unpackbits((o ^ base).view(np.uint8)).sum())
    assert 56 < np.mean(flips) < 72


def test_normals_are_standard_gaussian():
    g = _draw(42, range(10), range(5), range(200)).ravel()      # 30,000 values
    assert abs(g.mean()) < 4 / np.sqrt(g.size)
    assert abs(g.var() - 1) < 4 * np.sqrt(2 / g.size)
    assert abs(stats.skew(g)) < 0.1 and abs(stats.kurtosis(g)) < 0.2
    assert stats.kstest(g, "norm").pvalue > 1e-3


def test_normals_independent_across_keys():
    # correlation between streams that differ only in n, l, atom or axis is ~0
    a = _draw(5, [3], range(50), range(100))
    b = _draw(5, [4], range(50), range(100))
    c = _draw(5, [3], range(1, 51), range(100))
    d = _draw(6, [3], range(50), range(100))
    lim = 4 / np.sqrt(a.size)
    for other in (b, c, d):
        assert abs(np.corrcoef(a.ravel(), other.ravel())[0, 1]) < lim
    for i, j in ((0, 1), (0, 2), (1, 2)):
        assert abs(np.corrcoef(a[:, i], a[:, j])[0, 1]) < 4 / np.sqrt(a.shape[0])


def test_normals_reproducible():
    assert np.array_equal(O.normals3(1, 2, 3, 4), O.normals3(1, 2, 3, 4))
    assert not np.array_equal(O.normals3(1, 2, 3, 4), O.normals3(1, 2, 3, 5))
