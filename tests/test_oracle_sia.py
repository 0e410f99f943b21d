"""Pins of the interstitial-tracking oracle (Wigner-Seitz reading of the Voronoi analysis of
Sec. 3, residence times in units of the frame spacing): a periodic k-d tree query of a library
(scipy) for the nearest sites, the known well of a constructed dumbbell under translations and
box-vector images, hand-made well sequences, and the 95 % interval of a known sample."""
import numpy as np
import pytest

import oracle.sia as OS
import workloads as W


def test_nearest_sites_match_a_periodic_kdtree():
    spatial = pytest.importorskip("scipy.spatial")
    sites, box = W.bcc(4)
    g = W.rng(31, 1)
    q = g.uniform(-1.5, 2.5, size=(3, 500)) * box[:, None]       # outside the box too
    s = OS.nearest_sites(q, np.zeros(3), sites, box)
    tree = spatial.cKDTree(np.mod(sites.T, box), boxsize=box)
    _, ref = tree.query(np.mod(q.T, box))
    assert np.array_equal(s, ref)


@pytest.mark.parametrize("site", [0, 17, 64, 127])
def test_constructed_dumbbell_is_found_under_translation_and_images(site):
    sites, box = W.bcc(4)
    u = np.ones(3) / np.sqrt(3.0)
    q = np.concatenate([np.delete(sites, site, axis=1), (sites[:, site] + 1.1 * u)[:, None],
                        (sites[:, site] - 1.1 * u)[:, None]], axis=1)
    g = W.rng(32, site)
    frames = [q, q + np.array([[0.7], [-1.3], [2.2]]),                            # whole-cell translation
              q + g.normal(0.0, 0.05, size=q.shape)]
    well, occ = OS.locate(np.stack(frames), q, sites, box)
    assert np.all(well == site) and np.all(occ == 2)
    # unwrapped coordinates that carry box-vector offsets (in the frames and the reference alike)
    offs = box[:, None] * g.integers(-2, 3, size=q.shape)
    well, occ = OS.locate(np.stack(frames) + offs[None], q + offs, sites, box)
    assert np.all(well == site) and np.all(occ == 2)


def test_com_shift_is_the_mean_displacement():
    g = W.rng(33, 1)
    ref = g.normal(size=(3, 129))
    t = np.array([0.25, -3.0, 11.5])
    c = OS.com_shift(ref + t[:, None], ref)
    assert np.allclose(c, t, rtol=0, atol=1e-14)


def test_perfect_lattice_ties_go_to_the_smallest_site():
    sites, box = W.bcc(2)
    # every atom exactly on a site, and one extra atom exactly midway between sites 0 and 1
    mid = 0.5 * (sites[:, 0] + sites[:, 8])     # a corner site and its body-centre neighbour
    q = np.concatenate([sites, mid[:, None]], axis=1)
    s = OS.nearest_sites(q, np.zeros(3), sites, box)
    assert np.array_equal(s[:-1], np.arange(sites.shape[1]))
    d = np.sum((sites - mid[:, None]) ** 2, axis=0)
    assert s[-1] == int(np.flatnonzero(d == d.min())[0])


def test_synthetic_trajectory_wells():
    frames, sites, box, wells = W.sia_frames(4, 200, W.rng(34, 1), sigma=0.03, hop=0.1)
    well, occ = OS.locate(frames, frames[0], sites, box)
    assert np.array_equal(well, wells) and np.all(occ == 2)


def test_residence_runs():
    L, S = OS.residence(np.array([3, 3, 3, 5, 5, 3, 3, 7]))
    assert L.tolist() == [3, 2, 2] and S.tolist() == [3, 5, 3]
    for w in ([], [4], [4, 4, 4]):
        L, S = OS.residence(np.array(w, np.int32))
        assert L.size == 0 and S.size == 0
    L, _ = OS.residence(np.array([1, 2, 1, 2]))
    assert L.tolist() == [1, 1, 1]


def test_mean_ci95():
    m, h = OS.mean_ci95([1, 2, 3, 4])
    assert m == 2.5 and abs(h - 1.96 * np.sqrt(5.0 / 3.0) / 2.0) < 1e-15
