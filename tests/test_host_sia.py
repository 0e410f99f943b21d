"""Host-side parts of the interstitial tracking on the CPU: the C library's residence runs
(sia_residence) against the oracle's on random well sequences, and the binding's argument checks
(they run before anything touches a device)."""
import numpy as np
import pytest

import oracle.sia as OS
import paper_2212_10508_gb300 as P
import workloads as W


@pytest.mark.parametrize("seed", range(5))
def test_residence_runs_match_the_oracle(seed):
    g = W.rng(80, seed)
    n = int(g.integers(1, 3000))
    # runs of random lengths over a few sites, neighbouring runs on different sites
    w, site = [], int(g.integers(8))
    while len(w) < n:
        w += [site] * int(g.geometric(0.05))
        site = (site + int(g.integers(1, 8))) % 8
    w = np.array(w[:n], np.int32)
    L, S = P.sia_residence(w)
    oL, oS = OS.residence(w)
    assert np.array_equal(L, oL) and np.array_equal(S, oS)
    assert n - L.sum() >= 1 and (L.size == 0 or L.min() >= 1)   # the open last run is left out


def test_binding_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    sites, box = W.bcc(2)
    q = torch.as_tensor(sites)
    with pytest.raises(ValueError):
        P.sia_locate(q[None], q, q, box)


def test_batch_means_interval():
    """Batch means of residence times: every run is assigned to the block where it ends; with
    identical blocks the interval collapses to zero, and with two regimes of different mean (a
    slow switch) it is much wider than the per-exit interval, which ignores the correlation."""
    from paper_2212_10508_gb300.residence import batch_means, mean_ci95
    import numpy as np
    L = [5, 5, 10] * 40                      # 120 runs, 800 frames, the same pattern everywhere
    m, h, blocks = batch_means(L, 801, blocks=4)   # 800 frames of runs + the open last one
    assert len(blocks) == 4 and h == 0.0 and m == np.mean(blocks)
    rng = np.random.default_rng(1)
    slow = list(rng.exponential(200, 60).astype(int) + 1)
    fast = list(rng.exponential(50, 240).astype(int) + 1)
    L2 = slow + fast
    m2, h2, _ = batch_means(L2, int(np.sum(L2)) + 1, blocks=10)
    _, hp = mean_ci95(L2)
    assert h2 > 2 * hp
