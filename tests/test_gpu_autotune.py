"""Run-time shape of the batched FP32 fine kernel: results do not depend on it (bitwise), the
autotuner returns a valid shape and leaves its inputs untouched, bad shapes are rejected."""
import pytest
import torch

import workloads as W
from gpu_util import dev

pytestmark = pytest.mark.gpu


def _batch(nb, lo, hi, seed=11):
    import paper_2212_10508_gb300 as P
    q, v, box, beta, L, ids = W.batch_workload(master=seed, nbatch=nb, T=1500.0, lo=lo, hi=hi)
    d = dev()
    eng = P.Engine(q.shape[2], box, P.snap_params(precision=P.FP32_BULK), P.fs_params(),
                   beta=torch.as_tensor(beta, device=d))
    lp = P.langevin(dt=1e-3, gamma=1.0, T=1500.0, seed=5)
    t = lambda x: torch.as_tensor(x, device=d)
    return P, eng, t(q), t(v), t(L), t(ids), lp


@pytest.mark.parametrize("nb", [3, 20, 64])
def test_results_do_not_depend_on_shape(nb):
    # 3 members: few atoms per CTA (4-row warps), 20: 2-row warps, 64: full batches and the tail
    P, eng, q, v, L, ids, lp = _batch(nb, 5, 30)
    ref = None
    shapes = [dict(rows2_atoms=16, rows4_atoms=8, b_group=8, noise_stage=-1, warps=16),
              dict(rows2_atoms=0, rows4_atoms=0, b_group=4, noise_stage=2, warps=16),
              dict(rows2_atoms=16, rows4_atoms=0, b_group=10, noise_stage=5, warps=8),
              dict(rows2_atoms=8, rows4_atoms=4, b_group=1, noise_stage=0, warps=8)]
    for sh in shapes:
        eng.set_tuning(**sh)
        qq, vv = q.clone(), v.clone()
        eng.baoab_propagate_batch(P.FINE, qq, vv, L, ids, lp)
        eng.sync_status()
        if ref is None:
            ref = (qq, vv)
        else:
            assert torch.equal(qq, ref[0]) and torch.equal(vv, ref[1]), sh


def test_autotune_returns_valid_shape_and_keeps_inputs():
    P, eng, q, v, L, ids, lp = _batch(16, 20, 200)
    q0, v0, L0 = q.clone(), v.clone(), L.clone()
    shape, ms = eng.autotune(q, v, L, ids, lp, max_steps=16)
    assert torch.equal(q, q0) and torch.equal(v, v0) and torch.equal(L, L0)
    assert ms > 0
    assert 0 <= shape["rows2_atoms"] <= 16 and 0 <= shape["rows4_atoms"] <= 8
    assert 1 <= shape["b_group"] <= 10 and -1 <= shape["noise_stage"] <= 15 and shape["warps"] in (8, 16)
    assert eng.tuning() == shape


def test_bad_shapes_rejected():
    P, eng, *_ = _batch(2, 5, 6)
    for bad in (dict(rows2_atoms=17), dict(rows4_atoms=9), dict(b_group=0), dict(b_group=11), dict(noise_stage=-2),
                dict(warps=12)):
        with pytest.raises(P.PmdError):
            eng.set_tuning(**bad)
