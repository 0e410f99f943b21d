"""CPU propagators for the multi-rank parareal tests (test infrastructure): Finnis-Sinclair fine
and a perturbed Finnis-Sinclair coarse from the oracle, and a correction sweep written from
Algorithm 2's inner loop (cur_{n+1} = C(cur_n) + J_n, the running slab error in the
max-displacement metric, stop at the first error above delta_expl)."""
import numpy as np
import torch

import oracle as O
from oracle import parareal as PR
import workloads as W


class OracleOps:
    def __init__(self, box, L, lp, fine, coarse):
        self.box, self.L, self.lp = box, L, lp
        self.F = self._prop(fine)
        self.C = self._prop(coarse)

    def _prop(self, pot):
        def prop(states, ns):
            q = np.ascontiguousarray(np.array([s[0] for s in states]))
            v = np.ascontiguousarray(np.array([s[1] for s in states]))
            O.propagate(pot, q, v, self.box, [self.L] * len(ns), list(ns), self.lp)
            return [(q[i], v[i]) for i in range(len(ns))]
        return prop

    def fine(self, states, ids):
        s = states.numpy()
        out = self.F([(s[i, :3], s[i, 3:]) for i in range(s.shape[0])], ids.tolist())
        for i, (q, v) in enumerate(out):
            states[i, :3] = torch.as_tensor(q)
            states[i, 3:] = torch.as_tensor(v)

    def jumps(self, fine, cache):
        return fine - cache

    def sweep(self, a, b, jumps, prev, cur, cache, delta_expl):
        pv = {a + k: (prev[k, :3].numpy(), prev[k, 3:].numpy()) for k in range(b - a + 1)}
        cu = {a: (cur[0, :3].numpy().copy(), cur[0, 3:].numpy().copy())}
        delta, n_stop = PR.window_error(pv, cu, a, a, "maxdisp"), b
        for nn in range(a, b):
            c = self.C([cu[nn]], [nn])[0]
            cache[nn - a, :3] = torch.as_tensor(c[0])
            cache[nn - a, 3:] = torch.as_tensor(c[1])
            if jumps is not None:
                j = jumps[nn - a].numpy()
                c = (c[0] + j[:3], c[1] + j[3:])
            cu[nn + 1] = c
            cur[nn + 1 - a, :3] = torch.as_tensor(c[0])
            cur[nn + 1 - a, 3:] = torch.as_tensor(c[1])
            delta = PR.window_error(pv, cu, a, nn + 1, "maxdisp")
            if not np.isfinite(delta):
                delta = float("inf")
            if not (delta <= delta_expl):
                n_stop = nn
                break
        return delta, n_stop


def setup():
    pos, box = W.bcc_sia(3)
    q0 = W.displaced(pos, 0.05, W.rng(81, 1))
    v0 = W.velocities(pos.shape[1], 1500.0, W.rng(81, 2))
    lp = O.langevin(dt=2e-3, gamma=1.0, T=1500.0, seed=13, schedule=O.SCHED_ROBUST)
    coarse = dict(W.FS_W)
    coarse["A"] *= 1.3
    ops = OracleOps(box, 2, lp, O.potential(O.POT_FS), O.potential(O.POT_FS, fs=O.fs_params(**coarse)))
    return q0, v0, ops, 11, 1e-9, 0.002
