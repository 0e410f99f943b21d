"""Adaptive parareal (Algorithm 2, Sec. 2.2) with the fine batch of every iteration split across
the ranks of a torch.distributed process group (one GPU per rank).

Per parareal iteration on the slab [N_init, N_final):
  * every rank holds the slab's states cur and the coarse cache C(cur_n) (replicated);
  * rank r propagates its contiguous block of the slab's intervals with the fine propagator
    (the parallel part of the iteration, Sec. 2.1: F(prev_n) for every interval independently);
  * the blocks are all-gathered, so the sweeping rank (rank 0) has F(prev_n) for the whole slab;
  * rank 0 forms the jumps J_n = F(prev_n) - C(prev_n) and runs the sequential correction sweep
    (parareal_correct: cur_{n+1} = C(cur_n) + J_n, the slab error, the explosion test);
  * rank 0 broadcasts the corrected states, the new coarse cache and (delta, n_stop); every rank
    feeds them to its own copy of the Algorithm 2 state machine (adaptive_restart), so all ranks
    take the same decisions.
The only exchange is that of the sequential step: the fine states of each block go to the
sweeping rank and the corrected states come back.  Each interval's fine result does not depend
on which rank or batch computed it, so the states are bitwise those of a single-rank run.

The propagators come from an `ops` object: EngineOps wraps the library's engine (GPU, NCCL);
tests pass CPU propagators and run the ranks on gloo.
"""
import torch
import torch.distributed as dist

from . import ACT_ITERATE, FINE, Adaptive


class EngineOps:
    """The library's engine as the propagators of adaptive_parareal_dist (states [cnt, 6, n] on the
    engine's device; L sub-steps per interval; Langevin parameters lp; error metric)."""

    def __init__(self, engine, L, lp, metric, stream=None):
        self.engine, self.L, self.lp, self.metric, self.stream = engine, L, lp, metric, stream

    def fine(self, states, ids):
        nsteps = torch.full((states.shape[0],), self.L, dtype=torch.int32, device=states.device)
        self.engine.baoab_propagate_batch(FINE, states, None, nsteps, ids, self.lp, stream=self.stream)

    def sweep(self, a, b, jumps, prev, cur, cache, delta_expl):
        return self.engine.parareal_correct(a, b, jumps, prev, cur, cache, delta_expl, self.metric, self.L, self.lp,
                                            self.stream)

    def jumps(self, fine, cache):
        out = torch.empty_like(fine)
        self.engine.parareal_jumps(fine.shape[0], fine, cache, out, self.stream)
        return out


def block(a, b, rank, world):
    """Rank's contiguous share [lo, hi) of the intervals [a, b): sizes differ by at most one, the
    first (b - a) % world ranks take the larger share."""
    cnt = b - a
    base, extra = divmod(cnt, world)
    lo = a + rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def adaptive_parareal_dist(ops, q0, v0, N, delta_conv, delta_expl, group=None, max_iter=100000):
    """Algorithm 2 over the ranks of `group` (default: the world).  q0, v0 [3, n] on every rank.
    Returns (states [N+1, 6, n], Adaptive) on every rank."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    src = dist.get_global_rank(group, 0) if group is not None else 0
    n = q0.shape[-1]
    devc = q0.device
    cur = torch.empty(N + 1, 6, n, dtype=torch.float64, device=devc)
    cur[0, :3] = q0
    cur[0, 3:] = v0
    cache = torch.zeros(max(N, 1), 6, n, dtype=torch.float64, device=devc)
    ids_all = torch.arange(N, dtype=torch.int64, device=devc)
    st = Adaptive(N, delta_conv, delta_expl)
    act = st.adaptive_restart()
    scalars = torch.zeros(2, dtype=torch.float64, device=devc)
    iters = 0

    def share(a, b):   # rank 0's sweep results to every rank
        dist.broadcast(cur[a:b + 1], src, group=group)
        dist.broadcast(cache[a:b], src, group=group)
        dist.broadcast(scalars, src, group=group)

    while act.kind == ACT_ITERATE:
        a, b = act.n_in, act.n_fin
        cnt = b - a
        if act.open_slab:   # coarse initialisation of the slab: cur_{n+1} = C(cur_n)
            if rank == 0:
                ops.sweep(a, b, None, cur[a:b + 1], cur[a:b + 1], cache[a:b], float("inf"))
            share(a, b)
        prev = cur[a:b + 1].clone()
        lo, hi = block(a, b, rank, world)
        width = -(-cnt // world)
        mine = torch.zeros(width, 6, n, dtype=torch.float64, device=devc)
        if hi > lo:
            mine[:hi - lo] = prev[lo - a:hi - a]
            ops.fine(mine[:hi - lo], ids_all[lo:hi])
        parts = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine, group=group)
        if rank == 0:
            fine = torch.empty(cnt, 6, n, dtype=torch.float64, device=devc)
            for r in range(world):
                l2, h2 = block(a, b, r, world)
                fine[l2 - a:h2 - a] = parts[r][:h2 - l2]
            jumps = ops.jumps(fine, cache[a:b])
            delta, n_stop = ops.sweep(a, b, jumps, prev, cur[a:b + 1], cache[a:b], delta_expl)
            scalars[0], scalars[1] = float(delta), float(n_stop)
        share(a, b)
        act = st.adaptive_restart(float(scalars[0]), int(scalars[1]))
        iters += 1
        if iters > max_iter:
            raise RuntimeError("adaptive parareal did not terminate")
    return cur, st
