"""Classical and adaptive parareal, written in the order and notation of the paper.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``classical``  -- Algorithm 1 (Sec. 2.1) with the error of eq. (6).
* ``adaptive``   -- Algorithm 2 (Sec. 2.2) with the time-slab error E(q^{k-1}, q^k, N_init, N_final).
* ``cost_and_gains`` -- eqs. (7)-(9): Cost, Gamma_adapt = N C_f / Cost, Gamma_ideal = N / sum_i k^i.

A state is a pair ``(q, p)`` of numpy arrays (positions and velocities).  The propagators
are batch callables ``F(states, ns) -> states`` and ``C(states, ns) -> states`` where
``ns`` are the interval indices n (interval [n dt, (n+1) dt], noise key n).  Nothing is
cached: ``C(prev_n)`` is recomputed where Algorithm 2 asks for it.

Readings of the paper used here:
  * |.| is the Euclidean norm of the 3m-vector of (unwrapped) positions;
  * metric "maxdisp" (for thresholds in Angstrom) replaces the relative error by the
    largest per-atom displacement |q_i^k - q_i^{k-1}| over the sub-window;
  * when the explosion test fires at n = N_init, Algorithm 2's assignment N_final := n
    would leave an empty slab and loop forever; N_final is clamped to N_init + 1.
"""
import numpy as np


def _norm(q):
    return float(np.sqrt(np.sum(np.asarray(q, dtype=np.float64) ** 2)))


def _per_atom_disp_max(qa, qb):
    d = np.asarray(qa, dtype=np.float64) - np.asarray(qb, dtype=np.float64)
    if d.ndim == 2:          # [3, m]
        return float(np.max(np.sqrt(np.sum(d * d, axis=0)))) if d.shape[1] else 0.0
    return float(np.max(np.abs(d))) if d.size else 0.0


def window_error(prev, cur, n_lo, n_hi, metric="rel"):
    """E(q^{k-1}, q^k, n_lo, n_hi) = sum_{n=n_lo}^{n_hi} |q^k_n - q^{k-1}_n| / sum |q^{k-1}_n|
    (Sec. 2.2; eq. (6) is the case n_lo = 1, n_hi = N), or the max-displacement metric."""
    if metric == "rel":
        num = sum(_norm(cur[n][0] - prev[n][0]) for n in range(n_lo, n_hi + 1))
        den = sum(_norm(prev[n][0]) for n in range(n_lo, n_hi + 1))
        return num / den
    if metric == "maxdisp":
        return max(_per_atom_disp_max(cur[n][0], prev[n][0]) for n in range(n_lo, n_hi + 1))
    raise ValueError(metric)


def _add(s, j):
    return (s[0] + j[0], s[1] + j[1])


def _sub(s, t):
    return (s[0] - t[0], s[1] - t[1])


def classical(q0, p0, N, delta_conv, F, C, metric="rel", max_iter=None):
    """Algorithm 1.  Returns (cur, k_conv, deltas) with cur[n] = (q^k_n, p^k_n)."""
    cur = [None] * (N + 1)
    cur[0] = (np.array(q0, dtype=np.float64), np.array(p0, dtype=np.float64))
    for n in range(N):                                   # coarse initialisation, eq. (4)
        cur[n + 1] = C([cur[n]], [n])[0]
    k = 0
    delta = 2 * delta_conv
    deltas = []
    while delta >= delta_conv:
        k += 1
        prev = list(cur)
        fine = F([prev[n] for n in range(N)], list(range(N)))      # "in parallel"
        coarse = C([prev[n] for n in range(N)], list(range(N)))
        J = [_sub(fine[n], coarse[n]) for n in range(N)]
        for n in range(N):                                          # eq. (5)
            cur[n + 1] = _add(C([cur[n]], [n])[0], J[n])
        delta = window_error(prev, cur, 1, N, metric)               # eq. (6)
        deltas.append(delta)
        if max_iter is not None and k >= max_iter:
            break
    return cur, k, deltas


class AdaptiveLog:
    """Window log: windows[i] = {"n_init": N_init^i, "subs": [[N_final^{i,j}, k^{i,j}], ...]}."""

    def __init__(self):
        self.windows = []

    @property
    def n_slab(self):
        return len(self.windows)

    def k_conv(self):
        return [sum(k for _, k in w["subs"]) for w in self.windows]


def adaptive(q0, p0, N, delta_conv, delta_expl, F, C, metric="rel", max_iter=10000, trace=None):
    """Algorithm 2.  Returns (cur, log) with cur a dict n -> (q, p) for 0 <= n <= N.

    ``trace`` (optional list) receives one tuple per parareal iteration:
    (N_init, N_final before the sweep, delta, n at which the sweep stopped (N_final if it
    completed), N_final after the sweep)."""
    N_init, N_final = 0, 0
    delta = (delta_conv + delta_expl) / 2
    cur = {0: (np.array(q0, dtype=np.float64), np.array(p0, dtype=np.float64))}
    log = AdaptiveLog()
    iters = 0
    while N_final < N:
        if delta < delta_expl:
            N_init = N_final                                      # new time-slab
            N_final = N
            for n in range(N_init, N_final):
                cur[n + 1] = C([cur[n]], [n])[0]
            log.windows.append({"n_init": N_init, "subs": []})
        delta = (delta_conv + delta_expl) / 2
        log.windows[-1]["subs"].append([N_final, 0])
        while delta_conv <= delta <= delta_expl:
            prev = {n: cur[n] for n in range(N_init, N_final + 1)}
            ns = list(range(N_init, N_final))
            fine = F([prev[n] for n in ns], ns)                   # "in parallel"
            coarse = C([prev[n] for n in ns], ns)
            J = {n: _sub(f, c) for n, f, c in zip(ns, fine, coarse)}
            log.windows[-1]["subs"][-1][1] += 1                    # k^{N_slab}_conv += 1
            n_fin_before = N_final
            n_stop = N_final
            for n in range(N_init, N_final):
                cur[n + 1] = _add(C([cur[n]], [n])[0], J[n])
                delta = window_error(prev, cur, N_init, n + 1, metric)
                if delta > delta_expl:
                    n_stop = n
                    N_final = max(n, N_init + 1)                   # N_final := n (clamped)
                    break
            if trace is not None:
                trace.append((N_init, n_fin_before, delta, n_stop, N_final))
            iters += 1
            if iters > max_iter:
                raise RuntimeError("adaptive parareal did not terminate")
    return cur, log


def cost_and_gains(log: AdaptiveLog, N, C_f, C_c):
    """eq. (7) Cost, eq. (8) Gamma_adapt = N C_f / Cost, eq. (9) Gamma_ideal = N / sum_i k^i_conv."""
    cost = 0.0
    for w in log.windows:
        n_init = w["n_init"]
        cost += (N - n_init) * C_c
        for n_fin_ij, k_ij in w["subs"]:
            cost += k_ij * ((C_f + C_c) + (n_fin_ij - n_init) * C_c)
    g_adapt = N * C_f / cost
    g_ideal = N / sum(log.k_conv())
    return cost, g_adapt, g_ideal


def classical_cost(N, k_conv, C_f, C_c):
    """Total cost of Algorithm 1 stated in Sec. 2.1: N C_c + k_conv ((C_f + C_c) + N C_c)."""
    return N * C_c + k_conv * ((C_f + C_c) + N * C_c)
