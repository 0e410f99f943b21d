"""Pins for the oracle's Langevin schemes: eqs. (2)-(3), the corrected eqs. (11)-(12) with the
schedules (13)-(14), the closed forms of App. A.1 (V = 0) and App. A.2, and gamma = 0 physics."""
import numpy as np
import pytest

import oracle as O
import workloads as W

KB, FTOA = W.KB, W.FTOA


def _run(q, v, L, n, lp, pot=None, box=np.full(3, 1000.0)):
    pot = pot or O.potential(O.POT_ZERO)
    q = np.ascontiguousarray(q[None].copy())
    v = np.ascontiguousarray(v[None].copy())
    O.propagate(pot, q, v, box, [L], [n], lp)
    return q[0], v[0]


@pytest.mark.parametrize("schedule", [O.SCHED_NONE, O.SCHED_ROBUST])
def test_zero_force_closed_form(schedule):
    """App. A.1 (closed form of p_l) and its corrected form in App. A.2: with V = 0, for one noise
    realisation, p_L = mu^2 (1-g dt)^(L-1) p_0 + 2 mu sum_{i=1}^{L-1} (1-g dt)^(i-1) sqrt(th_{L-i}) G_{L-i}
                     + mu sqrt(th_0) (1-g dt)^(L-1) G_0 + sqrt(th_L) G_L,
    and q_L = q_0 + dt sum_l p_{l+1/2} with p_{l+1/2} = (1-g dt)^l p_{1/2} + 2 sum ... ."""
    rng = np.random.default_rng(0)
    m, L, n, seed = 7, 6, 11, 99
    lp = O.langevin(dt=2e-3, gamma=5.0, T=1500.0, seed=seed, schedule=schedule)
    q0 = rng.normal(size=(3, m))
    v0 = rng.normal(size=(3, m))
    qL, vL = _run(q0, v0, L, n, lp)
    kT_m = KB * lp.T / lp.mass * FTOA
    C = [(3.0 if l == 0 else 1.0) if schedule == O.SCHED_ROBUST else 1.0 for l in range(L + 1)]
    th = [0.5 * lp.gamma * kT_m * c * lp.dt for c in C]
    mu = 1 - 0.5 * lp.gamma * lp.dt
    r = 1 - lp.gamma * lp.dt
    G = np.array([[O.normals3(seed, n, l, i) for i in range(m)] for l in range(L + 1)])  # [l, i, axis]
    G = G.transpose(0, 2, 1)                                                            # [l, axis, i]
    pL = mu ** 2 * r ** (L - 1) * v0 + mu * np.sqrt(th[0]) * r ** (L - 1) * G[0] + np.sqrt(th[L]) * G[L]
    for i in range(1, L):
        pL = pL + 2 * mu * r ** (i - 1) * np.sqrt(th[L - i]) * G[L - i]
    assert np.allclose(vL, pL, rtol=1e-12, atol=1e-12)
    ph = mu * v0 + np.sqrt(th[0]) * G[0]                  # p_{1/2}
    qs = q0 + lp.dt * ph
    for l in range(1, L):
        ph = r * ph + 2 * np.sqrt(th[l]) * G[l]           # p_{l+1/2} = (1-g dt) p_{l-1/2} + 2 sqrt(th_l) G_l
        qs = qs + lp.dt * ph
    assert np.allclose(qL, qs, rtol=1e-12, atol=1e-12)


def _exact_stationary_var(L, dt, gamma, kT_m, C):
    """Fixed point of the finite-dt variance recursion of App. A.1 (uncorrected) / App. A.2."""
    mu = 1 - 0.5 * gamma * dt
    r = 1 - gamma * dt
    th = [0.5 * gamma * kT_m * c * dt for c in C]
    A = mu ** 4 * r ** (2 * (L - 1))
    B = mu ** 2 * th[0] * r ** (2 * (L - 1)) + th[L]
    for i in range(1, L):
        B += 4 * mu ** 2 * r ** (2 * (i - 1)) * th[L - i]
    return B / (1 - A)


@pytest.mark.parametrize("L,schedule,target", [(1, O.SCHED_NONE, 0.5), (1, O.SCHED_ROBUST, 1.0),
                                              (1, O.SCHED_L1_SYM, 1.0), (4, O.SCHED_NONE, 1 - 1 / 8),
                                              (4, O.SCHED_ROBUST, 1.0)])
def test_kinetic_temperature_fixed_point(L, schedule, target):
    """Sec. 2.4 / App. A: starting at the exact stationary variance, one interval of L
    steps keeps it (empirical, 4 sigma); the stationary value is K_eq = kT/m (1 - 1/(2L)) + O(dt)
    uncorrected and kT/m with the schedules of eqs. (13)-(14) (Tables 5-6)."""
    m = 40000
    lp = O.langevin(dt=1e-3, gamma=2.0, T=1000.0, seed=7, schedule=schedule)
    kT_m = KB * lp.T / lp.mass * FTOA
    if schedule == O.SCHED_ROBUST:
        C = [3.0] + [1.0] * L
    elif schedule == O.SCHED_L1_SYM:
        C = [2.0, 2.0]
    else:
        C = [1.0] * (L + 1)
    K = _exact_stationary_var(L, lp.dt, lp.gamma, kT_m, C)
    assert K / kT_m == pytest.approx(target, abs=3 * lp.gamma * lp.dt)      # leading order, eq. (10)
    rng = np.random.default_rng(1)
    v0 = rng.normal(0, np.sqrt(K), size=(3, m))
    _, vL = _run(np.zeros((3, m)), v0, L, 5, lp)
    var = np.mean(vL ** 2)
    assert abs(var - K) < 4 * K * np.sqrt(2 / vL.size)


def test_uncorrected_L1_underheats():
    """Table 5 (first row): with L = 1 and no schedule the kinetic temperature settles near
    beta^-1 / 2; iterate many intervals from rest to reach the fixed point."""
    m = 4000
    lp = O.langevin(dt=2e-3, gamma=20.0, T=600.0, seed=3, schedule=O.SCHED_NONE)
    kT_m = KB * lp.T / lp.mass * FTOA
    q, v = np.zeros((3, m)), np.zeros((3, m))
    for n in range(400):                         # gamma * t = 16
        q, v = _run(q, v, 1, n, lp)
    K = _exact_stationary_var(1, lp.dt, lp.gamma, kT_m, [1.0, 1.0])
    assert abs(np.mean(v ** 2) - K) < 4 * K * np.sqrt(2 / v.size)
    assert 0.45 < np.mean(v ** 2) / kT_m < 0.55


def _fs_system(ncell=3, seed=0, sigma=0.05, T=600.0, sia=True):
    pos, box = W.bcc_sia(ncell) if sia else W.bcc(ncell)
    rng = np.random.default_rng(seed)
    q = np.ascontiguousarray(pos + rng.normal(0, sigma, pos.shape))
    v = W.velocities(pos.shape[1], T, rng)
    return q, v, box


def _total_energy(q, v, box, mass=W.M_W):
    E, _ = O.fs_energy_forces(q, box)
    return E[0] + 0.5 * mass * np.sum(v ** 2) / FTOA


def test_gamma_zero_is_velocity_verlet():
    """gamma = 0 removes damping and noise: the scheme is velocity Verlet -- time
    reversible, energy error O(dt^2) with no drift; BAOAB reduces to the same map."""
    q0, v0, box = _fs_system()
    pot = O.potential(O.POT_FS)
    lp = O.langevin(dt=1e-3, gamma=0.0, T=1000.0, schedule=O.SCHED_NONE)
    q1, v1 = _run(q0, v0, 200, 0, lp, pot, box)
    qb, vb = _run(q1, -v1, 200, 0, lp, pot, box)
    assert np.abs(qb - q0).max() < 1e-10 and np.abs(vb + v0).max() < 1e-9
    lpb = O.langevin(dt=1e-3, gamma=0.0, T=1000.0, scheme=O.SCHEME_BAOAB)
    q2, v2 = _run(q0, v0, 200, 0, lpb, pot, box)
    assert np.abs(q2 - q1).max() < 1e-11 and np.abs(v2 - v1).max() < 1e-9
    # energy-error order on a cold perfect crystal: the FS pair cutoff c = 3.25 sits 0.085
    # Angstrom above the second shell, and a kink in the force there spoils the dt^2 scaling
    # once atoms cross it, so no pair may cross a cutoff in this check
    q0, v0, box = _fs_system(sigma=0.005, T=30.0, sia=False)
    devs = []
    for dt in (2e-3, 1e-3):
        lp = O.langevin(dt=dt, gamma=0.0, T=1000.0, schedule=O.SCHED_NONE)
        E0 = _total_energy(q0, v0, box)
        q, v, es = q0, v0, []
        for n in range(int(round(0.1 / dt / 10))):
            q, v = _run(q, v, 10, n, lp, pot, box)
            es.append(_total_energy(q, v, box) - E0)
        devs.append(np.max(np.abs(es)))
    assert 3.0 < devs[0] / devs[1] < 5.0                  # second order
    assert devs[1] < 1e-4


def test_baoab_zero_force_is_exact_ou():
    m = 40000
    lp = O.langevin(dt=5e-3, gamma=3.0, T=800.0, scheme=O.SCHEME_BAOAB, seed=5)
    kT_m = KB * lp.T / lp.mass * FTOA
    rng = np.random.default_rng(2)
    v0 = rng.normal(0, np.sqrt(kT_m), size=(3, m))
    _, v = _run(np.zeros((3, m)), v0, 3, 0, lp)
    assert abs(np.mean(v ** 2) - kT_m) < 4 * kT_m * np.sqrt(2 / v.size)
    c1 = np.exp(-lp.gamma * lp.dt)
    assert np.corrcoef(v0.ravel(), v.ravel())[0, 1] == pytest.approx(c1 ** 3, abs=0.02)


def test_l1_sym_rejects_longer_intervals():
    lp = O.langevin(schedule=O.SCHED_L1_SYM)
    with pytest.raises(ValueError):
        _run(np.zeros((3, 2)), np.zeros((3, 2)), 2, 0, lp)
