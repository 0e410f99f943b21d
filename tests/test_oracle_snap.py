"""Pins for the oracle's SNAP (fine potential V_F, Sec. 3.1; method cited from Thompson
et al. 2015): component counts (Table 1 names), closed forms from SU(2) character theory,
an independent brute-force bispectrum, invariances, and forces = -grad E."""
import itertools

import numpy as np
import pytest

import oracle as O
import workloads as W

RCUT, RFAC0 = 4.73, 0.99363


def test_component_counts_match_snap_names():
    # SNAP-6, -15, -31, -56, -92, -141, -205 (Table 1): 1 + number of bispectrum triples
    for tj, name in [(2, 6), (4, 15), (6, 31), (8, 56), (10, 92), (12, 141), (14, 205)]:
        assert 1 + len(O.snap_triples(tj)) == name


def _cluster(rng, nnb, rmin=2.3, rmax=4.6):
    """atom 0 at the centre of a large box with nnb neighbours inside rcut (far from others)."""
    L = 60.0
    c = np.full(3, L / 2)
    pts = [c]
    while len(pts) < nnb + 1:
        v = rng.normal(size=3)
        v *= rng.uniform(rmin, rmax) / np.linalg.norm(v)
        p = c + v
        if all(np.linalg.norm(p - q) > 1.6 for q in pts):
            pts.append(p)
    return np.ascontiguousarray(np.array(pts).T), np.full(3, L)


def _quat(rv):
    r = np.linalg.norm(rv)
    th = RFAC0 * np.pi * r / RCUT
    return np.concatenate([[np.cos(th)], np.sin(th) * rv / r])


def test_B_j0j_equals_character_sum():
    """B_{j,0,j} = u0 * sum_{k,l} w_k w_l chi_j(alpha_kl), chi_j = sin((2j+1)a)/sin(a),
    cos(alpha_kl) = u_k . u_l (unit quaternions; self term u = (1,0,0,0), w = 1)."""
    rng = np.random.default_rng(7)
    pos, box = _cluster(rng, 9)
    tri = O.snap_triples(8)
    nt = len(tri)
    beta = np.zeros(1 + nt)
    _, _, _, Bat = O.snap_energy_forces(pos, box, beta, want_B=True)
    us, ws = [np.array([1.0, 0, 0, 0])], [1.0]
    for k in range(1, pos.shape[1]):
        rv = pos[:, k] - pos[:, 0]
        r = np.linalg.norm(rv)
        if r < RCUT:
            us.append(_quat(rv))
            ws.append(0.5 * (np.cos(np.pi * r / RCUT) + 1))
    u0 = sum(ws)
    for t, (tj1, tj2, tj) in enumerate(tri):
        if tj2 != 0:
            continue
        s = 0.0
        for (uk, wk), (ul, wl) in itertools.product(zip(us, ws), zip(us, ws)):
            c = np.clip(np.dot(uk, ul), -1.0, 1.0)
            al = np.arccos(c)
            chi = (tj + 1.0) if abs(np.sin(al)) < 1e-7 else np.sin((tj + 1) * al) / np.sin(al)
            s += wk * wl * chi
        assert Bat[0, 0, t] == pytest.approx(u0 * s, rel=1e-11, abs=1e-10)


def test_perfect_lattice_values():
    pos, box = W.bcc(4)
    nt = len(O.snap_triples(8))
    beta = np.zeros(1 + nt)
    beta[1:] = np.random.default_rng(0).normal(0, 0.01, nt)
    _, F, _, Bat = O.snap_energy_forces(pos, box, beta, want_B=True)
    assert np.abs(F).max() < 1e-12                         # symmetric sites: no force
    assert np.allclose(Bat[0], Bat[0][0], rtol=1e-12)       # all sites equivalent
    r1, r2, r3 = W.A_W * np.sqrt(3) / 2, W.A_W, W.A_W * np.sqrt(2)
    fc = lambda r: 0.5 * (np.cos(np.pi * r / RCUT) + 1)
    u0 = 1 + 8 * fc(r1) + 6 * fc(r2) + 12 * fc(r3)          # 26 neighbours inside 4.73
    assert Bat[0, 0, 0] == pytest.approx(u0 ** 3, rel=1e-12)  # B_000 = u0^3


def _sym_power(M, tj):
    n = tj + 1
    dim = 2 ** tj
    V = np.zeros((dim, n))
    for idx in range(dim):
        V[idx, bin(idx).count("1")] = 1.0
    V /= np.linalg.norm(V, axis=0)
    K = np.array([[1.0 + 0j]])
    for _ in range(tj):
        K = np.kron(K, M)
    return V.T @ K @ V


def test_bispectrum_brute_force_2J4():
    """Tiny brute force: U^j as the symmetric tensor power of the 2x2 SU(2) matrix,
    Clebsch-Gordan from sympy, the triple sum written out -- compared with the oracle."""
    sympy = pytest.importorskip("sympy")
    from sympy.physics.quantum.cg import CG
    h = sympy.S(1) / 2
    cg = lambda a, b, c, d, e, f: float(CG(a * h, b * h, c * h, d * h, e * h, f * h).doit())
    rng = np.random.default_rng(11)
    pos, box = _cluster(rng, 3)
    p = O.snap_params(twojmax=4)
    tri = O.snap_triples(4)
    _, _, _, Bat = O.snap_energy_forces(pos, box, np.zeros(1 + len(tri)), params=p, want_B=True)
    Ut = {tj: np.eye(tj + 1, dtype=complex) for tj in range(5)}
    for k in range(1, pos.shape[1]):
        rv = pos[:, k] - pos[:, 0]
        r = np.linalg.norm(rv)
        th = RFAC0 * np.pi * r / RCUT
        a = np.cos(th) - 1j * np.sin(th) * rv[2] / r
        b = np.sin(th) * (rv[1] - 1j * rv[0]) / r
        g = np.array([[a, b], [-np.conj(b), np.conj(a)]])
        Uh = g[::-1, ::-1]                      # basis order m = -1/2, +1/2
        for tj in range(5):
            Ut[tj] += 0.5 * (np.cos(np.pi * r / RCUT) + 1) * _sym_power(Uh, tj)
    for t, (tj1, tj2, tj) in enumerate(tri):
        B = 0
        for p_, q_ in itertools.product(range(tj + 1), repeat=2):
            tm, tmp = 2 * p_ - tj, 2 * q_ - tj
            for tm1, tm1p in itertools.product(range(-tj1, tj1 + 1, 2), repeat=2):
                tm2, tm2p = tm - tm1, tmp - tm1p
                if abs(tm2) > tj2 or abs(tm2p) > tj2:
                    continue
                B += np.conj(Ut[tj][p_, q_]) * cg(tj1, tm1, tj2, tm2, tj, tm) * cg(tj1, tm1p, tj2, tm2p, tj, tmp) * \
                    Ut[tj1][(tm1 + tj1) // 2, (tm1p + tj1) // 2] * Ut[tj2][(tm2 + tj2) // 2, (tm2p + tj2) // 2]
        assert abs(B.imag) < 1e-10 * max(1, abs(B.real))        # the bispectrum is real
        assert Bat[0, 0, t] == pytest.approx(B.real, rel=1e-11, abs=1e-11)


def _random_rotation(rng):
    Q, R = np.linalg.qr(rng.normal(size=(3, 3)))
    Q *= np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    return Q


def test_bispectrum_invariances():
    rng = np.random.default_rng(3)
    pos, box = _cluster(rng, 12)
    tri = O.snap_triples(8)
    beta = np.zeros(1 + len(tri))
    _, _, _, B0 = O.snap_energy_forces(pos, box, beta, want_B=True)
    c = pos[:, :1]
    R = _random_rotation(rng)
    rot = np.ascontiguousarray(R @ (pos - c) + c)
    _, _, _, B1 = O.snap_energy_forces(rot, box, beta, want_B=True)
    perm = np.concatenate([[0], 1 + rng.permutation(pos.shape[1] - 1)])
    _, _, _, B2 = O.snap_energy_forces(np.ascontiguousarray(pos[:, perm]), box, beta, want_B=True)
    tr = np.ascontiguousarray(pos + rng.uniform(-3, 3, size=(3, 1)))
    _, _, _, B3 = O.snap_energy_forces(tr, box, beta, want_B=True)
    scale = np.abs(B0[0, 0]).max()
    for B in (B1, B3):
        assert np.abs(B[0, 0] - B0[0, 0]).max() < 1e-12 * scale
    assert np.abs(B2[0, 0] - B0[0, 0]).max() < 1e-12 * scale


def test_forces_are_minus_gradient():
    P, box, beta = W.small_system(nconf=2)
    E, F, sB = O.snap_energy_forces(P[:1], box, beta)
    assert np.abs(F[0].sum(axis=1)).max() < 1e-11                # momentum conservation
    assert E[0] == pytest.approx(float(beta @ sB[0]), rel=1e-13)  # E = sum_t beta_t sum_i B_t
    h = 1e-5
    rng = np.random.default_rng(0)
    for _ in range(6):
        al, i = int(rng.integers(3)), int(rng.integers(P.shape[2]))
        qp, qm = P[:1].copy(), P[:1].copy()
        qp[0, al, i] += h
        qm[0, al, i] -= h
        fd = -(O.snap_energy_forces(qp, box, beta)[0][0] - O.snap_energy_forces(qm, box, beta)[0][0]) / (2 * h)
        assert F[0, al, i] == pytest.approx(fd, rel=1e-6, abs=1e-7)
