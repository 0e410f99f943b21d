"""Pins for the oracle's Clebsch-Gordan coefficients and Wigner U^j (the building blocks
of the SNAP bispectrum, cited method of Thompson et al. 2015, Sec. 3.1)."""
import itertools

import numpy as np
import pytest

import oracle as O

sympy = pytest.importorskip("sympy")
from sympy.physics.quantum.cg import CG  # noqa: E402


def _sym_cg(tj1, tm1, tj2, tm2, tJ, tM):
    h = sympy.S(1) / 2
    return float(CG(tj1 * h, tm1 * h, tj2 * h, tm2 * h, tJ * h, tM * h).doit())


def test_cg_matches_sympy_small():
    for tj1, tj2 in itertools.product(range(5), range(5)):
        for tJ in range(abs(tj1 - tj2), tj1 + tj2 + 1, 2):
            for tm1 in range(-tj1, tj1 + 1, 2):
                for tm2 in range(-tj2, tj2 + 1, 2):
                    if abs(tm1 + tm2) > tJ:
                        continue
                    assert O.cg(tj1, tm1, tj2, tm2, tJ, tm1 + tm2) == pytest.approx(
                        _sym_cg(tj1, tm1, tj2, tm2, tJ, tm1 + tm2), abs=1e-13)


def test_cg_matches_sympy_sampled_2J8():
    rng = np.random.default_rng(0)
    done = 0
    while done < 150:
        tj1, tj2 = rng.integers(0, 9, size=2)
        tJ = rng.integers(0, 9)
        if not (abs(tj1 - tj2) <= tJ <= tj1 + tj2 and (tj1 + tj2 + tJ) % 2 == 0):
            continue
        tm1 = rng.integers(0, tj1 + 1) * 2 - tj1
        tm2 = rng.integers(0, tj2 + 1) * 2 - tj2
        if abs(tm1 + tm2) > tJ:
            continue
        assert O.cg(tj1, tm1, tj2, tm2, tJ, tm1 + tm2) == pytest.approx(
            _sym_cg(tj1, tm1, tj2, tm2, tJ, tm1 + tm2), abs=1e-12)
        done += 1


def test_cg_orthogonality_2J8():
    for tj1, tj2 in itertools.product(range(9), range(9)):
        Js = [tJ for tJ in range(abs(tj1 - tj2), tj1 + tj2 + 1, 2)]
        for tM in range(-(tj1 + tj2), tj1 + tj2 + 1, 2):
            rows = [(tm1, tM - tm1) for tm1 in range(-tj1, tj1 + 1, 2) if abs(tM - tm1) <= tj2]
            cols = [tJ for tJ in Js if abs(tM) <= tJ]
            C = np.array([[O.cg(tj1, m1, tj2, m2, tJ, tM) for tJ in cols] for m1, m2 in rows])
            assert C.shape[0] == C.shape[1]
            assert np.allclose(C.T @ C, np.eye(len(cols)), atol=1e-12)


def _rand_su2(rng):
    v = rng.normal(size=4)
    v /= np.linalg.norm(v)
    return complex(v[0], v[1]), complex(v[2], v[3])


def _g(a, b):
    return np.array([[a, b], [-np.conj(b), np.conj(a)]])


def _sym_power(M, tj):
    """Independent construction of the spin-j matrix: the restriction of M^{(x)2j} to the
    symmetric subspace, in the normalised basis |j m> (m = -j..j) built from basis vector
    0 = (m=-1/2) and 1 = (m=+1/2)."""
    n = tj + 1
    dim = 2 ** tj
    V = np.zeros((dim, n))
    for idx in range(dim):
        ups = bin(idx).count("1")
        V[idx, ups] = 1.0
    V /= np.linalg.norm(V, axis=0)
    K = np.array([[1.0 + 0j]])
    for _ in range(tj):
        K = np.kron(K, M)
    return V.T @ K @ V


def test_wigner_half_is_g_and_group_properties():
    rng = np.random.default_rng(1)
    a, b = _rand_su2(rng)
    U = O.wigner_u(1, a, b)
    # rows/cols ordered m = -1/2, +1/2 : reversing both gives g itself
    assert np.allclose(U[::-1, ::-1], _g(a, b), atol=1e-15)
    a2, b2 = _rand_su2(rng)
    g12 = _g(a, b) @ _g(a2, b2)
    for tj in range(9):
        U1, U2 = O.wigner_u(tj, a, b), O.wigner_u(tj, a2, b2)
        assert np.allclose(U1 @ U2, O.wigner_u(tj, g12[0, 0], g12[0, 1]), atol=1e-13)   # homomorphism
        assert np.allclose(U1.conj().T @ U1, np.eye(tj + 1), atol=1e-13)                 # unitary
        assert np.allclose(O.wigner_u(tj, 1.0, 0.0), np.eye(tj + 1), atol=0)             # U(I) = I


def test_wigner_equals_symmetric_tensor_power():
    rng = np.random.default_rng(2)
    a, b = _rand_su2(rng)
    Uhalf = O.wigner_u(1, a, b)
    for tj in range(1, 7):
        assert np.allclose(O.wigner_u(tj, a, b), _sym_power(Uhalf, tj), atol=1e-13)


def test_clebsch_gordan_series_couples_U():
    """U^{j1}_{m1m1'} U^{j2}_{m2m2'} = sum_J C^{J,m1+m2}_{j1m1j2m2} C^{J,m1'+m2'}_{j1m1'j2m2'} U^J."""
    rng = np.random.default_rng(3)
    a, b = _rand_su2(rng)
    for tj1, tj2 in [(1, 1), (2, 1), (3, 2), (4, 4), (8, 3)]:
        U1, U2 = O.wigner_u(tj1, a, b), O.wigner_u(tj2, a, b)
        UJ = {tJ: O.wigner_u(tJ, a, b) for tJ in range(abs(tj1 - tj2), tj1 + tj2 + 1, 2)}
        for p1, q1, p2, q2 in itertools.product(range(tj1 + 1), range(tj1 + 1), range(tj2 + 1), range(tj2 + 1)):
            tm1, tm1p, tm2, tm2p = 2 * p1 - tj1, 2 * q1 - tj1, 2 * p2 - tj2, 2 * q2 - tj2
            rhs = 0
            for tJ, U in UJ.items():
                tM, tMp = tm1 + tm2, tm1p + tm2p
                if abs(tM) > tJ or abs(tMp) > tJ:
                    continue
                rhs += O.cg(tj1, tm1, tj2, tm2, tJ, tM) * O.cg(tj1, tm1p, tj2, tm2p, tJ, tMp) * \
                    U[(tM + tJ) // 2, (tMp + tJ) // 2]
            assert abs(U1[p1, q1] * U2[p2, q2] - rhs) < 1e-13
