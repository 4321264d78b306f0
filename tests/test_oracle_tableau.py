"""Pins of the oracle's tableau and transform against the paper and closed forms."""
import json
import math
import os

import numpy as np
import pytest

from oracle import tableau as tab

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def pade_denominator_roots(s):
    """Roots of Q(z) = sum_j (-1)^j (2s-j)! s! / ((2s)! j! (s-j)!) z^j.

    The stability function of s-stage Gauss is the (s,s) Pade approximant
    P(z)/Q(z) of exp(z); the poles of R are 1/eig(A0), so eig(A0^{-1}) are
    the roots of Q (Hairer-Wanner, Sec. IV.3-IV.5).
    """
    coef = [(-1) ** j * math.factorial(2 * s - j) * math.factorial(s)
            / (math.factorial(2 * s) * math.factorial(j) * math.factorial(s - j))
            for j in range(s + 1)]
    return np.roots(coef[::-1])


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5])
def test_gauss_order_conditions(s):
    """B(2s), C(s), D(s) simplifying conditions of Gauss collocation."""
    A, b, c = tab.gauss(s)
    for k in range(1, 2 * s + 1):
        assert abs(b @ c ** (k - 1) - 1.0 / k) < 2e-14
    for k in range(1, s + 1):
        np.testing.assert_allclose(A @ c ** (k - 1), c ** k / k, atol=2e-14)
        np.testing.assert_allclose(b * c ** (k - 1) @ A, b * (1 - c ** k) / k, atol=2e-14)


def test_gauss2_closed_form():
    A, b, c = tab.gauss(2)
    r3 = math.sqrt(3.0)
    np.testing.assert_allclose(c, [0.5 - r3 / 6, 0.5 + r3 / 6], atol=1e-15)
    np.testing.assert_allclose(A, [[0.25, 0.25 - r3 / 6], [0.25 + r3 / 6, 0.25]], atol=1e-15)
    np.testing.assert_allclose(b, [0.5, 0.5], atol=1e-15)
    np.testing.assert_allclose(np.linalg.inv(A), [[3, 2 * r3 - 3], [-3 - 2 * r3, 3]], atol=1e-13)


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5])
def test_eigenvalues_are_pade_poles(s):
    A, _, _ = tab.gauss(s)
    Q0, R0, blocks = tab.real_schur(np.linalg.inv(A))
    ev = []
    for (k, m), bc in zip(blocks, tab.block_constants(R0, blocks)):
        if m == 1:
            ev.append(complex(bc["eta"], 0))
        else:
            ev += [complex(bc["eta"], bc["beta"]), complex(bc["eta"], -bc["beta"])]
    want = pade_denominator_roots(s)
    key = lambda z: (round(z.real, 6), round(z.imag, 6))  # noqa: E731
    np.testing.assert_allclose(sorted(ev, key=key), sorted(want, key=key), atol=1e-10)


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_schur_form_and_table1(s):
    """Q0 orthogonal, Q0 R0 Q0^T = A0^{-1}, standardized 2x2 blocks; Table 1."""
    A, _, _ = tab.gauss(s)
    Ainv = np.linalg.inv(A)
    Q0, R0, blocks = tab.real_schur(Ainv)
    np.testing.assert_allclose(Q0 @ Q0.T, np.eye(s), atol=1e-14)
    np.testing.assert_allclose(Q0 @ R0 @ Q0.T, Ainv, atol=1e-12)
    for (k, m) in blocks:
        assert np.all(np.abs(R0[k + m:, k:k + m]) < 1e-12)
        if m == 2:
            assert abs(R0[k, k] - R0[k + 1, k + 1]) < 1e-12
            assert R0[k, k + 1] * R0[k + 1, k] < 0
    bounds = sorted(math.ceil(100 * tab.kappa_bound(bc["eta"], bc["beta"]) - 1e-9) / 100
                    for bc in tab.block_constants(R0, blocks))
    assert bounds == sorted(GOLDEN["table1_gauss_kappa_bounds"][str(s)])


def test_gamma_star_values():
    want = {2: [4.0], 3: [4.6444, 7.0253], 4: [6.3118, 10.9211], 5: [7.2935, 8.5159, 15.6205]}
    for s, g in want.items():
        A, _, _ = tab.gauss(s)
        Q0, R0, blocks = tab.real_schur(np.linalg.inv(A))
        got = sorted(bc["gamma_star"] for bc in tab.block_constants(R0, blocks))
        np.testing.assert_allclose(got, g, atol=1e-4)


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_d_vector_sum_rule(s):
    """sum_i (d_{k,l})_i = delta_{kl} by orthogonality of Q0 (Sec. 3.2)."""
    A, _, _ = tab.gauss(s)
    Q0, _, _ = tab.real_schur(np.linalg.inv(A))
    d = tab.d_vectors(Q0)
    np.testing.assert_allclose(d.sum(axis=-1), np.eye(s), atol=1e-14)


def _pair_invariant(d):
    diag = sorted([tuple(np.round(d[0, 0], 3)), tuple(np.round(d[1, 1], 3))])
    off = np.round(np.abs(d[0, 1]), 3)
    return diag, tuple(off)


def test_gauss4_and_radau3_phat_example():
    """Eq. Gauss4Radau3_example, up to the non-unique ordering/sign of the Schur basis."""
    A, _, _ = tab.gauss(2)
    Q0, _, _ = tab.real_schur(np.linalg.inv(A))
    g = GOLDEN["gauss4_Phat"]
    want = np.array([[g["d11"], g["d12"]], [g["d21"], g["d22"]]])
    assert _pair_invariant(tab.d_vectors(Q0)) == _pair_invariant(want)
    Ar = np.array([[5 / 12, -1 / 12], [3 / 4, 1 / 4]])  # 2-stage Radau IIA
    Q0, R0, blocks = tab.real_schur(np.linalg.inv(Ar))
    r = GOLDEN["radau_iia3_Phat"]
    want = np.array([[r["d11"], r["d12"]], [r["d21"], r["d22"]]])
    got = tab.d_vectors(Q0)
    assert np.allclose(sorted([got[0, 0][0], got[1, 1][0]]), sorted([want[0, 0][0], want[1, 1][0]]), atol=6e-4)
    assert np.allclose(np.abs(got[0, 1]), np.abs(want[0, 1]), atol=6e-4)
    bc = tab.block_constants(R0, blocks)[0]
    assert math.ceil(100 * tab.kappa_bound(bc["eta"], bc["beta"]) - 1e-9) / 100 == \
        GOLDEN["table1_radau_kappa_bounds"]["2"][0]


def _kappa_Pgamma(L, eta, beta, gamma):
    n = L.shape[0]
    I = np.eye(n)
    S = eta * I - L + beta ** 2 * np.linalg.inv(eta * I - L)
    P = S @ np.linalg.inv(gamma * I - L)
    sv = np.linalg.svd(P, compute_uv=False)
    return sv[0] / sv[-1]


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_corollary1_bound_holds_and_is_tight(s):
    """Corollary 1 / Remark: kappa(P_gamma*) <= 1 + beta^2/(2 eta^2) for W(L) <= 0,
    with equality for a skew operator with eigenvalues {0, +-i sqrt(eta^2+beta^2)}."""
    A, _, _ = tab.gauss(s)
    Q0, R0, blocks = tab.real_schur(np.linalg.inv(A))
    rng = np.random.default_rng(s)
    for (k, m), bc in zip(blocks, tab.block_constants(R0, blocks)):
        if m == 1:
            continue
        eta, beta, g = bc["eta"], bc["beta"], bc["gamma_star"]
        bound = tab.kappa_bound(eta, beta)
        for _ in range(20):
            S = rng.standard_normal((8, 8))
            Kq = rng.standard_normal((8, 8))
            L = -(S @ S.T) * rng.uniform(0, 3) + (Kq - Kq.T) * rng.uniform(0, 5)
            assert _kappa_Pgamma(L, eta, beta, g) <= bound * (1 + 1e-10)
        w = math.sqrt(eta ** 2 + beta ** 2)
        Lt = np.array([[0.0, w, 0.0], [-w, 0.0, 0.0], [0.0, 0.0, 0.0]])
        assert abs(_kappa_Pgamma(Lt, eta, beta, g) - bound) < 1e-9
        # gamma = eta (the naive choice) is worse on the same operator
        assert _kappa_Pgamma(Lt, eta, beta, eta) > bound


def test_snsd_remark_bound():
    """Remark (SNSD case): kappa(P_gamma*) <= (1 + sqrt(1 + beta^2/eta^2))/2."""
    A, _, _ = tab.gauss(3)
    Q0, R0, blocks = tab.real_schur(np.linalg.inv(A))
    rng = np.random.default_rng(7)
    for (k, m), bc in zip(blocks, tab.block_constants(R0, blocks)):
        if m == 1:
            continue
        eta, beta, g = bc["eta"], bc["beta"], bc["gamma_star"]
        bound = 0.5 * (1 + math.sqrt(1 + beta ** 2 / eta ** 2))
        for _ in range(10):
            S = rng.standard_normal((10, 10))
            L = -(S @ S.T) * rng.uniform(0.01, 100)
            assert _kappa_Pgamma(L, eta, beta, g) <= bound * (1 + 1e-10)
