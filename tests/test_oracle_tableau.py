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


def _kappa_P(L1, L2, eta, beta, gamma):
    """Condition number of the right-preconditioned Schur complement
    [eta I - L2 + beta^2 (eta I - L1)^{-1}] (gamma I - L2)^{-1} (Eq. P_gamma)."""
    I = np.eye(L1.shape[0])
    P = (eta * I - L2 + beta ** 2 * np.linalg.inv(eta * I - L1)) @ np.linalg.inv(gamma * I - L2)
    sv = np.linalg.svd(P, compute_uv=False)
    return sv[0] / sv[-1]


def _rotation_blocks(rng, n, a_range, b_sign):
    """Block-diagonal real normal matrix with 2x2 blocks [[a, b], [-b, a]]:
    eigenvalues a +- i b, a <= 0 drawn from a_range, b of sign b_sign."""
    D = np.zeros((n, n))
    for i in range(0, n, 2):
        a = rng.uniform(*a_range)
        b = b_sign * rng.uniform(0, 20)
        D[i:i + 2, i:i + 2] = [[a, b], [-b, a]]
    return D


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_theorem2_bound_for_distinct_operators(s):
    """Theorem (conditioning of the preconditioned operator, L1 != L2): with
    W(L1), W(L2) <= 0 and <L1 w, L2 w> >= 0 for all w, kappa(P_gamma*) <=
    2 + beta^2/eta^2 for every 2x2 block of Gauss(s).  Operator pairs: a
    non-normal L1 with L2 a positive multiple of it, and commuting normal
    pairs (shared orthogonal basis, eigenvalues a_k +- i b_k with a_k <= 0 and
    b1_k b2_k >= 0).  Both satisfy the assumptions, which the test also checks
    numerically."""
    A, _, _ = tab.gauss(s)
    Q0, R0, blocks = tab.real_schur(np.linalg.inv(A))
    rng = np.random.default_rng(100 + s)
    n = 10
    for (k, m), bc in zip(blocks, tab.block_constants(R0, blocks)):
        if m == 1:
            continue
        eta, beta, g = bc["eta"], bc["beta"], bc["gamma_star"]
        bound = 2.0 + beta ** 2 / eta ** 2
        pairs = []
        for _ in range(15):
            S = rng.standard_normal((n, n))
            Kq = rng.standard_normal((n, n))
            L1 = -(S @ S.T) * rng.uniform(0, 3) + (Kq - Kq.T) * rng.uniform(0, 5)
            pairs.append((L1, rng.uniform(0.1, 5.0) * L1))
            Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
            sign = rng.choice([-1.0, 1.0])
            D1 = _rotation_blocks(rng, n, (-30, 0), sign)
            D2 = _rotation_blocks(rng, n, (-30, 0), sign)
            pairs.append((Q @ D1 @ Q.T, Q @ D2 @ Q.T))
        for L1, L2 in pairs:
            for L in (L1, L2):  # W(L) <= 0
                assert np.linalg.eigvalsh(0.5 * (L + L.T)).max() <= 1e-9
            M = L1.T @ L2  # <L1 w, L2 w> >= 0
            assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() >= -1e-9
            kap = _kappa_P(L1, L2, eta, beta, g)
            assert kap <= bound * (1 + 1e-10), (s, kap, bound)


def _gmres_relres(M, rhs, maxit):
    """Relative residuals of unrestarted GMRES from x = 0 on a small dense
    system (Arnoldi with modified Gram-Schmidt, least squares per iteration)."""
    n = rhs.size
    b0 = np.linalg.norm(rhs)
    V = np.zeros((n, maxit + 1))
    H = np.zeros((maxit + 1, maxit))
    V[:, 0] = rhs / b0
    out = []
    for j in range(maxit):
        w = M @ V[:, j]
        for i in range(j + 1):
            H[i, j] = V[:, i] @ w
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        e1 = np.zeros(j + 2)
        e1[0] = b0
        y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
        out.append(np.linalg.norm(H[:j + 2, :j + 1] @ y - e1) / b0)
        if H[j + 1, j] <= 1e-14 * b0:
            break
        V[:, j + 1] = w / H[j + 1, j]
    return out


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_block_preconditioner_with_exact_schur_complement_two_iterations(s):
    """Sec. 4, Eqs. block0, Lprec, Schur: the block lower-triangular L_P with
    the exact Schur complement S makes GMRES on the right-preconditioned 2x2
    block system converge in two iterations.  The block system is assembled
    from the entries of R0; L_P and S from the oracle's (eta, beta, phi), so a
    wrong block constant leaves the iteration unconverged at two (checked
    with the sign of the coupling entry flipped)."""
    A, _, _ = tab.gauss(s)
    Q0, R0, blocks = tab.real_schur(np.linalg.inv(A))
    rng = np.random.default_rng(200 + s)
    n = 12
    I, Z = np.eye(n), np.zeros((n, n))
    for (k, m), bc in zip(blocks, tab.block_constants(R0, blocks)):
        if m == 1:
            continue
        eta, beta, phi = bc["eta"], bc["beta"], bc["phi"]
        S1, S2 = rng.standard_normal((n, n)), rng.standard_normal((n, n))
        K1, K2 = rng.standard_normal((n, n)), rng.standard_normal((n, n))
        L1 = -(S1 @ S1.T) + (K1 - K1.T)
        L2 = -(S2 @ S2.T) + (K2 - K2.T)
        blk = np.block([[R0[k, k] * I - L1, R0[k, k + 1] * I],
                        [R0[k + 1, k] * I, R0[k + 1, k + 1] * I - L2]])
        rhs = rng.standard_normal(2 * n)
        for coupling, converged in ((-beta ** 2 / phi, True), (beta ** 2 / phi, False)):
            schur = eta * I - L2 + beta ** 2 * np.linalg.inv(eta * I - L1)
            LP = np.linalg.inv(np.block([[eta * I - L1, Z], [coupling * I, schur]]))
            res = _gmres_relres(blk @ LP, rhs, 4)
            assert res[0] > 1e-6
            if converged:
                assert len(res) >= 2 and res[1] <= 1e-10, (s, res)
            else:
                assert res[1] > 1e-6, (s, res)


# ---------------------------------------------------------------------------
# Radau IIA and Lobatto IIIC (the other rows of Table 1)

def _order_conditions(A, b, c, p, q, r):
    """B(p), C(q), D(r) simplifying conditions (Butcher)."""
    for k in range(1, p + 1):
        assert abs(b @ c ** (k - 1) - 1.0 / k) < 5e-14, ("B", k)
    for k in range(1, q + 1):
        np.testing.assert_allclose(A @ c ** (k - 1), c ** k / k, atol=5e-14, err_msg=f"C{k}")
    for k in range(1, r + 1):
        np.testing.assert_allclose(b * c ** (k - 1) @ A, b * (1 - c ** k) / k, atol=5e-14,
                                   err_msg=f"D{k}")


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5])
def test_radau_iia_order_conditions(s):
    """Radau IIA: B(2s-1), C(s), D(s-1); c_s = 1 and b = last row (stiffly accurate)."""
    A, b, c = tab.radau_iia(s)
    _order_conditions(A, b, c, 2 * s - 1, s, s - 1)
    assert c[-1] == 1.0
    np.testing.assert_allclose(A[-1], b, atol=1e-14)
    # one order short of Gauss: B(2s) fails
    assert abs(b @ c ** (2 * s - 1) - 1.0 / (2 * s)) > 1e-6


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_lobatto_iiic_order_conditions(s):
    """Lobatto IIIC: B(2s-2), C(s-1), D(s-1); a_i1 = b_1; c_1 = 0, c_s = 1."""
    A, b, c = tab.lobatto_iiic(s)
    _order_conditions(A, b, c, 2 * s - 2, s - 1, s - 1)
    np.testing.assert_allclose(A[:, 0], b[0], atol=1e-15)
    assert c[0] == 0.0 and c[-1] == 1.0
    np.testing.assert_allclose(A[-1], b, atol=1e-14)


def test_radau_lobatto_textbook_tableaux():
    """Two- and three-stage tableaux as tabulated by Hairer and Wanner (vol. II, IV.5)."""
    A, b, c = tab.radau_iia(2)
    np.testing.assert_allclose(A, [[5 / 12, -1 / 12], [3 / 4, 1 / 4]], atol=1e-15)
    np.testing.assert_allclose(b, [3 / 4, 1 / 4], atol=1e-15)
    np.testing.assert_allclose(c, [1 / 3, 1.0], atol=1e-15)
    r6 = math.sqrt(6.0)
    A, b, c = tab.radau_iia(3)
    np.testing.assert_allclose(c, [(4 - r6) / 10, (4 + r6) / 10, 1.0], atol=1e-15)
    np.testing.assert_allclose(b, [(16 - r6) / 36, (16 + r6) / 36, 1 / 9], atol=1e-15)
    np.testing.assert_allclose(A[0], [(88 - 7 * r6) / 360, (296 - 169 * r6) / 1800,
                                      (-2 + 3 * r6) / 225], atol=1e-15)
    A, b, c = tab.lobatto_iiic(2)
    np.testing.assert_allclose(A, [[0.5, -0.5], [0.5, 0.5]], atol=1e-15)
    A, b, c = tab.lobatto_iiic(3)
    np.testing.assert_allclose(A, [[1 / 6, -1 / 3, 1 / 6], [1 / 6, 5 / 12, -1 / 12],
                                   [1 / 6, 2 / 3, 1 / 6]], atol=1e-15)
    np.testing.assert_allclose(b, [1 / 6, 2 / 3, 1 / 6], atol=1e-15)


def _pade(k, j, z):
    """(k, j) Pade approximant of exp(z) (Hairer-Wanner, Thm. IV.3.11)."""
    P = sum(math.factorial(k + j - i) * math.factorial(k)
            / (math.factorial(k + j) * math.factorial(i) * math.factorial(k - i)) * z ** i
            for i in range(k + 1))
    Q = sum(math.factorial(k + j - i) * math.factorial(j)
            / (math.factorial(k + j) * math.factorial(i) * math.factorial(j - i)) * (-z) ** i
            for i in range(j + 1))
    return P / Q


@pytest.mark.parametrize("family,s,k", [("gauss", s, s) for s in (1, 2, 3, 4, 5)]
                         + [("radau", s, s - 1) for s in (1, 2, 3, 4, 5)]
                         + [("lobatto", s, s - 2) for s in (2, 3, 4, 5)])
def test_stability_function_is_pade(family, s, k):
    """R(z) = 1 + z b^T (I - zA)^{-1} 1 equals the (k, s) Pade approximant:
    k = s (Gauss), s-1 (Radau IIA), s-2 (Lobatto IIIC)."""
    A, b, _ = tab.tableau(family, s)
    for z in (-0.3, -2.0 + 1.5j, 0.7j, -40.0, 1.2 - 0.4j):
        R = 1 + z * b @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))
        assert abs(R - _pade(k, s, z)) < 1e-12 * max(1.0, abs(R)), z


@pytest.mark.parametrize("family,key", [("radau", "table1_radau_kappa_bounds"),
                                        ("lobatto", "table1_lobatto_kappa_bounds")])
@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_table1_radau_lobatto(family, key, s):
    """Table 1 rows for Radau IIA and Lobatto IIIC (Corollary 1 bounds).  Most
    printed values are rounded up, two (Radau s=5: 2.6021 -> 2.60, Lobatto s=5:
    1.1918 -> 1.19) to nearest, so each must be one of the two roundings."""
    A, _, _ = tab.tableau(family, s)
    Ainv = np.linalg.inv(A)
    Q0, R0, blocks = tab.real_schur(Ainv)
    np.testing.assert_allclose(Q0 @ R0 @ Q0.T, Ainv, atol=1e-11)
    bounds = sorted(tab.kappa_bound(bc["eta"], bc["beta"]) for bc in tab.block_constants(R0, blocks))
    printed = sorted(GOLDEN[key][str(s)])
    assert len(bounds) == len(printed)
    for got, want in zip(bounds, printed):
        up = math.ceil(100 * got - 1e-9) / 100
        near = round(100 * got) / 100
        assert want in (up, near), (got, want)
    # Assumption of Sec. 2: A0^{-1} positive stable
    assert all(bc["eta"] > 0 for bc in tab.block_constants(R0, blocks))


@pytest.mark.parametrize("family", ["gauss", "radau", "lobatto"])
@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_eigen_basis(family, s):
    """A0^{-1} = T R T^{-1} with R = diag of [[eta, beta], [-beta, eta]] blocks whose
    eta, beta are the Schur blocks' (the eigenvalues); d-vectors sum to delta_kl."""
    A, _, _ = tab.tableau(family, s)
    Ainv = np.linalg.inv(A)
    T, R, blocks = tab.real_eigen_basis(Ainv)
    np.testing.assert_allclose(T @ R @ np.linalg.inv(T), Ainv, atol=1e-11)
    mask = np.zeros((s, s), bool)
    for (k, m) in blocks:
        mask[k:k + m, k:k + m] = True
        if m == 2:
            assert R[k, k] == R[k + 1, k + 1] and R[k, k + 1] == -R[k + 1, k] > 0
    assert np.all(R[~mask] == 0)
    _, R0, sblocks = tab.real_schur(Ainv)
    se = sorted((round(b["eta"], 10), round(b["beta"], 10)) for b in tab.block_constants(R0, sblocks))
    ee = sorted((round(R[k, k], 10), round(R[k, k + 1] if m == 2 else 0.0, 10)) for (k, m) in blocks)
    assert se == ee
    d = tab.d_vectors(T, np.linalg.inv(T))
    np.testing.assert_allclose(d.sum(axis=-1), np.eye(s), atol=1e-12)


def test_newton_like_1_lumping_on_radau3_example():
    """Newton-like(1) on the Radau IIA(3) example (Sec. 3.2): block i keeps only the
    stage of the largest |d_ii| entry, giving diag(L1, L2) there."""
    A, _, _ = tab.radau_iia(2)
    Q0, _, _ = tab.real_schur(np.linalg.inv(A))
    d = tab.d_vectors(Q0)
    picks = sorted(int(np.argmax(np.abs(d[i, i]))) for i in range(2))
    assert picks == [0, 1]
    np.testing.assert_allclose(sorted(np.max(np.abs(d[i, i])) for i in range(2)),
                               [GOLDEN["radau_iia3_Phat"]["d11"][0]] * 2, atol=6e-4)


def _tree_conditions(A, b, c):
    """Elementary weights minus 1/gamma(t) for the 17 rooted trees of order
    <= 5 (Butcher's order conditions, Hairer-Norsett-Wanner Sec. II.2),
    grouped by order."""
    Ac = A @ c
    out = {1: [b.sum() - 1.0],
           2: [b @ c - 1 / 2],
           3: [b @ c ** 2 - 1 / 3, b @ Ac - 1 / 6],
           4: [b @ c ** 3 - 1 / 4, b @ (c * Ac) - 1 / 8, b @ (A @ c ** 2) - 1 / 12,
               b @ (A @ Ac) - 1 / 24],
           5: [b @ c ** 4 - 1 / 5, b @ (c ** 2 * Ac) - 1 / 10, b @ (c * (A @ c ** 2)) - 1 / 15,
               b @ (c * (A @ Ac)) - 1 / 30, b @ (Ac * Ac) - 1 / 20, b @ (A @ c ** 3) - 1 / 20,
               b @ (A @ (c * Ac)) - 1 / 40, b @ (A @ (A @ c ** 2)) - 1 / 60,
               b @ (A @ (A @ Ac)) - 1 / 120]}
    return out


@pytest.mark.parametrize("s,order", [(1, 1), (2, 2), (3, 3), (5, 4)])
def test_sdirk_order_exactly(s, order):
    """Every tree condition up to the claimed order holds; one of the next
    order fails (so a dropped or mistyped coefficient cannot hide)."""
    A, b, c = tab.sdirk(s)
    np.testing.assert_allclose(A.sum(axis=1), c, atol=1e-15)
    conds = _tree_conditions(A, b, c)
    for p in range(1, order + 1):
        assert max(abs(x) for x in conds[p]) < 1e-13, (p, conds[p])
    assert max(abs(x) for x in conds[order + 1]) > 1e-4


@pytest.mark.parametrize("s", [1, 2, 3, 5])
def test_sdirk_structure_and_l_stability(s):
    """Lower triangular with one diagonal value, stiffly accurate (b = last
    row), R(inf) = 1 - b^T A^{-1} 1 = 0, |R(iy)| <= 1 (A-stability: the only
    pole 1/gamma lies in the right half-plane)."""
    A, b, c = tab.sdirk(s)
    g = A[0, 0]
    assert np.allclose(np.triu(A, 1), 0.0)
    np.testing.assert_allclose(np.diag(A), g, atol=0)
    np.testing.assert_allclose(b, A[-1], atol=0)
    assert abs(c[-1] - 1.0) < 1e-15
    e = np.ones(s)
    assert abs(1.0 - b @ np.linalg.solve(A, e)) < 1e-13
    for y in np.concatenate([np.logspace(-3, 6, 200), [1e9]]):
        R = 1.0 + 1j * y * (b @ np.linalg.solve(np.eye(s) - 1j * y * A, e))
        assert abs(R) <= 1.0 + 1e-13


def test_sdirk_closed_forms():
    """gamma of the 2-stage method solves gamma^2 - 2 gamma + 1/2 = 0 (order 2
    with b = last row); Alexander's gamma is the root near 0.4358665215 of
    its cubic; the order-4 method has the nodes 1/4, 3/4, 11/20, 1/2, 1."""
    A2, _, _ = tab.sdirk(2)
    g2 = A2[0, 0]
    assert abs(g2 * g2 - 2 * g2 + 0.5) < 1e-15
    A3, _, _ = tab.sdirk(3)
    assert abs(A3[0, 0] - 0.4358665215) < 1e-10
    A5, b5, c5 = tab.sdirk(5)
    np.testing.assert_allclose(c5, [1 / 4, 3 / 4, 11 / 20, 1 / 2, 1.0], atol=1e-15)


def test_sdirk_reversal_schur_form():
    """A0^{-1} of an SDIRK tableau is lower triangular: with the reversal
    permutation J (orthogonal), J A0^{-1} J is upper triangular with every
    diagonal entry 1/gamma, i.e. a real Schur form with 1x1 blocks only, and
    all off-diagonal d-vectors (J_km J_ml, k != l) vanish."""
    for s in (2, 3, 5):
        A, _, _ = tab.sdirk(s)
        Ainv = np.linalg.inv(A)
        J = np.eye(s)[::-1]
        R = J @ Ainv @ J
        assert np.allclose(np.tril(R, -1), 0.0, atol=1e-13)
        np.testing.assert_allclose(np.diag(R), 1.0 / A[0, 0], rtol=1e-13)
        d = tab.d_vectors(J)
        for k in range(s):
            for l in range(s):
                if k != l:
                    assert np.all(d[k, l] == 0.0)
