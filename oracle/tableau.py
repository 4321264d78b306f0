"""Butcher tableau and the A0^{-1} transform (oracle side; test infrastructure).

Gauss collocation (Sec. 1.1, Eq. update/stages): the abscissae c_i are the
Gauss-Legendre nodes mapped to [0,1]; a_ij = int_0^{c_i} l_j(tau) dtau and
b_j = int_0^1 l_j(tau) dtau with l_j the Lagrange basis on the nodes.
Radau IIA is collocation on the right Radau nodes (zeros of P_s - P_{s-1}).
Lobatto IIIC (Table 1) uses the Lobatto nodes (zeros of P_s - P_{s-2}),
b = the Lobatto weights, a_i1 = b_1 and the conditions
sum_j a_ij c_j^{q-1} = c_i^q / q for q = 1..s-1.
SDIRK (the diagonally implicit methods the paper compares against, Sec. 7):
lower triangular A with one diagonal value gamma, stiffly accurate.

Real Schur form (Sec. 3.1): A0^{-1} = Q0 R0 Q0^T with Q0 orthogonal and R0
block upper triangular, 1x1 blocks for real eigenvalues and standardized
2x2 blocks [[eta, phi], [-beta^2/phi, eta]] for pairs eta +- i beta.
d_{k,l} has entries (Q0^T)_{k,i} (Q0)_{i,l} (Eq. Q0approx).
gamma* = eta + beta^2/eta (Eq. gamma*).

Eigenvector basis: A0^{-1} = T R T^{-1} with T the real and imaginary parts
of eigenvectors and R block diagonal ([[eta, beta], [-beta, eta]] per pair);
then d_{k,l} has entries (T^{-1})_{k,i} T_{i,l}.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
from numpy.polynomial import legendre as npleg
from numpy.polynomial import polynomial as nppoly


def gauss(s: int):
    """Return (A, b, c) of the s-stage Gauss method (order 2s)."""
    if not 1 <= s <= 8:
        raise ValueError("stage count out of range")
    x, _ = npleg.leggauss(s)
    c = np.sort((x + 1.0) / 2.0)
    A, b = _lagrange_integrals(c)
    return A, b, c


def _lagrange_integrals(c):
    """(A, b) with a_ij = int_0^{c_i} l_j and b_j = int_0^1 l_j (collocation)."""
    s = len(c)
    A = np.zeros((s, s))
    b = np.zeros(s)
    for j in range(s):
        others = np.delete(c, j)
        coef = nppoly.polyfromroots(others) / np.prod(c[j] - others)
        icoef = nppoly.polyint(coef)
        b[j] = nppoly.polyval(1.0, icoef)
        for i in range(s):
            A[i, j] = nppoly.polyval(c[i], icoef)
    return A, b


def _legendre_difference_nodes(s: int, k: int):
    """Zeros of P_s - P_{s-k} mapped to [0,1], increasing."""
    coef = np.zeros(s + 1)
    coef[s] = 1.0
    coef[s - k] = -1.0
    x = np.real(npleg.legroots(coef))
    x[np.abs(x - 1.0) < 1e-12] = 1.0
    x[np.abs(x + 1.0) < 1e-12] = -1.0
    return np.sort((x + 1.0) / 2.0)


def radau_iia(s: int):
    """Return (A, b, c) of the s-stage Radau IIA method (order 2s - 1)."""
    if not 1 <= s <= 8:
        raise ValueError("stage count out of range")
    c = _legendre_difference_nodes(s, 1)
    A, b = _lagrange_integrals(c)
    return A, b, c


def lobatto_iiic(s: int):
    """Return (A, b, c) of the s-stage Lobatto IIIC method (order 2s - 2)."""
    if not 2 <= s <= 8:
        raise ValueError("stage count out of range")
    c = _legendre_difference_nodes(s, 2)
    _, b = _lagrange_integrals(c)
    A = np.zeros((s, s))
    for i in range(s):
        M = np.zeros((s, s))
        r = np.zeros(s)
        M[0, 0] = 1.0
        r[0] = b[0]
        for q in range(1, s):
            M[q] = c ** (q - 1)
            r[q] = c[i] ** q / q
        A[i] = np.linalg.solve(M, r)
    return A, b, c


def sdirk(s: int):
    """Return (A, b, c) of the L-stable, stiffly accurate SDIRK method with s
    stages used as the diagonally implicit comparison (Sec. 2.1, Sec. 7):
    s = 1 backward Euler (order 1); s = 2 gamma = 1 - sqrt(2)/2 (order 2);
    s = 3 Alexander's method, gamma the root in (1/6, 1/2) of
    x^3 - 3x^2 + 3x/2 - 1/6 (order 3); s = 5 the order-4 method of
    Hairer and Wanner (Sec. IV.6), gamma = 1/4, rational coefficients.
    """
    if s == 1:
        return np.array([[1.0]]), np.array([1.0]), np.array([1.0])
    if s == 2:
        g = 1.0 - np.sqrt(2.0) / 2.0
        A = np.array([[g, 0.0], [1.0 - g, g]])
    elif s == 3:
        r = np.roots([1.0, -3.0, 1.5, -1.0 / 6.0])
        g = float(np.real(r[(np.abs(r.imag) < 1e-12) & (r.real > 1 / 6) & (r.real < 0.5)][0]))
        t2 = 0.5 * (1.0 + g)
        b1 = -(6.0 * g * g - 16.0 * g + 1.0) / 4.0
        b2 = (6.0 * g * g - 20.0 * g + 5.0) / 4.0
        A = np.array([[g, 0.0, 0.0], [t2 - g, g, 0.0], [b1, b2, g]])
    elif s == 5:
        A = np.array([[1 / 4, 0, 0, 0, 0],
                      [1 / 2, 1 / 4, 0, 0, 0],
                      [17 / 50, -1 / 25, 1 / 4, 0, 0],
                      [371 / 1360, -137 / 2720, 15 / 544, 1 / 4, 0],
                      [25 / 24, -49 / 48, 125 / 16, -85 / 12, 1 / 4]])
    else:
        raise ValueError("SDIRK stage count must be 1, 2, 3 or 5")
    return A, A[-1].copy(), A.sum(axis=1)


def tableau(family: str, s: int):
    """(A, b, c) by family name: 'gauss', 'radau', 'lobatto' or 'sdirk'."""
    return {"gauss": gauss, "radau": radau_iia, "lobatto": lobatto_iiic,
            "sdirk": sdirk}[family](s)


def real_eigen_basis(Ainv: np.ndarray):
    """A0^{-1} = T R T^{-1}, R block diagonal with [[eta, beta], [-beta, eta]].

    Returns (T, R, blocks).  Groups are ordered by increasing real part (then
    imaginary part); each pair contributes the real and imaginary parts of the
    eigenvector of eta + i beta (beta > 0), any scaling.
    """
    s = Ainv.shape[0]
    lam, vecs = np.linalg.eig(Ainv)
    groups = []
    used = np.zeros(s, bool)
    for k in np.argsort(lam.real + 1e-9 * np.abs(lam.imag)):
        if used[k]:
            continue
        if abs(lam[k].imag) < 1e-9 * max(1.0, abs(lam[k])):
            used[k] = True
            groups.append((lam[k].real, 0.0, np.real(vecs[:, k])))
        else:
            j = int(np.argmin(np.abs(lam - np.conj(lam[k])) + used * 1e9 + (np.arange(s) == k) * 1e9))
            used[k] = used[j] = True
            kk = k if lam[k].imag > 0 else j
            groups.append((lam[kk].real, lam[kk].imag, vecs[:, kk]))
    T = np.zeros((s, s))
    R = np.zeros((s, s))
    blocks = []
    off = 0
    for eta, beta, z in groups:
        if beta == 0.0:
            T[:, off] = z / np.linalg.norm(z)
            R[off, off] = eta
            blocks.append((off, 1))
            off += 1
        else:
            T[:, off] = z.real
            T[:, off + 1] = z.imag
            R[off:off + 2, off:off + 2] = [[eta, beta], [-beta, eta]]
            blocks.append((off, 2))
            off += 2
    return T, R, blocks


def real_schur(Ainv: np.ndarray):
    """Standardized real Schur form of A0^{-1} (Sec. 3.1).

    Returns (Q0, R0, blocks) where blocks is a list of (start, size).
    SciPy's LAPACK-backed routine already returns standardized 2x2 blocks
    (equal diagonals, off-diagonals of opposite sign).
    """
    R0, Q0 = scipy.linalg.schur(Ainv, output="real")
    s = Ainv.shape[0]
    blocks = []
    k = 0
    while k < s:
        if k + 1 < s and abs(R0[k + 1, k]) > 1e-13 * np.abs(R0).max():
            blocks.append((k, 2))
            k += 2
        else:
            blocks.append((k, 1))
            k += 1
    return Q0, R0, blocks


def block_constants(R0: np.ndarray, blocks):
    """eta, beta, phi, gamma* per diagonal block (Sec. 3.1, Eq. gamma*)."""
    out = []
    for (k, m) in blocks:
        if m == 1:
            eta = R0[k, k]
            out.append(dict(eta=eta, beta=0.0, phi=0.0, gamma_star=eta))
        else:
            eta = 0.5 * (R0[k, k] + R0[k + 1, k + 1])
            phi = R0[k, k + 1]
            beta2 = -R0[k, k + 1] * R0[k + 1, k]
            out.append(dict(eta=eta, beta=np.sqrt(beta2), phi=phi,
                            gamma_star=eta + beta2 / eta))
    return out


def d_vectors(Q0: np.ndarray, Tinv: np.ndarray | None = None) -> np.ndarray:
    """d[k, l, i] = (T^{-1})_{k,i} T_{i,l} (Eq. Q0approx); T = Q0, T^{-1} = Q0^T
    unless Tinv is given."""
    Ti = Q0.T if Tinv is None else Tinv
    return np.einsum("ki,il->kli", Ti, Q0)


def kappa_bound(eta: float, beta: float) -> float:
    """Corollary 1: kappa(P_gamma*) <= 1 + beta^2 / (2 eta^2)."""
    return 1.0 + beta * beta / (2.0 * eta * eta)
