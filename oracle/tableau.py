"""Butcher tableau and the A0^{-1} transform (oracle side; test infrastructure).

Gauss collocation (Sec. 1.1, Eq. update/stages): the abscissae c_i are the
Gauss-Legendre nodes mapped to [0,1]; a_ij = int_0^{c_i} l_j(tau) dtau and
b_j = int_0^1 l_j(tau) dtau with l_j the Lagrange basis on the nodes.

Real Schur form (Sec. 3.1): A0^{-1} = Q0 R0 Q0^T with Q0 orthogonal and R0
block upper triangular, 1x1 blocks for real eigenvalues and standardized
2x2 blocks [[eta, phi], [-beta^2/phi, eta]] for pairs eta +- i beta.
d_{k,l} has entries (Q0^T)_{k,i} (Q0)_{i,l} (Eq. Q0approx).
gamma* = eta + beta^2/eta (Eq. gamma*).
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
    A = np.zeros((s, s))
    b = np.zeros(s)
    for j in range(s):
        others = np.delete(c, j)
        coef = nppoly.polyfromroots(others) / np.prod(c[j] - others)
        icoef = nppoly.polyint(coef)  # antiderivative vanishing at 0
        b[j] = nppoly.polyval(1.0, icoef)
        for i in range(s):
            A[i, j] = nppoly.polyval(c[i], icoef)
    return A, b, c


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


def d_vectors(Q0: np.ndarray) -> np.ndarray:
    """d[k, l, i] = (Q0^T)_{k,i} (Q0)_{i,l} (Eq. Q0approx)."""
    return np.einsum("ik,il->kli", Q0, Q0)


def kappa_bound(eta: float, beta: float) -> float:
    """Corollary 1: kappa(P_gamma*) <= 1 + beta^2 / (2 eta^2)."""
    return 1.0 + beta * beta / (2.0 * eta * eta)
