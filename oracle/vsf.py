"""Vorticity-streamfunction helpers (oracle; test infrastructure).

The constraint of the DAE (Sec. 6, Eq. dae) is G(omega, psi) = -L psi - omega = 0
with L the periodic 5-point Laplacian.  On zero-mean fields it is inverted
exactly with the FFT: the 5-point symbol of -L at wavenumber (kx, ky) is
(4/h^2)(sin^2(pi kx/n) + sin^2(pi ky/n)); the (0,0) mode is set to zero.

`reduced_step` is the full-size variant of the exact-Newton reference: the
constraint is linear and index-1, so with consistent psi_n and invertible A0
every psi-stage satisfies -L Y^psi_i = Y^omega_i; eliminating psi leaves the
ODE omega' = J_A(P omega, omega) + nu L omega with P = (-L)^{-1}.  Newton on
its stage equations uses matrix-free GMRES (rtol 1e-13) on the exact
linearisation d -> J_A(P w, d) + J_A(P d, w) + nu L d.  psi_{n+1} = P omega_{n+1}.
"""
from __future__ import annotations

import time

import numpy as np
import scipy.sparse.linalg as spla

from .operators import Problem, arakawa
from . import tableau as tab
from .irk import NewtonInfo


def neg_laplacian_symbol(n: int, h: float) -> np.ndarray:
    k = np.arange(n)
    s1 = np.sin(np.pi * k / n) ** 2
    return (4.0 / (h * h)) * (s1[:, None] + s1[None, :])


def poisson_solve(omega: np.ndarray, h: float) -> np.ndarray:
    """psi with -L psi = omega - mean(omega), mean(psi) = 0."""
    n = omega.shape[-1]
    sym = neg_laplacian_symbol(n, h)
    sym[0, 0] = 1.0
    wh = np.fft.fft2(omega)
    ph = wh / sym
    ph[0, 0] = 0.0
    return np.real(np.fft.ifft2(ph))


def initial_state(omega0: np.ndarray, h: float) -> np.ndarray:
    """Consistent (omega, psi) state: psi solves -L psi = omega with zero mean."""
    return np.stack([omega0, poisson_solve(omega0, h)])


def reduced_step(prob: Problem, s: int, state: np.ndarray, t_n: float, dt: float, *,
                 rtol: float = 1e-10, extra: int = 1, maxit: int = 30,
                 gmres_rtol: float = 1e-13, family: str = "gauss"):
    """One IRK step (Gauss unless `family` is 'radau' or 'lobatto') of the
    psi-eliminated VSF system by exact Newton."""
    assert prob.op == "vsf"
    A, b, c = tab.tableau(family, s)
    h, nu = prob.h, prob.nu
    w_n = np.asarray(state[0], dtype=np.float64)
    n = prob.n
    lap = lambda f: (np.roll(f, -1, 1) + np.roll(f, 1, 1) + np.roll(f, -1, 0)  # noqa: E731
                     + np.roll(f, 1, 0) - 4.0 * f) / (h * h)

    def nred(w):
        return arakawa(poisson_solve(w, h), w, h) + nu * lap(w)

    K = np.zeros((s, n, n))
    info = NewtonInfo()
    t0 = time.perf_counter()

    def resid(K):
        Y = w_n[None] + dt * np.tensordot(A, K, axes=(1, 0))
        return np.stack([K[i] - nred(Y[i]) for i in range(s)]), Y

    F, Y = resid(K)
    f0 = np.linalg.norm(F)
    info.residuals.append(f0)
    remaining = None
    for _ in range(maxit):
        if remaining is None and np.linalg.norm(F) <= rtol * f0:
            remaining = extra
        if remaining is not None:
            if remaining == 0:
                break
            remaining -= 1
        Ps = [poisson_solve(Y[i], h) for i in range(s)]

        def matvec(x, Y=Y, Ps=Ps):
            X = x.reshape(s, n, n)
            out = X.copy()
            for i in range(s):
                d = dt * np.tensordot(A[i], X, axes=(0, 0))
                out[i] -= arakawa(Ps[i], d, h) + arakawa(poisson_solve(d, h), Y[i], h) + nu * lap(d)
            return out.ravel()
        op = spla.LinearOperator((s * n * n, s * n * n), matvec=matvec, dtype=np.float64)
        counter = [0]

        def cb(_):
            counter[0] += 1
        dk, flag = spla.gmres(op, -F.ravel(), rtol=gmres_rtol, atol=0.0, restart=200,
                              maxiter=50, callback=cb, callback_type="pr_norm")
        if flag != 0:
            raise RuntimeError("oracle GMRES did not converge")
        info.linear_iterations += counter[0]
        K = K + dk.reshape(K.shape)
        info.iterations += 1
        F, Y = resid(K)
        info.residuals.append(np.linalg.norm(F))
    else:
        if remaining is None:
            raise RuntimeError("oracle Newton did not converge")
    w_next = w_n + dt * np.tensordot(b, K, axes=(0, 0))
    info.seconds = time.perf_counter() - t0
    return np.stack([w_next, poisson_solve(w_next, h)]), K, info
