"""Exact-Newton reference for one Gauss-IRK step (oracle; test infrastructure).

Follows Sec. 1.1: u_{n+1} = u_n + dt sum_i b_i k_i (Eq. update) with
0 = M k_i - N(u_n + dt sum_j a_ij k_j, t_n + c_i dt) (Eq. stages).  For the
vorticity-streamfunction DAE (Sec. 6, Eq. dae_stage) the state is
(omega, psi), M = diag(I, 0), the second row of N is the constraint G, and
psi_{n+1} = psi_n + dt sum_i b_i l_i with l_i the psi-stage increments.

Newton: k^(0) = 0; every iteration assembles the full sN x sN Jacobian of
the stage equations, block (i, j) = delta_ij M - dt a_ij dN/du(Y_i)
(Eq. k0, with the exact linearisation L_i = dN/du at stage i), solves it
with a sparse LU (SuperLU) or with restarted GMRES to rtol 1e-13, and
updates k.  It stops when ||F(k)||_2 <= rtol * ||F(0)||_2 (discrete 2-norm
over all stages, components and points) and then takes `extra` further
iterations so the stored result sits at the rounding floor.

DAE null space: with periodic boundaries the psi-increments are fixed only
up to one constant per stage.  The direct solve replaces the constraint row
at grid point 0 of each stage by l_i[0] = 0 and every correction is then
projected to zero mean in psi (a constant psi changes no other equation).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .operators import Problem
from . import tableau as tab


@dataclass
class NewtonInfo:
    iterations: int = 0
    residuals: list = field(default_factory=list)
    linear_iterations: int = 0
    seconds: float = 0.0


def stage_states(u_n: np.ndarray, K: np.ndarray, dt: float, A: np.ndarray) -> np.ndarray:
    """Y_i = u_n + dt sum_j a_ij k_j for all i."""
    return u_n[None] + dt * np.tensordot(A, K, axes=(1, 0))


def stage_residual(prob: Problem, u_n, K, t_n, dt, A, c) -> np.ndarray:
    """F_i = M k_i - N(Y_i, t_n + c_i dt) (Eq. stages; Eq. dae_stage for VSF)."""
    Y = stage_states(u_n, K, dt, A)
    m = prob.mass.reshape((prob.ncomp,) + (1,) * prob.dim)
    F = np.empty_like(K)
    for i in range(K.shape[0]):
        F[i] = m * K[i] - prob.N(Y[i], t_n + c[i] * dt)
    return F


def newton_matrix(prob: Problem, u_n, K, dt, A) -> sp.csr_matrix:
    """Jacobian of the stage equations: block (i,j) = d_ij M - dt a_ij N'(Y_i)."""
    s = K.shape[0]
    Y = stage_states(u_n, K, dt, A)
    Mdiag = sp.diags(np.repeat(prob.mass, prob.npts))
    Js = [prob.jacobian(Y[i]) for i in range(s)]
    blocks = [[(Mdiag if i == j else None) for j in range(s)] for i in range(s)]
    for i in range(s):
        for j in range(s):
            term = -dt * A[i, j] * Js[i]
            blocks[i][j] = term if blocks[i][j] is None else blocks[i][j] + term
    return sp.bmat(blocks, format="csc")


def _pin_dae(prob: Problem, J: sp.csc_matrix, rhs: np.ndarray, s: int):
    """Replace the constraint row at point 0 of each stage by l_i[0] = 0."""
    if prob.op != "vsf":
        return J, rhs
    J = J.tolil()
    rhs = rhs.copy()
    for i in range(s):
        row = i * prob.size + prob.npts  # first psi row of stage i
        J.rows[row] = [row]
        J.data[row] = [1.0]
        rhs[row] = 0.0
    return J.tocsc(), rhs


def _project_psi(prob: Problem, dK: np.ndarray) -> np.ndarray:
    if prob.op == "vsf":
        dK[:, 1] -= dK[:, 1].mean(axis=(-2, -1), keepdims=True)
    return dK


def step(prob: Problem, s: int, u_n: np.ndarray, t_n: float, dt: float, *,
         linear: str = "direct", rtol: float = 1e-10, extra: int = 1,
         maxit: int = 30, gmres_rtol: float = 1e-13, family: str = "gauss"):
    """One IRK step (Gauss unless `family` says 'radau' or 'lobatto') by exact
    Newton.  Returns (u_{n+1}, K, NewtonInfo)."""
    A, b, c = tab.tableau(family, s)
    u_n = np.asarray(u_n, dtype=np.float64).reshape(prob.shape)
    K = np.zeros((s,) + prob.shape)
    info = NewtonInfo()
    t0 = time.perf_counter()
    F = stage_residual(prob, u_n, K, t_n, dt, A, c)
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
        J = newton_matrix(prob, u_n, K, dt, A)
        rhs = -F.ravel()
        if linear == "direct":
            Jp, rp = _pin_dae(prob, J, rhs, s)
            dk = spla.splu(Jp).solve(rp)
        elif linear == "gmres":
            counter = [0]

            def cb(_):
                counter[0] += 1
            dk, flag = spla.gmres(J, rhs, rtol=gmres_rtol, atol=0.0, restart=200,
                                  maxiter=50, callback=cb, callback_type="pr_norm")
            if flag != 0:
                raise RuntimeError(f"oracle GMRES did not converge (flag {flag})")
            info.linear_iterations += counter[0]
        else:
            raise ValueError(linear)
        dK = _project_psi(prob, dk.reshape(K.shape))
        K = K + dK
        info.iterations += 1
        F = stage_residual(prob, u_n, K, t_n, dt, A, c)
        info.residuals.append(np.linalg.norm(F))
        if not np.isfinite(info.residuals[-1]):
            raise FloatingPointError("oracle Newton diverged")
    else:
        if remaining is None:
            raise RuntimeError("oracle Newton did not converge")
    u_next = u_n + dt * np.tensordot(b, K, axes=(0, 0))
    info.seconds = time.perf_counter() - t0
    return u_next, K, info


def integrate(prob: Problem, s: int, u0, t0: float, dt: float, nsteps: int, **kw):
    """nsteps steps from u0; returns the final state and per-step infos."""
    u = np.asarray(u0, dtype=np.float64).reshape(prob.shape)
    infos = []
    t = t0
    for _ in range(nsteps):
        u, _, info = step(prob, s, u, t, dt, **kw)
        infos.append(info)
        t += dt
    return u, infos
