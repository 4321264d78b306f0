"""Pins of the oracle's operators and Newton step against mathematics that fixes them."""
import math

import numpy as np
import pytest

import workloads
from oracle import irk, tableau as tab, vsf
from oracle.operators import Problem, arakawa

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


@pytest.mark.parametrize("op,length", [("diffusion1d", 1.0), ("burgers1d", 1.0),
                                       ("burgers2d", 1.0), ("vsf", 2 * math.pi)])
def test_jacobian_matches_finite_differences(op, length):
    p = Problem(op, 12, 0.013, length)
    rng = np.random.default_rng(3)
    U, V = rng.standard_normal(p.shape), rng.standard_normal(p.shape)
    e = 1e-6
    fd = (p.N(U + e * V) - p.N(U - e * V)) / (2 * e)
    assert np.abs(fd - p.jvp(U, V)).max() < 1e-8 * np.abs(fd).max()


def test_arakawa_conservation_and_consistency():
    """Arakawa (1966): sum J = sum psi J = sum w J = 0 on a periodic grid, and
    J_A -> psi_x w_y - psi_y w_x at second order."""
    rng = np.random.default_rng(0)
    n = 16
    psi, w = rng.standard_normal((2, n, n))
    J = arakawa(psi, w, 0.3)
    for weight in (np.ones_like(psi), psi, w):
        assert abs(np.sum(weight * J)) < 1e-11 * np.sum(np.abs(J))
    errs = []
    for n in (32, 64, 128):
        h = 2 * np.pi / n
        x = np.arange(n) * h
        X, Y = np.meshgrid(x, x, indexing="xy")
        psi = np.sin(X) * np.cos(2 * Y)
        w = np.cos(3 * X + Y)
        exact = (np.cos(X) * np.cos(2 * Y)) * (-np.sin(3 * X + Y)) \
            - (-2 * np.sin(X) * np.sin(2 * Y)) * (-3 * np.sin(3 * X + Y))
        errs.append(np.abs(arakawa(psi, w, h) - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.9)


def test_burgers2d_consistency_and_burgers1d_conservation():
    errs = []
    for n in (32, 64, 128):
        p = Problem("burgers2d", n, 0.01)
        x = np.arange(n) * p.h
        X, Y = np.meshgrid(x, x, indexing="xy")
        tp = 2 * np.pi
        u, v = np.sin(tp * X) * np.cos(tp * Y), 0.5 * np.cos(tp * X)
        ux, uy = tp * np.cos(tp * X) * np.cos(tp * Y), -tp * np.sin(tp * X) * np.sin(tp * Y)
        vx, vy = -0.5 * tp * np.sin(tp * X), 0.0 * X
        lapu, lapv = -2 * tp * tp * u, -tp * tp * v
        exact = np.stack([-u * ux - v * uy + 0.01 * lapu, -u * vx - v * vy + 0.01 * lapv])
        errs.append(np.abs(p.N(np.stack([u, v])) - exact).max())
    assert np.all(np.log2(np.array(errs[:-1]) / np.array(errs[1:])) > 1.9)
    p = Problem("burgers1d", 64, 0.01)
    u = np.random.default_rng(1).standard_normal((1, 64))
    assert abs(p.N(u).sum()) < 1e-11 * np.abs(p.N(u)).sum()


def _brute_force_step(p, s, u_n, dt, iters=8):
    """Dense Newton with a finite-difference Jacobian of the stage residual,
    solved by numpy.linalg (lstsq for the singular periodic DAE: the
    minimum-norm correction has zero-mean psi increments)."""
    A, b, c = tab.gauss(s)
    K = np.zeros((s,) + p.shape)
    m = K.size
    for _ in range(iters):
        F = irk.stage_residual(p, u_n, K, 0.0, dt, A, c).ravel()
        J = np.empty((m, m))
        e = 1e-6
        for col in range(m):
            d = np.zeros(m)
            d[col] = e
            Fp = irk.stage_residual(p, u_n, K + d.reshape(K.shape), 0.0, dt, A, c).ravel()
            Fm = irk.stage_residual(p, u_n, K - d.reshape(K.shape), 0.0, dt, A, c).ravel()
            J[:, col] = (Fp - Fm) / (2 * e)
        dk = np.linalg.lstsq(J, -F, rcond=1e-7)[0]
        K = K + dk.reshape(K.shape)
    return u_n + dt * np.tensordot(b, K, axes=(0, 0))


@pytest.mark.parametrize("op,n,s,dt,length,nu", [
    ("burgers1d", 16, 2, 1e-2, 1.0, 0.02),
    ("burgers1d", 16, 3, 1e-2, 1.0, 0.02),
    ("burgers2d", 6, 2, 1e-2, 1.0, 0.02),
    ("vsf", 6, 2, 2e-2, 2 * math.pi, 0.05),
])
def test_sparse_newton_matches_dense_brute_force(op, n, s, dt, length, nu):
    p = Problem(op, n, nu, length)
    rng = np.random.default_rng(5)
    if op == "vsf":
        w0 = rng.standard_normal((n, n))
        u_n = vsf.initial_state(w0 - w0.mean(), p.h)
    else:
        u_n = rng.standard_normal(p.shape)
    u_sparse, _, info = irk.step(p, s, u_n, 0.0, dt)
    u_dense = _brute_force_step(p, s, u_n, dt)
    if op == "vsf":  # convention: psi has zero mean (the periodic constraint fixes it up to a constant)
        u_dense[1] -= u_dense[1].mean()
    assert np.linalg.norm(u_sparse - u_dense) <= 1e-12 * np.linalg.norm(u_dense)
    assert info.residuals[-1] <= 1e-10 * info.residuals[0]


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5])
def test_linear_diffusion_matches_pade_per_mode(s):
    """Each Fourier mode m of u_t = nu L u is multiplied per step by
    R(dt lambda_m) = P(z)/P(-z), the (s,s) Pade approximant of exp, with
    lambda_m = -(4 nu/h^2) sin^2(pi m/n)."""
    n, nu, dt = 32, 0.05, 0.01
    p = Problem("diffusion1d", n, nu)
    u0 = np.random.default_rng(s).standard_normal((1, n))
    u1, _, _ = irk.step(p, s, u0, 0.0, dt)
    coef = [math.factorial(2 * s - j) * math.factorial(s)
            / (math.factorial(2 * s) * math.factorial(j) * math.factorial(s - j)) for j in range(s + 1)]
    m = np.arange(n)
    z = -dt * (4 * nu / p.h ** 2) * np.sin(np.pi * m / n) ** 2
    R = np.polyval(coef[::-1], z) / np.polyval(coef[::-1], -z)
    np.testing.assert_allclose(np.fft.fft(u1[0]), R * np.fft.fft(u0[0]), atol=1e-12 * np.abs(np.fft.fft(u0[0])).max())


@pytest.mark.parametrize("s", [1, 2, 3])
def test_observed_order_is_2s_on_manufactured_solution(s):
    """Semi-discrete manufactured solution: zero spatial error, so the error at
    T is pure time-integration error of order 2s."""
    p = Problem("burgers1d", 32, 0.02, forcing=1)
    T = 1.0
    errs = []
    steps = {1: (8, 16, 32), 2: (8, 16, 32), 3: (8, 16, 32)}[s]
    for nst in steps:
        dt = T / nst
        u, _ = irk.integrate(p, s, p.exact_manufactured(0.0), 0.0, dt, nst)
        errs.append(np.abs(u - p.exact_manufactured(T)).max())
    assert errs[-1] > 1e-12
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2 * s) < 0.35), rates


@pytest.mark.parametrize("s", [1, 2, 3, 5])
def test_sdirk_linear_diffusion_matches_stability_function(s):
    """SDIRK on u_t = nu L u multiplies mode m by R(z) = 1 + z b^T (I - z A)^{-1} 1
    (the stability function's definition), z = dt lambda_m; for backward
    Euler that is 1/(1 - z)."""
    n, nu, dt = 32, 0.05, 0.01
    p = Problem("diffusion1d", n, nu)
    u0 = np.random.default_rng(10 + s).standard_normal((1, n))
    u1, _, _ = irk.step(p, s, u0, 0.0, dt, family="sdirk")
    A, b, _ = tab.sdirk(s)
    m = np.arange(n)
    z = -dt * (4 * nu / p.h ** 2) * np.sin(np.pi * m / n) ** 2
    R = np.array([1.0 + zz * (b @ np.linalg.solve(np.eye(s) - zz * A, np.ones(s))) for zz in z])
    if s == 1:
        np.testing.assert_allclose(R, 1.0 / (1.0 - z), rtol=1e-14)
    np.testing.assert_allclose(np.fft.fft(u1[0]), R * np.fft.fft(u0[0]),
                               atol=1e-12 * np.abs(np.fft.fft(u0[0])).max())


@pytest.mark.parametrize("s,order", [(1, 1), (2, 2), (3, 3), (5, 4)])
def test_sdirk_observed_order_on_manufactured_solution(s, order):
    """Same manufactured solution as above: SDIRK's error falls at its
    classical order (1, 2, 3, 4) once dt is in the asymptotic range."""
    p = Problem("burgers1d", 32, 0.02, forcing=1)
    errs = []
    for nst in (16, 32, 64):
        u, _ = irk.integrate(p, s, p.exact_manufactured(0.0), 0.0, 1.0 / nst, nst, family="sdirk")
        errs.append(np.abs(u - p.exact_manufactured(1.0)).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - order) < 0.3), rates


def test_newton_quadratic_convergence_config0():
    p = Problem("burgers1d", 256, 0.01)
    u0 = workloads.burgers1d_initial(256, seed=0)[None]
    _, _, info = irk.step(p, 2, u0, 0.0, 1e-3, extra=0)
    r = np.array(info.residuals) / info.residuals[0]
    assert r[-1] <= 1e-10
    # quadratic: log r_{k+1} ~ 2 log r_k
    assert math.log10(r[2]) < 1.6 * math.log10(r[1])


def test_conservation_of_mean():
    p = Problem("burgers1d", 64, 0.01)
    u0 = workloads.burgers1d_initial(64, seed=3)[None]
    u, _ = irk.integrate(p, 2, u0, 0.0, 1e-2, 3)
    assert abs(u.mean() - u0.mean()) < 1e-14
    q = Problem("vsf", 16, 1e-2, 2 * math.pi)
    st = vsf.initial_state(workloads.double_shear_layer_vorticity(16), q.h)
    st1, _, _ = irk.step(q, 2, st, 0.0, 1e-2)
    assert abs(st1[0].mean()) < 1e-13 and abs(st1[1].mean()) < 1e-13


def test_vsf_direct_matches_psi_eliminated_variant():
    n = 16
    p = Problem("vsf", n, 1e-3, 2 * math.pi)
    st = vsf.initial_state(workloads.double_shear_layer_vorticity(n), p.h)
    u1, _, _ = irk.step(p, 3, st, 0.0, 5e-3)
    u2, _, _ = vsf.reduced_step(p, 3, st, 0.0, 5e-3)
    assert np.linalg.norm(u1 - u2) <= 1e-12 * np.linalg.norm(u1)
    # constraint -L psi = omega holds after the step
    g = p.N(u1)[1]
    assert np.abs(g).max() <= 1e-10 * np.abs(u1[0]).max()


def test_burgers2d_direct_matches_gmres_variant():
    p = Problem("burgers2d", 24, 5e-3)
    u0 = workloads.random_fourier_2d(24, seed=1)
    u1, _, _ = irk.step(p, 3, u0, 0.0, 2e-3)
    u2, _, _ = irk.step(p, 3, u0, 0.0, 2e-3, linear="gmres")
    assert np.linalg.norm(u1 - u2) <= 1e-12 * np.linalg.norm(u1)
