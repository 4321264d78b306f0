"""Seeded synthetic inputs for the Gauss-IRK stage-solve workloads.

This module is shared by the oracle, the tests and the benchmark.  It only
draws random numbers and evaluates closed-form initial fields on a periodic
grid; it contains none of the time-integration or solver arithmetic.

Workloads (all periodic):

* ``burgers1d_initial``  -- 1D viscous Burgers, x in [0,1):
  u0 = sin(2 pi x) + 0.5 sin(4 pi x) + 1e-3 N(0,1) noise.
* ``random_fourier_2d``  -- 2D viscous Burgers (u,v), [0,1)^2: per component a
  sum of 16 distinct integer wavevectors with 1 <= |k| <= 8, amplitude
  N(0,1)/|k|^2 and a uniform random phase.
* ``double_shear_layer_vorticity`` -- vorticity of the double shear layer
  on [0,2 pi)^2 (Bell-Colella-Glaz form, rho=30, delta=0.05) plus a seeded
  1e-3 N(0,1) perturbation, with the discrete mean removed.  The consistent
  streamfunction is *not* produced here: each solver derives it from the
  constraint with its own Poisson solve.

Arrays are float64, C-contiguous; 2D fields are indexed [y, x].
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "grid_1d",
    "grid_2d",
    "burgers1d_initial",
    "random_fourier_2d",
    "double_shear_layer_vorticity",
    "serving_requests",
]


def grid_1d(n: int, length: float = 1.0) -> np.ndarray:
    """Periodic grid points x_i = i*h, h = length/n."""
    return np.arange(n, dtype=np.float64) * (length / n)


def grid_2d(n: int, length: float = 1.0):
    """Periodic 2D grid; returns (X, Y) with arrays indexed [y, x]."""
    x = grid_1d(n, length)
    X, Y = np.meshgrid(x, x, indexing="xy")
    return X, Y


def burgers1d_initial(n: int = 256, seed: int = 0, noise: float = 1e-3) -> np.ndarray:
    """u0(x) = sin(2 pi x) + 0.5 sin(4 pi x) + noise * N(0,1) on [0,1)."""
    x = grid_1d(n, 1.0)
    rng = np.random.default_rng(seed)
    u = np.sin(2 * np.pi * x) + 0.5 * np.sin(4 * np.pi * x)
    return u + noise * rng.standard_normal(n)


def _random_wavevectors(rng: np.random.Generator, count: int, kmax: int):
    cands = [
        (kx, ky)
        for kx in range(-kmax, kmax + 1)
        for ky in range(-kmax, kmax + 1)
        if 1.0 <= np.hypot(kx, ky) <= kmax
    ]
    idx = rng.choice(len(cands), size=count, replace=False)
    return [cands[i] for i in idx]


def random_fourier_2d(n: int = 512, seed: int = 1, modes: int = 16, kmax: int = 8,
                      components: int = 2) -> np.ndarray:
    """Sum of `modes` random Fourier modes per component on [0,1)^2.

    Returns shape (components, n, n).  For each component: `modes` distinct
    integer wavevectors with 1 <= |k| <= kmax drawn uniformly, amplitude
    a ~ N(0,1)/|k|^2, phase ~ U[0, 2 pi); u = sum a cos(2 pi k.x + phase).
    """
    rng = np.random.default_rng(seed)
    X, Y = grid_2d(n, 1.0)
    out = np.zeros((components, n, n))
    for c in range(components):
        ks = _random_wavevectors(rng, modes, kmax)
        amp = rng.standard_normal(modes)
        phase = rng.uniform(0.0, 2 * np.pi, modes)
        for (kx, ky), a, ph in zip(ks, amp, phase):
            kk = kx * kx + ky * ky
            out[c] += (a / kk) * np.cos(2 * np.pi * (kx * X + ky * Y) + ph)
    return out


def double_shear_layer_vorticity(n: int = 1024, seed: int = 2, rho: float = 30.0,
                                 delta: float = 0.05, perturb: float = 1e-3) -> np.ndarray:
    """Double-shear-layer vorticity on [0, 2 pi)^2, indexed [y, x].

    w0 = delta cos x - rho sech^2(rho (y - pi/2))       for y <= pi
    w0 = delta cos x + rho sech^2(rho (3 pi/2 - y))     for y >  pi
    plus perturb * N(0,1) pointwise; the discrete mean is subtracted.
    """
    X, Y = grid_2d(n, 2 * np.pi)
    lower = delta * np.cos(X) - rho / np.cosh(rho * (Y - np.pi / 2)) ** 2
    upper = delta * np.cos(X) + rho / np.cosh(rho * (3 * np.pi / 2 - Y)) ** 2
    w = np.where(Y <= np.pi, lower, upper)
    rng = np.random.default_rng(seed)
    w = w + perturb * rng.standard_normal((n, n))
    return w - w.mean()


def serving_requests(count: int = 512, seed: int = 4, grids=(64, 128, 256, 512),
                     stages=(2, 3, 4), nu_range=(1e-3, 1e-1)):
    """Request descriptors for the serving mix: list of dicts with keys
    id, n, s, nu (log-uniform), seed (= request id)."""
    rng = np.random.default_rng(seed)
    out = []
    lo, hi = np.log(nu_range[0]), np.log(nu_range[1])
    for r in range(count):
        out.append({
            "id": r,
            "n": int(rng.choice(grids)),
            "s": int(rng.choice(stages)),
            "nu": float(np.exp(rng.uniform(lo, hi))),
            "seed": r,
        })
    return out
