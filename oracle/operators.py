"""Periodic finite-difference right-hand sides N(u,t) and their Jacobians.

Oracle side, test infrastructure only.  Every operator acts on a state array
of shape (ncomp, n) in 1D or (ncomp, n, n) in 2D (2D indexed [y, x]); the
flattened state is component-major.  h = length / n.

Operators (the problem M u' = N(u,t) of Sec. 1.1, Eq. problem):

* diffusion1d  N(u) = nu * D2 u                                    (M = I)
* burgers1d    N(u) = -(u_{i+1}^2 - u_{i-1}^2)/(4h) + nu * D2 u     (M = I)
               conservative central form of u_t + (u^2/2)_x = nu u_xx
* burgers2d    N(u,v) = (-u Dx u - v Dy u + nu L u,
                         -u Dx v - v Dy v + nu L v)                 (M = I)
               advective central form; Dx, Dy central differences and L the
               5-point Laplacian
* vsf          state (omega, psi), M = diag(I, 0)  (Sec. 6, Eq. dae):
               N_omega = J_A(psi, omega) + nu L omega
               G       = -L psi - omega        (algebraic row, the DAE's G)
               J_A is Arakawa's (1966) energy- and enstrophy-conserving
               average of the three second-order Jacobians approximating
               psi_x omega_y - psi_y omega_x; velocity u = (psi_y, -psi_x),
               so J_A(psi, omega) approximates -(u . grad) omega.

Forcing 1 (1D operators only) adds the manufactured source
f(t) = u*'(t) - N_h(u*(t)) for u*(x,t) = sin(2 pi x)(1 + 0.5 sin t)
+ 0.25 cos(4 pi x) cos(2t), so that u*(t) is the exact solution of the
semi-discrete system and only time-integration error remains.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

OPS = ("diffusion1d", "burgers1d", "burgers2d", "vsf")


def _shift1(n: int, d: int) -> sp.csr_matrix:
    """(S u)_i = u_{(i+d) mod n}."""
    rows = np.arange(n)
    cols = (rows + d) % n
    return sp.csr_matrix((np.ones(n), (rows, cols)), shape=(n, n))


def _roll(u: np.ndarray, dx: int = 0, dy: int = 0) -> np.ndarray:
    """Value at (i+dx, j+dy) of a periodic field indexed [..., y, x] or [..., x]."""
    if u.ndim >= 2 and dy:
        u = np.roll(u, -dy, axis=-2)
    if dx:
        u = np.roll(u, -dx, axis=-1)
    return u


# Arakawa (1966) Jacobian as a list of bilinear terms:
# J_A(psi, w) = (1 / (12 h^2)) * sum coef * psi(ax, ay) * w(bx, by)
# with f(ax, ay) the value at (i+ax, j+ay).  Each of the three forms
# J++, J+x, Jx+ contributes 8 terms with coefficient +-1, divided by 4h^2,
# and the average divides by 3.
_ARAKAWA_TERMS = (
    # J++ = (psi_x)(w_y) - (psi_y)(w_x) with central differences
    (+1, (1, 0), (0, 1)), (-1, (1, 0), (0, -1)), (-1, (-1, 0), (0, 1)), (+1, (-1, 0), (0, -1)),
    (-1, (0, 1), (1, 0)), (+1, (0, 1), (-1, 0)), (+1, (0, -1), (1, 0)), (-1, (0, -1), (-1, 0)),
    # J+x = d_x(psi w_y) - d_y(psi w_x)
    (+1, (1, 0), (1, 1)), (-1, (1, 0), (1, -1)), (-1, (-1, 0), (-1, 1)), (+1, (-1, 0), (-1, -1)),
    (-1, (0, 1), (1, 1)), (+1, (0, 1), (-1, 1)), (+1, (0, -1), (1, -1)), (-1, (0, -1), (-1, -1)),
    # Jx+ = d_y(w psi_x) - d_x(w psi_y)
    (+1, (1, 1), (0, 1)), (-1, (-1, 1), (0, 1)), (-1, (1, -1), (0, -1)), (+1, (-1, -1), (0, -1)),
    (-1, (1, 1), (1, 0)), (+1, (1, -1), (1, 0)), (+1, (-1, 1), (-1, 0)), (-1, (-1, -1), (-1, 0)),
)


def arakawa(psi: np.ndarray, w: np.ndarray, h: float) -> np.ndarray:
    """Arakawa Jacobian J_A(psi, w) written from the three central forms."""
    def f(a, dx, dy):
        return _roll(a, dx, dy)
    jpp = ((f(psi, 1, 0) - f(psi, -1, 0)) * (f(w, 0, 1) - f(w, 0, -1))
           - (f(psi, 0, 1) - f(psi, 0, -1)) * (f(w, 1, 0) - f(w, -1, 0)))
    jpx = (f(psi, 1, 0) * (f(w, 1, 1) - f(w, 1, -1))
           - f(psi, -1, 0) * (f(w, -1, 1) - f(w, -1, -1))
           - f(psi, 0, 1) * (f(w, 1, 1) - f(w, -1, 1))
           + f(psi, 0, -1) * (f(w, 1, -1) - f(w, -1, -1)))
    jxp = (f(w, 0, 1) * (f(psi, 1, 1) - f(psi, -1, 1))
           - f(w, 0, -1) * (f(psi, 1, -1) - f(psi, -1, -1))
           - f(w, 1, 0) * (f(psi, 1, 1) - f(psi, 1, -1))
           + f(w, -1, 0) * (f(psi, -1, 1) - f(psi, -1, -1)))
    return (jpp + jpx + jxp) / (12.0 * h * h)


@dataclass
class Problem:
    op: str
    n: int
    nu: float
    length: float = 1.0
    forcing: int = 0

    def __post_init__(self):
        if self.op not in OPS:
            raise ValueError(f"unknown operator {self.op}")
        if self.forcing and self.dim != 1:
            raise ValueError("manufactured forcing is defined for 1D operators only")

    # ---- shapes -------------------------------------------------------
    @property
    def dim(self) -> int:
        return 1 if self.op in ("diffusion1d", "burgers1d") else 2

    @property
    def ncomp(self) -> int:
        return 1 if self.dim == 1 else 2

    @property
    def h(self) -> float:
        return self.length / self.n

    @property
    def npts(self) -> int:
        return self.n ** self.dim

    @property
    def shape(self):
        return (self.ncomp,) + (self.n,) * self.dim

    @property
    def size(self) -> int:
        return self.ncomp * self.npts

    @property
    def mass(self) -> np.ndarray:
        """Diagonal of M per component (VSF: diag(I, 0))."""
        if self.op == "vsf":
            return np.array([1.0, 0.0])
        return np.ones(self.ncomp)

    # ---- stencils -----------------------------------------------------
    def _lap(self, u):
        h2 = self.h * self.h
        if self.dim == 1:
            return (_roll(u, 1) - 2.0 * u + _roll(u, -1)) / h2
        return (_roll(u, 1, 0) + _roll(u, -1, 0) + _roll(u, 0, 1) + _roll(u, 0, -1) - 4.0 * u) / h2

    def _dx(self, u):
        return (_roll(u, 1, 0) - _roll(u, -1, 0)) / (2.0 * self.h)

    def _dy(self, u):
        return (_roll(u, 0, 1) - _roll(u, 0, -1)) / (2.0 * self.h)

    def N(self, U: np.ndarray, t: float = 0.0) -> np.ndarray:
        """Right-hand side (for VSF: (N_omega, G))."""
        U = np.asarray(U, dtype=np.float64).reshape(self.shape)
        nu, h = self.nu, self.h
        if self.op == "diffusion1d":
            out = nu * self._lap(U)
        elif self.op == "burgers1d":
            u = U[0]
            out = (-(_roll(u, 1) ** 2 - _roll(u, -1) ** 2) / (4.0 * h) + nu * self._lap(u))[None]
        elif self.op == "burgers2d":
            u, v = U
            out = np.stack([
                -u * self._dx(u) - v * self._dy(u) + nu * self._lap(u),
                -u * self._dx(v) - v * self._dy(v) + nu * self._lap(v),
            ])
        else:  # vsf
            w, psi = U
            out = np.stack([arakawa(psi, w, h) + nu * self._lap(w),
                            -self._lap(psi) - w])
        if self.forcing:
            out = out + self.forcing_term(t)
        return out

    # ---- manufactured solution (1D) ------------------------------------
    def exact_manufactured(self, t: float) -> np.ndarray:
        x = np.arange(self.n) * self.h
        u = (np.sin(2 * np.pi * x) * (1.0 + 0.5 * np.sin(t))
             + 0.25 * np.cos(4 * np.pi * x) * np.cos(2.0 * t))
        return u[None]

    def _exact_manufactured_dt(self, t: float) -> np.ndarray:
        x = np.arange(self.n) * self.h
        return (np.sin(2 * np.pi * x) * 0.5 * np.cos(t)
                - 0.5 * np.cos(4 * np.pi * x) * np.sin(2.0 * t))[None]

    def forcing_term(self, t: float) -> np.ndarray:
        ustar = self.exact_manufactured(t)
        saved, self.forcing = self.forcing, 0
        try:
            nh = self.N(ustar, t)
        finally:
            self.forcing = saved
        return self._exact_manufactured_dt(t) - nh

    # ---- sparse Jacobian dN/du ------------------------------------------
    def _sparse_ops(self):
        n = self.n
        if self.dim == 1:
            E, W = _shift1(n, 1), _shift1(n, -1)
            I = sp.identity(n, format="csr")
            return dict(I=I, S=lambda dx, dy=0: _shift1(n, dx))
        I1 = sp.identity(n, format="csr")
        I = sp.identity(n * n, format="csr")

        def S(dx, dy=0):
            return sp.kron(_shift1(n, dy), _shift1(n, dx), format="csr")
        return dict(I=I, S=S)

    def jacobian(self, U: np.ndarray) -> sp.csr_matrix:
        """Exact Jacobian dN/du at U as a sparse (size x size) matrix."""
        U = np.asarray(U, dtype=np.float64).reshape(self.shape)
        ops = self._sparse_ops()
        I, S = ops["I"], ops["S"]
        h, nu = self.h, self.nu
        diag = lambda a: sp.diags(np.ravel(a))  # noqa: E731
        if self.dim == 1:
            L = (S(1) - 2.0 * I + S(-1)) / (h * h)
        else:
            L = (S(1, 0) + S(-1, 0) + S(0, 1) + S(0, -1) - 4.0 * I) / (h * h)
        if self.op == "diffusion1d":
            return (nu * L).tocsr()
        if self.op == "burgers1d":
            u = U[0]
            # (Jv)_i = -(u_{i+1} v_{i+1} - u_{i-1} v_{i-1}) / (2h) + nu (L v)_i
            return (-(S(1) - S(-1)) @ diag(u) / (2.0 * h) + nu * L).tocsr()
        Dx = (S(1, 0) - S(-1, 0)) / (2.0 * h)
        Dy = (S(0, 1) - S(0, -1)) / (2.0 * h)
        if self.op == "burgers2d":
            u, v = U
            uu = -diag(self._dx(u)) - diag(u) @ Dx - diag(v) @ Dy + nu * L
            uv = -diag(self._dy(u))
            vu = -diag(self._dx(v))
            vv = -diag(u) @ Dx - diag(self._dy(v)) - diag(v) @ Dy + nu * L
            return sp.bmat([[uu, uv], [vu, vv]], format="csr")
        # vsf: d/dw J_A(psi, w) = sum c diag(psi(a)) S(b); d/dpsi = sum c diag(w(b)) S(a)
        w, psi = U
        scale = 1.0 / (12.0 * h * h)
        dw = sp.csr_matrix((self.npts, self.npts))
        dpsi = sp.csr_matrix((self.npts, self.npts))
        for coef, a, b in _ARAKAWA_TERMS:
            dw = dw + coef * scale * (diag(_roll(psi, *a)) @ S(*b))
            dpsi = dpsi + coef * scale * (diag(_roll(w, *b)) @ S(*a))
        return sp.bmat([[dw + nu * L, dpsi], [-I, -L]], format="csr")

    def jvp(self, U: np.ndarray, V: np.ndarray) -> np.ndarray:
        return (self.jacobian(U) @ np.ravel(V)).reshape(self.shape)
