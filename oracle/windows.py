"""Window functions of Sec. 4 and their Fourier transforms.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain FP64 numpy.

All windows are 1D functions W0(x) on the support |x| <= w = P h / 2; the 3D
window is the tensor product W0(x) W0(y) W0(z) (Sec. 4).
"""
from __future__ import annotations

import numpy as np
from scipy.special import i0, i1


def gaussian(x, w, alpha):
    """Truncated Gaussian window, Eq. (gaussian)."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(np.abs(x) <= w, np.exp(-alpha * (x / w) ** 2), 0.0)


def gaussian_dx(x, w, alpha):
    x = np.asarray(x, dtype=np.float64)
    return np.where(np.abs(x) <= w, -2.0 * alpha * x / w ** 2 * np.exp(-alpha * (x / w) ** 2), 0.0)


def gaussian_hat(k, w, alpha):
    """Fourier transform of the untruncated Gaussian (the one the scaling uses, Sec. 4)."""
    k = np.asarray(k, dtype=np.float64)
    return np.sqrt(np.pi / alpha) * w * np.exp(-k * k * w * w / (4.0 * alpha))


def kaiser(x, w, beta):
    """Kaiser-Bessel window, Eq. (kaiser_window)."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.clip(1.0 - (x / w) ** 2, 0.0, None))
    return np.where(np.abs(x) <= w, i0(beta * s) / i0(beta), 0.0)


def kaiser_dx(x, w, beta):
    """d/dx of Eq. (kaiser_window): I1(beta s) beta ds/dx / I0(beta), s = sqrt(1-(x/w)^2),
    written with I1(z)/z (-> 1/2 at z = 0) so that it stays finite at |x| = w."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.clip(1.0 - (x / w) ** 2, 0.0, None))
    z = beta * s
    i1_over_z = np.where(z > 1e-8, i1(z) / np.where(z > 1e-8, z, 1.0), 0.5)
    return np.where(np.abs(x) <= w, -beta * beta * i1_over_z * x / (w * w) / i0(beta), 0.0)


def kaiser_hat(k, w, beta):
    """Eq. (kaiser_ft): 2 w sinh(sqrt(beta^2 - k^2 w^2)) / (I0(beta) sqrt(beta^2 - k^2 w^2)),
    continued by sin(sqrt(k^2 w^2 - beta^2)) / sqrt(.) past k w = beta."""
    k = np.asarray(k, dtype=np.float64)
    a = beta * beta - (k * w) ** 2
    ra = np.sqrt(np.abs(a))
    with np.errstate(invalid="ignore", divide="ignore"):
        f = np.where(a > 0, np.sinh(ra) / np.where(ra > 0, ra, 1.0),
                     np.where(ra > 0, np.sin(ra) / np.where(ra > 0, ra, 1.0), 1.0))
    f = np.where(ra == 0, 1.0, f)
    return 2.0 * w * f / i0(beta)


class PKB:
    """Polynomial Kaiser-Bessel window (Sec. 4.1): on each of the P subintervals
    [x_i, x_i + h] of the support, a degree-nu polynomial in the monomial basis
    of xbar = 2 (x - x_i)/h - 1, fitted to W_KB at the nu + 1 Chebyshev points
    xbar_k = cos(pi (k - 1/2)/(nu + 1)), Eqs. (polynomial-ansatz), (polynomial-linsys)."""

    def __init__(self, P: int, h: float, beta: float, nu: int, target=None):
        self.P, self.h, self.beta, self.nu = P, h, beta, nu
        self.w = P * h / 2.0
        f = target if target is not None else (lambda x: kaiser(x, self.w, beta))
        k = np.arange(1, nu + 2)
        self.nodes = np.cos(np.pi * (k - 0.5) / (nu + 1))
        self.V = self.nodes[:, None] ** np.arange(nu + 1)[None, :]
        self.coef = np.empty((P, nu + 1))
        for i in range(P):
            xi_left = -self.w + i * h
            rhs = f((self.nodes + 1.0) / 2.0 * h + xi_left)
            self.coef[i] = np.linalg.solve(self.V, rhs)

    def _locate(self, x):
        x = np.asarray(x, dtype=np.float64)
        i = np.floor((x + self.w) / self.h).astype(np.int64)
        i = np.clip(i, 0, self.P - 1)
        xb = 2.0 * (x - (-self.w + i * self.h)) / self.h - 1.0
        return x, i, xb

    def __call__(self, x):
        x, i, xb = self._locate(x)
        c = self.coef[i]
        val = np.zeros_like(xb)
        for j in range(self.nu, -1, -1):
            val = val * xb + c[..., j]
        return np.where(np.abs(x) <= self.w, val, 0.0)

    def dx(self, x):
        """Exact derivative of the fitted piecewise polynomial (d xbar / dx = 2/h)."""
        x, i, xb = self._locate(x)
        c = self.coef[i]
        val = np.zeros_like(xb)
        for j in range(self.nu, 0, -1):
            val = val * xb + j * c[..., j]
        return np.where(np.abs(x) <= self.w, val * 2.0 / self.h, 0.0)

    def stencil(self, frac, k):
        """Values at the P support points of a particle whose grid coordinate has
        fractional part ``frac``: point k (counted from the lowest index) lies in
        subinterval P-1-k at the common offset xbar = 2 frac - 1 (Sec. 4.1: all
        evaluation points share one offset within their subintervals)."""
        xb = 2.0 * np.asarray(frac, dtype=np.float64) - 1.0
        c = self.coef[self.P - 1 - np.asarray(k)]
        val = np.zeros(np.broadcast(xb, np.asarray(k)).shape)
        for j in range(self.nu, -1, -1):
            val = val * xb + c[..., j]
        return val

    def stencil_dx(self, frac, k):
        """d/dx of :meth:`stencil` (d xbar / dx = 2/h)."""
        xb = 2.0 * np.asarray(frac, dtype=np.float64) - 1.0
        c = self.coef[self.P - 1 - np.asarray(k)]
        val = np.zeros(np.broadcast(xb, np.asarray(k)).shape)
        for j in range(self.nu, 0, -1):
            val = val * xb + j * c[..., j]
        return val * 2.0 / self.h

    def cond(self) -> float:
        """Condition number of the Vandermonde matrix at the Chebyshev points (Sec. 4.1)."""
        return float(np.linalg.cond(self.V))


class Window:
    """One of the three windows used by the method: 'gaussian' (Eq. gaussian with
    the untruncated transform), 'kb' (Eq. kaiser_window, exact), 'pkb' (the
    polynomial approximation of KB with the exact KB transform in the scaling)."""

    def __init__(self, kind: str, P: int, h: float, shape: float, nu: int | None = None):
        self.kind, self.P, self.h, self.shape = kind, P, h, shape
        self.w = P * h / 2.0
        if kind == "pkb":
            self.pkb = PKB(P, h, shape, nu)

    def __call__(self, x):
        if self.kind == "gaussian":
            return gaussian(x, self.w, self.shape)
        if self.kind == "kb":
            return kaiser(x, self.w, self.shape)
        return self.pkb(x)

    def dx(self, x):
        if self.kind == "gaussian":
            return gaussian_dx(x, self.w, self.shape)
        if self.kind == "kb":
            return kaiser_dx(x, self.w, self.shape)
        return self.pkb.dx(x)

    def stencil(self, frac, dist, grad=False):
        """Window values (and x-derivatives) at the P support points of each
        particle; ``frac`` (N, 3) fractional grid coordinates, ``dist`` (N, 3, P)
        = x_m - x_j.  The PKB is evaluated per support point (Sec. 4.1); the
        other windows are plain functions of the distance."""
        if self.kind != "pkb":
            return self(dist), (self.dx(dist) if grad else None)
        k = np.arange(self.P)[None, None, :]
        f = np.asarray(frac)[:, :, None]
        return self.pkb.stencil(f, k), (self.pkb.stencil_dx(f, k) if grad else None)

    def hat(self, k):
        if self.kind == "gaussian":
            return gaussian_hat(k, self.w, self.shape)
        return kaiser_hat(k, self.w, self.shape)
