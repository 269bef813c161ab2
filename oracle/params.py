"""Parameter rules of the Spectral Ewald method (Secs. 3.3, 5 and 6).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Plain FP64 Python.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import lambertw

# Eq. (fc-expression): curve-fitted constants of f_c.
FC_C1, FC_C2, FC_C3, FC_C4 = 12.62, 0.8909, 0.01411, 4.315e-5
# Sec. 5.2: c^2 of the Gaussian shape parameter.
GAUSS_C2 = 0.91
# Table (lambda), Sec. 6; no entry for D = 3.
LAMBDA = {"gaussian": {0: 1.0, 1: 1.5, 2: 1.5}, "pkb": {0: 1.3, 1: 2.4, 2: 2.4}}
LAMBDA["kb"] = LAMBDA["pkb"]
# Sec. 6: zero-mode / free-space upsampling factors.
S0 = {0: 2.8, 1: 2.5, 2: 2.0}


def f_c(x: float) -> float:
    """Eq. (fc-expression)."""
    return math.exp(-FC_C1 / x ** 2) * (FC_C2 + FC_C3 * x + FC_C4 * x ** 2)


def scale_B(Q: float, xi: float, L: float) -> float:
    """B = sqrt(Q) f_c(xi L) / L, the magnitude of the potential (Sec. 5.2)."""
    return math.sqrt(Q) * f_c(xi * L) / L


def kp_real(Q, xi, L, rc):
    """Kolafa-Perram real-space rms truncation error, Eq. (KP_real_space)."""
    return math.sqrt(Q) * xi ** -2 * (L * rc) ** -1.5 * math.exp(-(xi * rc) ** 2)


def kp_fourier(Q, xi, L, M):
    """Kolafa-Perram k-space rms truncation error, Eq. (KP_fourier_space), k_inf = M/2."""
    kinf = M / 2.0
    return math.sqrt(Q) * xi / math.pi ** 2 * kinf ** -1.5 * math.exp(-(math.pi * kinf / (xi * L)) ** 2)


def kp_rc(Q, xi, L, eps):
    """Cut-off radius from Eq. (KP_rc)."""
    arg = 4.0 / 3.0 * (Q / (xi * L ** 3 * eps ** 2)) ** (2.0 / 3.0)
    return math.sqrt(3.0) / (2.0 * xi) * math.sqrt(lambertw(arg).real)


def kp_kinf(Q, xi, L, eps):
    """Maximum wavenumber index from Eq. (KP_kinf)."""
    arg = 4.0 / 3.0 * (Q / (math.pi * xi * L ** 3 * eps ** 2)) ** (2.0 / 3.0)
    return math.sqrt(3.0) * xi * L / (2.0 * math.pi) * math.sqrt(lambertw(arg).real)


def approx_error(window: str, P: int, B: float) -> float:
    """Simplified approximation-error estimates: 2 B e^{-(pi/2) P c} (Gaussian),
    10 B e^{-2.5 P} (PKB / KB), Sec. 5.2."""
    if window == "gaussian":
        return 2.0 * B * math.exp(-(math.pi / 2.0) * P * math.sqrt(GAUSS_C2))
    return 10.0 * B * math.exp(-2.5 * P)


def pollution_limit(window: str, x: float) -> float:
    """f_W of Eq. (error_pollution), evaluated at x = M / (xi L)."""
    if window == "gaussian":
        return x * x + 0.2 * x + 2.25
    return 0.7 * x * x + 0.2 * x + 1.8


def even_up(v: float) -> int:
    """Smallest even integer >= v (the rounding of P, s0 M~ and s M~, Sec. 6)."""
    n = math.ceil(v - 1e-12)
    return n + (n & 1)


def shape(window: str, P: int) -> float:
    """alpha = (pi/2) P c^2 (Gaussian) or beta = 2.5 P (KB), Sec. 6."""
    if window == "gaussian":
        return math.pi / 2.0 * P * GAUSS_C2
    return 2.5 * P


def degree(P: int) -> int:
    """nu = min(P/2 + 2, 9), Sec. 6."""
    return min(P // 2 + 2, 9)


def from_tolerance(eps: float, xi: float, L: float, Q: float, window: str = "pkb"):
    """Sec. 6: grid size M = 2 k_inf from Eq. (KP_kinf) and support P from the
    approximation-error estimate, followed by the error-pollution correction."""
    B = scale_B(Q, xi, L)
    M = 2 * math.ceil(kp_kinf(Q, xi, L, eps))
    if window == "gaussian":
        P = math.log(2.0 * B / eps) / ((math.pi / 2.0) * math.sqrt(GAUSS_C2))
    else:
        P = math.log(10.0 * B / eps) / 2.5
    P = max(2, even_up(P))
    if P > pollution_limit(window, M / (xi * L)):
        M = even_up(1.05 * M)
        P = P + 4
    return M, P


def grid(D: int, L: float, M: int, P: int, window: str, eps_rel: float = 1e-10,
         lam: float | None = None, s0: float | None = None):
    """Alg. 4 step 0 and the AFT parameters of Sec. 6:
    h, M~ = 2 ceil((M + lambda P)/2), L~ = h M~, R = sqrt(3-D) L~, delta_L,
    s0 M~, s M~ (both rounded up to even integers) and n_l.
    ``eps_rel`` stands for eps_rms / B in Eqs. (estimate-s), (estimate-nl)."""
    h = L / M
    out = {"D": D, "L": L, "M": M, "P": P, "h": h, "window": window}
    if D == 3:
        out.update(Mt=M, Lt=L, R=0.0, dL=0.0, s0Mt=M, sMt=M, nl=0)
        return out
    if lam is None:
        lam = LAMBDA[window][D]
    Mt = 2 * math.ceil((M + lam * P) / 2.0)
    Lt = h * Mt
    out.update(Mt=Mt, Lt=Lt, R=math.sqrt(3 - D) * Lt, dL=Lt - L)
    s0v = S0[D] if s0 is None else s0
    out["s0Mt"] = even_up(s0v * Mt)
    if D == 0:
        out.update(sMt=2 * Mt, nl=0)
        return out
    lg = math.log(1.0 / (2.0 * eps_rel)) / (2.0 * math.pi)
    out["sMt"] = even_up(M / Mt * (1.0 + lg) * Mt)
    out["nl"] = max(0, math.ceil(M / (Mt - M) * lg - 1.0))
    return out


def q_sum_sq(q) -> float:
    """Q = sum q_n^2 (Sec. 5.1)."""
    q = np.asarray(q, dtype=np.float64)
    return float(np.dot(q, q))
