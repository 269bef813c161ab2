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


def box_grid(L, M: int):
    """Box sides and grid intervals per axis for a common spacing h = L_x / M
    (Sec. 2: the domain need not be a cube).  Every side must be an even
    multiple of h."""
    Lv = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,)).copy()
    h = Lv[0] / M
    Mv = []
    for v in Lv:
        m = int(round(v / h))
        if m < 2 or m % 2 or abs(m * h - v) > 1e-9 * v:
            raise ValueError("each box side must be an even multiple of h = L_x / M")
        Mv.append(m)
    return Lv, h, Mv


def grid(D: int, L, M: int, P: int, window: str, eps_rel: float = 1e-10,
         lam: float | None = None, s0: float | None = None):
    """Alg. 4 step 0 and the AFT parameters of Sec. 6 for a box with sides L
    (a number for the cube) and M intervals along x; h = L_x / M on every axis.
    Per free direction i: M~_i = 2 ceil((M_i + lambda P)/2), L~_i = h M~_i,
    delta_L_i = L~_i - L_i; R = |(L~_i)_free| (sqrt(3 - D) L~ for the cube);
    s0 M~_i and s M~_i rounded up to even integers, with s0 raised to
    1 + R / L~_i where that is larger (the oversampled grid must hold the
    truncated kernel, Sec. 3.4); n_l from Eq. (estimate-nl) per free
    direction.  The set I of Eq. (I) is the box |k_j| < 2 pi (n_l + 1) / L_f
    around k = 0 (its largest extent over the free directions f), i.e. mode
    indices |m_j| <= nI_j along each periodic direction j; for the cube
    nI_j = n_l.  The scalar entries are those of the first free axis (the
    cube's values).  ``eps_rel`` stands for eps_rms / B in Eqs. (estimate-s),
    (estimate-nl)."""
    Lv, h, Mv = box_grid(L, M)
    out = {"D": D, "L": float(Lv[0]), "Lv": Lv, "M": M, "Mv": Mv, "P": P, "h": h, "window": window}
    if D == 3:
        out.update(Mt=M, Lt=float(Lv[0]), R=0.0, dL=0.0, s0Mt=M, sMt=M, nl=0,
                   Mt_v=list(Mv), Lt_v=Lv.copy(), dL_v=np.zeros(3), s0Mt_v=list(Mv), sMt_v=list(Mv),
                   nI=[0, 0, 0])
        return out
    if lam is None:
        lam = LAMBDA[window][D]
    free = list(range(D, 3))
    Mt_v = [Mv[i] if i < D else 2 * math.ceil((Mv[i] + lam * P) / 2.0) for i in range(3)]
    Lt_v = np.array([h * m for m in Mt_v])
    R = math.sqrt(sum(Lt_v[i] ** 2 for i in free))
    s0v = S0[D] if s0 is None else s0
    s0Mt_v = [Mv[i] if i < D else even_up(max(s0v, 1.0 + R / Lt_v[i]) * Mt_v[i]) for i in range(3)]
    f = free[0]
    out.update(Mt=Mt_v[f], Lt=float(Lt_v[f]), R=R, dL=float(Lt_v[f] - Lv[f]), Mt_v=Mt_v, Lt_v=Lt_v,
               dL_v=Lt_v - Lv, s0Mt=s0Mt_v[f], s0Mt_v=s0Mt_v)
    if D == 0:
        out.update(sMt=2 * Mt_v[f], sMt_v=[2 * m for m in Mt_v], nl=0, nI=[0, 0, 0])
        return out
    lg = math.log(1.0 / (2.0 * eps_rel)) / (2.0 * math.pi)
    sMt_v = [Mv[i] if i < D else even_up(Mv[i] * (1.0 + lg)) for i in range(3)]
    nl_v = {i: max(0, math.ceil(Mv[i] / (Mt_v[i] - Mv[i]) * lg - 1.0)) for i in free}
    out.update(sMt=sMt_v[f], sMt_v=sMt_v, nl=nl_v[f], nl_v=nl_v)
    out["nI"] = i_box(D, Lv, nl_v)
    return out


def i_box(D: int, Lv, nl_v) -> list:
    """Mode-index half-widths of the set I along the periodic directions: the
    box |k_j| < k_l = max_f 2 pi (n_l,f + 1) / L_f, i.e. |m_j| <= ceil(k_l L_j / 2 pi) - 1."""
    kl = max(2.0 * math.pi * (nl_v[f] + 1) / Lv[f] for f in nl_v)
    out = [0, 0, 0]
    for j in range(D):
        out[j] = max(0, math.ceil(kl * Lv[j] / (2.0 * math.pi) - 1e-9) - 1)
    return out


def q_sum_sq(q) -> float:
    """Q = sum q_n^2 (Sec. 5.1)."""
    q = np.asarray(q, dtype=np.float64)
    return float(np.dot(q, q))
