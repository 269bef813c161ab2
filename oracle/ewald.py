"""Oracle A: direct FP64 Ewald sums (Sec. 2 of Shamshirgar, Bagge & Tornberg).

TEST INFRASTRUCTURE ONLY -- imported by the tests, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``; never by the product library.

This module compiles ``ewald_direct.c`` (plain C, FP64, OpenMP over targets)
with gcc on first use and wraps each routine for numpy arrays.  Every function
takes sources ``x`` (N, 3), charges ``q`` (N,), targets ``xt`` (Nt, 3) and
returns ``(phi, grad)`` with ``grad`` the gradient of ``phi`` with respect to
the target position.  The force on a target particle of charge q_t is
``-q_t * grad``.  The box side ``L`` is a number (cube) or three numbers
(sides along x, y, z; Sec. 2: the domain need not be a cube).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ewald_direct.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle_ewald.so")
_lock = threading.Lock()
_lib = None

EULER_GAMMA = 0.57721566490153286061


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build`` (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            d = ctypes.c_double
            i = ctypes.c_int
            p = ctypes.c_void_p
            _lib.oa_special.restype = d
            _lib.oa_special.argtypes = [i, d, d]
            for name, args in {
                "oa_fourier_3p": [i, p, p, i, p, p, d, p, p, p],
                "oa_fourier_0p": [i, p, p, i, p, d, p, p],
                "oa_fourier_2p": [i, p, p, i, p, p, d, p, p, p],
                "oa_fourier_1p": [i, p, p, i, p, p, d, p, p, p],
                "oa_real": [i, i, p, p, i, p, p, d, d, p, p],
                "oa_coulomb_0p": [i, p, p, i, p, p, p],
                "oa_fourier_xi_route": [i, i, p, p, i, p, p, d, d, d, p, p],
            }.items():
                f = getattr(_lib, name)
                f.restype = None
                f.argtypes = args
    return _lib


def _prep(x, q, xt):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1)
    xt = x if xt is None else np.ascontiguousarray(xt, dtype=np.float64).reshape(-1, 3)
    phi = np.zeros(xt.shape[0])
    grad = np.zeros((xt.shape[0], 3))
    return x, q, xt, phi, grad


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def box(L) -> np.ndarray:
    """The three box sides from a number (cube) or a sequence of three."""
    b = np.broadcast_to(np.asarray(L, dtype=np.float64), (3,)).copy()
    if not np.all(b > 0):
        raise ValueError("box sides must be positive")
    return b


def kmax_n(xi: float, L: float, tail: float = 1e-20) -> int:
    """Largest |n| kept in the k-sums: e^{-k^2/(4 xi^2)} < tail at k = 2 pi n / L."""
    kmax = 2.0 * xi * np.sqrt(np.log(1.0 / tail))
    return int(np.ceil(kmax * L / (2.0 * np.pi)))


def fourier(D: int, x, q, L, xi: float, xt=None, nmax: int | None = None):
    """Fourier-space part phi^{DP,F} of Eq. (fourier_space_nonzero_ewald) in its
    closed forms: 3P k-sum (Eq. fourier_space_explicit_3P, k = 0 dropped),
    2P Eqs. (2pno0)+(2p0), 1P Eqs. (1pno0)+(1p0), 0P sum of q erf(xi r)/r."""
    lib = _load()
    x, q, xt, phi, grad = _prep(x, q, xt)
    N, Nt = x.shape[0], xt.shape[0]
    b = box(L)
    if nmax is None:
        nm = np.array([kmax_n(xi, v) for v in b], dtype=np.int32)
    else:
        nm = np.array([nmax] * 3, dtype=np.int32)
    if D == 3:
        lib.oa_fourier_3p(N, _ptr(x), _ptr(q), Nt, _ptr(xt), _ptr(b), xi, _ptr(nm), _ptr(phi), _ptr(grad))
    elif D == 2:
        lib.oa_fourier_2p(N, _ptr(x), _ptr(q), Nt, _ptr(xt), _ptr(b), xi, _ptr(nm), _ptr(phi), _ptr(grad))
    elif D == 1:
        lib.oa_fourier_1p(N, _ptr(x), _ptr(q), Nt, _ptr(xt), _ptr(b), xi, _ptr(nm), _ptr(phi), _ptr(grad))
    elif D == 0:
        lib.oa_fourier_0p(N, _ptr(x), _ptr(q), Nt, _ptr(xt), xi, _ptr(phi), _ptr(grad))
    else:
        raise ValueError("D must be 0..3")
    return phi, grad


def fourier_xi_route(D: int, x, q, L, xi: float, xt=None, xi2: float | None = None):
    """phi^{DP,F} for D = 1, 2 through the splitting-parameter independence of
    the total potential (Sec. 2): total evaluated at a small xi2 where only the
    zero mode survives.  Cost O(Nt N (images)), usable at large N."""
    if D not in (1, 2):
        raise ValueError("the xi route is for D = 1, 2")
    lib = _load()
    x, q, xt, phi, grad = _prep(x, q, xt)
    b = box(L)
    if xi2 is None:
        xi2 = 0.4 / float(np.max(b[:D]))
    rc = 6.5 / xi2
    lib.oa_fourier_xi_route(D, x.shape[0], _ptr(x), _ptr(q), xt.shape[0], _ptr(xt),
                            _ptr(b), xi, xi2, rc, _ptr(phi), _ptr(grad))
    return phi, grad


def real(D: int, x, q, L, xi: float, rc: float, xt=None):
    """Real-space sum, Eq. (real_space_ewald), images in the D periodic directions."""
    lib = _load()
    x, q, xt, phi, grad = _prep(x, q, xt)
    b = box(L)
    lib.oa_real(D, x.shape[0], _ptr(x), _ptr(q), xt.shape[0], _ptr(xt), _ptr(b), xi, rc,
                _ptr(phi), _ptr(grad))
    return phi, grad


def self_term(q, xi: float):
    """phi^self_m = -2 xi / sqrt(pi) q_m (Sec. 2)."""
    return -2.0 * xi / np.sqrt(np.pi) * np.asarray(q, dtype=np.float64)


def coulomb_0p(x, q, xt=None):
    """Direct free-space Coulomb sum, Eq. (potential) with D = 0."""
    lib = _load()
    x, q, xt, phi, grad = _prep(x, q, xt)
    lib.oa_coulomb_0p(x.shape[0], _ptr(x), _ptr(q), xt.shape[0], _ptr(xt), _ptr(phi), _ptr(grad))
    return phi, grad


def total(D: int, x, q, L, xi: float, rc: float | None = None):
    """Full Ewald potential phi^R + phi^F + phi^self at the sources (Eq. potential_split)."""
    if rc is None:
        rc = 6.5 / xi
    pr, gr = real(D, x, q, L, xi, rc)
    pf, gf = fourier(D, x, q, L, xi)
    return pr + pf + self_term(q, xi), gr + gf


# --- special functions, exposed for their pins -------------------------------

def erfcx(z):
    return _load().oa_special(0, float(z), 0.0)


def e1(x):
    return _load().oa_special(1, float(x), 0.0)


def ein(x):
    return _load().oa_special(2, float(x), 0.0)


def kinc(a, b):
    """Incomplete modified Bessel K0(a, b) = int_1^inf e^{-a t - b/t}/t dt (Eq. 1pno0)."""
    return _load().oa_special(3, float(a), float(b))


def kinc_db(a, b):
    return _load().oa_special(4, float(a), float(b))


def ekz_erfc(k, z):
    """e^{k z} erfc(k/2 + z) (xi = 1), the building block of Eq. (2pno0)."""
    return _load().oa_special(5, float(k), float(z))
