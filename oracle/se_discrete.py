"""Oracle B: the Spectral Ewald k-space algorithm (Alg. 4) written out plainly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  FP64 numpy; numpy's
FFT serves as the transform step (a library primitive), everything else is
plain array code in the order of Alg. 4:

  0. set-up: h, M~, L~, R, delta_L (Alg. 4 step 0; Sec. 3.3);
  1. gridding, Eq. (gridding), on M^D x M~^(3-D) points;
  2. FFT (D = 3), AFT (Alg. 1, D = 1, 2) or (2 M~)^3-point FFT (D = 0);
  3. scaling, Eq. (scale), with G^{DP} of Eqs. (G_hat_3d)-(G_hat_0d), or the
     precomputed G^{0P}_R of Alg. 3 for D = 0;
  4. IFFT / AIFT (Alg. 2, truncating to M~ in each free direction);
  5. gathering, Eq. (complete_integral) by the trapezoidal rule, and its
     gradient, Eq. (force-method-1).
Forces by method 2 of Sec. 7.2: the scaling of step 3 is multiplied by i k_a
for each direction a, steps 4-5 run once per direction, and the gathering uses
W itself.  At the Nyquist index of an even-length transform the factor i k_a
is set to zero: it is the odd part of a real signal that the real-valued
inverse transform cannot represent (taking the real part of the complex
inverse transform removes exactly this term).

Discrete scaling (derived from Def. 1 with the trapezoidal rule; the paper
does not print it): with an unnormalised forward DFT and a 1/n inverse over
the (padded) transform length,
    phi_m = 4 pi h^3 sum_j W(x_m - x_j) [IDFT(sigma * DFT(H))]_j,
since the free-direction quadrature weight (Delta kappa / 2 pi) = 1/(s_f M~ h)
equals the inverse-DFT factor of the padded length.

Grid arrays are indexed [ix, iy, iz]; x (and y for D = 2) are the periodic
directions, the free ones come last.  Free-direction node j sits at
-delta_L/2 + j h, periodic node j at j h.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import j0, j1

from . import params as prm
from .windows import Window


def ik_factor(n: int, d: float):
    """i k for the n-point DFT with spacing d: k = 2 pi m / (n d) at signed index m,
    zero at the Nyquist index m = -n/2 of an even n (method 2 of Sec. 7.2)."""
    k = 2.0 * np.pi * np.fft.fftfreq(n, d=d)
    if n % 2 == 0:
        k[n // 2] = 0.0
    return 1j * k


def green(D: int, R: float, kper2, kap):
    """Modified Green's functions G^{DP}([k, kappa]) of Eqs. (G_hat_3d), (G_hat_2d),
    (G_hat_1d), (G_hat_0d).  ``kper2`` = |k|^2 of the periodic part (0 for D = 0),
    ``kap`` = |kappa| of the free part (0 for D = 3)."""
    kper2 = np.asarray(kper2, dtype=np.float64)
    kap = np.asarray(kap, dtype=np.float64)
    kper2, kap = np.broadcast_arrays(kper2, kap)
    out = np.empty(kper2.shape)
    tot = kper2 + kap * kap
    with np.errstate(divide="ignore", invalid="ignore"):
        if D == 3:
            out = np.where(tot > 0, 1.0 / np.where(tot > 0, tot, 1.0), 0.0)
        elif D == 0:
            k = kap
            ks = np.where(k > 0, k, 1.0)
            out = np.where(k > 0, 2.0 * (np.sin(R * ks / 2.0) / ks) ** 2, R * R / 2.0)
        else:
            zero = kper2 == 0
            ks = np.where(kap > 0, kap, 1.0)
            if D == 2:
                g0 = np.where(kap > 0, (1.0 - np.cos(R * ks) - R * ks * np.sin(R * ks)) / ks ** 2,
                              -R * R / 2.0)
            else:
                g0 = np.where(kap > 0,
                              (1.0 - j0(R * ks)) / ks ** 2 - R * math.log(R) * j1(R * ks) / ks,
                              R * R / 4.0 * (1.0 - 2.0 * math.log(R)))
            out = np.where(zero, g0, 1.0 / np.where(tot > 0, tot, 1.0))
    return out


class SEOracle:
    """Discrete Spectral Ewald evaluation with the paper's parameters.

    window: 'gaussian', 'kb' or 'pkb'.  ``L`` is the cube's side or the three
    box sides (each an even multiple of h = L_x / M).  ``lam``, ``s0``,
    ``s_mt`` (= s M~, a number or one per axis), ``nl`` (the half-width of
    the set I in mode indices, a number or one per axis) override the Sec. 6
    rules; ``eps_rel`` feeds Eqs. (estimate-s), (estimate-nl).
    """

    def __init__(self, D: int, L, xi: float, M: int, P: int, window: str = "pkb",
                 eps_rel: float = 1e-10, lam=None, s0=None, s_mt=None, nl=None, nu=None,
                 shape=None):
        if M % 2 or P % 2 or P > M:
            raise ValueError("M and P must be even with P <= M (Sec. 3.3)")
        self.g = prm.grid(D, L, M, P, window, eps_rel=eps_rel, lam=lam, s0=s0)
        self.D, self.xi, self.M, self.P = D, xi, M, P
        self.Lv = self.g["Lv"]
        self.L = float(self.Lv[0])
        if s_mt is not None:
            sv = list(np.broadcast_to(np.asarray(s_mt), (3,)))
            self.g["sMt_v"] = [self.g["Mv"][i] if i < D else int(sv[i]) for i in range(3)]
            self.g["sMt"] = self.g["sMt_v"][min(D, 2)]
        if nl is not None:
            nv = list(np.broadcast_to(np.asarray(nl), (3,)))
            self.g["nI"] = [int(nv[i]) if i < D else 0 for i in range(3)]
            self.g["nl"] = self.g["nI"][0]
        self.h = self.g["h"]
        self.Mt = self.g["Mt"]
        self.Mv = self.g["Mv"]
        self.Mt_v = self.g["Mt_v"]
        self.n = [self.Mv[i] if i < D else self.Mt_v[i] for i in range(3)]
        self.off = [0.0 if i < D else self.g["dL_v"][i] / 2.0 for i in range(3)]
        kind = window
        self.shape = prm.shape("gaussian" if kind == "gaussian" else "kb", P) if shape is None else shape
        self.nu = prm.degree(P) if nu is None else nu
        self.win = Window(kind, P, self.h, self.shape, self.nu)
        if D == 0:
            self.GR = self._precompute_free_space()

    # ---- Alg. 3 ---------------------------------------------------------
    def _precompute_free_space(self):
        """Alg. 3: sample G^{0P} on s0M~_0 x s0M~_1 x s0M~_2 points at
        k_i = 2 pi n / (s0M~_i h), inverse FFT, keep the indices
        -M~_i <= j <= M~_i - 1 (wrapped) on a 2M~_0 x 2M~_1 x 2M~_2 grid, FFT.
        The result is G^{0P}_R at k_i = pi n / L~_i, n = -M~_i..M~_i-1 (FFT order)."""
        Mt, R, h = self.Mt_v, self.g["R"], self.h
        ns = self.g["s0Mt_v"]
        k = [2.0 * np.pi * np.fft.fftfreq(ns[i], d=h) for i in range(3)]
        kk = np.sqrt(k[0][:, None, None] ** 2 + k[1][None, :, None] ** 2 + k[2][None, None, :] ** 2)
        G = np.fft.ifftn(green(0, R, 0.0, kk)).real
        idx = [np.arange(-Mt[i], Mt[i]) for i in range(3)]
        GR = np.zeros(tuple(2 * m for m in Mt))
        GR[np.ix_(idx[0] % (2 * Mt[0]), idx[1] % (2 * Mt[1]), idx[2] % (2 * Mt[2]))] = \
            G[np.ix_(idx[0] % ns[0], idx[1] % ns[1], idx[2] % ns[2])]
        return np.fft.fftn(GR).real

    # ---- step 1 ----------------------------------------------------------
    def _stencil(self, x):
        """Grid coordinate t = (x + offset)/h per axis, the P support indices
        j = floor(t) - P/2 + 1 ... floor(t) + P/2, and x_m - x_j = (t - j) h."""
        P = self.P
        t = (np.asarray(x, dtype=np.float64) + np.array(self.off)) / self.h      # (N, 3)
        j = np.floor(t)[:, :, None] + np.arange(-P // 2 + 1, P // 2 + 1)[None, None, :]
        dist = (t[:, :, None] - j) * self.h                                      # (N, 3, P)
        frac = t - np.floor(t)
        j = j.astype(np.int64)
        for a in range(3):
            if a < self.D:
                j[:, a, :] %= self.n[a]
            elif j[:, a, :].min() < 0 or j[:, a, :].max() >= self.n[a]:
                raise ValueError("support leaves the extended box in a free direction")
        return j, dist, frac

    def grid_charges(self, x, q):
        """Eq. (gridding): H_j = sum_n q_n W(x_j - x_n)_* on the M^D x M~^(3-D) grid."""
        j, dist, frac = self._stencil(x)
        w, _ = self.win.stencil(frac, dist)                                      # (N, 3, P)
        H = np.zeros(self.n)
        q = np.asarray(q, dtype=np.float64)
        P = self.P
        nx, ny, nz = self.n
        for a in range(P):
            for b in range(P):
                # all P support points along z of the (a, b) column at once
                flat = (j[:, 0, a, None] * ny + j[:, 1, b, None]) * nz + j[:, 2, :]
                val = (q * w[:, 0, a] * w[:, 1, b])[:, None] * w[:, 2, :]
                H.reshape(-1)[:] += np.bincount(flat.ravel(), weights=val.ravel(), minlength=H.size)
        return H

    # ---- steps 2-4 -------------------------------------------------------
    def _sigma(self, kper2, kvecs_hat, kap, kap_hats):
        """Eq. (scale): e^{-|k|^2/4 xi^2} W^(k)^{-2} G^{DP}(k) with the 3D W^ the
        product of 1D transforms."""
        xi = self.xi
        tot = kper2 + kap ** 2
        what = kvecs_hat * kap_hats
        return np.exp(-tot / (4.0 * xi * xi)) / what ** 2 * green(self.D, self.g["R"], kper2, kap)

    def convolve(self, H, deriv=None):
        """Steps 2-4 of Alg. 4: returns H~ on the same grid as H.  With deriv = a
        (0, 1, 2) the scaling also multiplies by i k_a (method 2 of Sec. 7.2),
        which gives the derivative of H~ along direction a."""
        D, h = self.D, self.h
        hat = self.win.hat
        if D == 3:
            k = [2.0 * np.pi * np.fft.fftfreq(m, d=h) for m in self.Mv]
            kx, ky, kz = np.meshgrid(*k, indexing="ij")
            sig = self._sigma(kx ** 2 + ky ** 2 + kz ** 2, hat(kx) * hat(ky) * hat(kz), 0.0, 1.0)
            if deriv is not None:
                sig = sig * self._ik_along(deriv, list(self.Mv))
            return np.fft.ifftn(sig * np.fft.fftn(H)).real
        if D == 0:
            Mt = self.Mt_v
            n2 = [2 * m for m in Mt]
            Hp = np.zeros(tuple(n2))
            Hp[:Mt[0], :Mt[1], :Mt[2]] = H
            k = [2.0 * np.pi * np.fft.fftfreq(m, d=h) for m in n2]                 # pi n / L~_i
            kx, ky, kz = np.meshgrid(*k, indexing="ij")
            sig = np.exp(-(kx ** 2 + ky ** 2 + kz ** 2) / (4.0 * self.xi ** 2)) \
                / (hat(kx) * hat(ky) * hat(kz)) ** 2 * self.GR
            if deriv is not None:
                sig = sig * self._ik_along(deriv, n2)
            return np.fft.ifftn(sig * np.fft.fftn(Hp)).real[:Mt[0], :Mt[1], :Mt[2]]
        return self._aft_scale_aift(H, deriv)

    def _ik_along(self, a, shape):
        """i k_a on a transform grid of the given per-axis lengths (spacing h)."""
        f = ik_factor(shape[a], self.h)
        sh = [1, 1, 1]
        sh[a] = shape[a]
        return f.reshape(sh)

    def _classes(self):
        """Periodic-mode classes of Sec. 3.4: zero mode, I (Eq. I: a box of
        mode indices |m_j| <= nI_j around k = 0), J (the rest), with the
        free-direction transform lengths s0 M~_i, s M~_i and M~_i per free
        axis (Eq. upsamplings).  Returns (mask over the periodic mode grid,
        lengths of the free axes)."""
        D = self.D
        grids = np.meshgrid(*[np.fft.fftfreq(self.Mv[j], d=1.0 / self.Mv[j]).astype(np.int64) for j in range(D)],
                            indexing="ij")
        zero = np.all(np.stack([g == 0 for g in grids]), axis=0)
        inner = np.all(np.stack([np.abs(grids[j]) <= self.g["nI"][j] for j in range(D)]), axis=0) & ~zero
        outer = ~zero & ~inner
        free = range(D, 3)
        return [(zero, [self.g["s0Mt_v"][i] for i in free]), (inner, [self.g["sMt_v"][i] for i in free]),
                (outer, [self.Mt_v[i] for i in free])]

    def _aft_scale_aift(self, H, deriv=None):
        """Alg. 1 (AFT), scaling, Alg. 2 (AIFT) for D = 1, 2; deriv as in convolve."""
        D, h = self.D, self.h
        hat = self.win.hat
        per_axes = tuple(range(D))
        free_axes_n = 3 - D
        Mtf = [self.Mt_v[i] for i in range(D, 3)]
        Hk = np.fft.fftn(H, axes=per_axes)                       # Alg. 1 step 1
        kp = [2.0 * np.pi * np.fft.fftfreq(self.Mv[j], d=h) for j in range(D)]
        kgrid = np.meshgrid(*kp, indexing="ij")
        kper2_all = sum(g ** 2 for g in kgrid)
        khat_all = np.prod([hat(g) for g in kgrid], axis=0)
        out = np.empty_like(Hk)
        for mask, nf in self._classes():                         # Alg. 1 steps 2-4
            if not mask.any():
                continue
            lines = Hk[mask]                                     # (nc, Mt[, Mt])
            padded = np.zeros((lines.shape[0],) + tuple(nf), dtype=complex)
            sl = (slice(None),) + tuple(slice(0, m) for m in Mtf)
            padded[sl] = lines
            fax = tuple(range(1, 1 + free_axes_n))
            Fk = np.fft.fftn(padded, axes=fax)
            kf = [2.0 * np.pi * np.fft.fftfreq(m, d=h) for m in nf]   # 2 pi n / (s_f L~_i)
            if free_axes_n == 1:
                kap = np.abs(kf[0])[None, :]
                kaph = hat(kf[0])[None, :]
            else:
                a, b = np.meshgrid(kf[0], kf[1], indexing="ij")
                kap = np.sqrt(a ** 2 + b ** 2)[None]
                kaph = (hat(a) * hat(b))[None]
            kper2 = kper2_all[mask].reshape((-1,) + (1,) * free_axes_n)
            khat = khat_all[mask].reshape((-1,) + (1,) * free_axes_n)
            sig = self._sigma(kper2, khat, kap, kaph)
            if deriv is not None and deriv < D:                  # periodic direction
                ika = np.meshgrid(*[ik_factor(self.Mv[j], h) if j == deriv else np.ones(self.Mv[j])
                                    for j in range(D)], indexing="ij")
                sig = sig * np.prod(ika, axis=0)[mask].reshape((-1,) + (1,) * free_axes_n)
            elif deriv is not None:                              # free direction deriv - D of the class grid
                shp = [1] * (1 + free_axes_n)
                shp[1 + deriv - D] = nf[deriv - D]
                sig = sig * ik_factor(nf[deriv - D], h).reshape(shp)
            back = np.fft.ifftn(sig * Fk, axes=fax)               # Alg. 2 steps 1-3
            out[mask] = back[sl]                                 # truncate to M~, merge (step 4)
        return np.fft.ifftn(out, axes=per_axes).real             # Alg. 2 step 5

    # ---- step 5 ----------------------------------------------------------
    def gather(self, Ht, xt, grad: bool = False):
        """Eq. (complete_integral) by the trapezoidal rule, and with grad=True
        Eq. (force-method-1): the gradient with W' in place of W per axis."""
        j, dist, frac = self._stencil(xt)
        w, dw = self.win.stencil(frac, dist, grad)
        scale = 4.0 * math.pi * self.h ** 3
        P = self.P
        phi = np.zeros(j.shape[0])
        g = np.zeros((j.shape[0], 3)) if grad else None
        for a in range(P):
            for b in range(P):
                for c in range(P):
                    v = Ht[j[:, 0, a], j[:, 1, b], j[:, 2, c]]
                    phi += w[:, 0, a] * w[:, 1, b] * w[:, 2, c] * v
                    if grad:
                        g[:, 0] += dw[:, 0, a] * w[:, 1, b] * w[:, 2, c] * v
                        g[:, 1] += w[:, 0, a] * dw[:, 1, b] * w[:, 2, c] * v
                        g[:, 2] += w[:, 0, a] * w[:, 1, b] * dw[:, 2, c] * v
        phi *= scale
        if grad:
            g *= scale
        return phi, g

    def potential(self, x, q, xt=None, grad: bool = False, force_method: int = 1):
        """phi~^{DP,F} (Eq. fourier_space_ewald) at the targets (default: the
        sources) and, with grad=True, its gradient with respect to the target:
        method 1 (Eq. force-method-1, W' in the gathering) or method 2 of
        Sec. 7.2 (i k in the scaling, one inverse transform and one gathering
        with W per direction)."""
        H = self.grid_charges(x, q)
        Ht = self.convolve(H)
        xt = x if xt is None else xt
        if not grad or force_method == 1:
            return self.gather(Ht, xt, grad)
        if force_method != 2:
            raise ValueError("force_method is 1 or 2")
        phi, _ = self.gather(Ht, xt)
        g = np.stack([self.gather(self.convolve(H, deriv=a), xt)[0] for a in range(3)], axis=1)
        return phi, g
