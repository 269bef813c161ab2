"""Pins of oracle A (direct Ewald sums) against facts fixed outside it.

Each test checks the oracle against something it does not compute itself: a
textbook constant, a mathematical identity, a library special function, or
numerical quadrature of the defining Fourier integral.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.special as sp
from scipy import integrate

from oracle import ewald as E
from paper_1712_04732_gb300 import workloads as wl

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _system(N=40, seed=5, L=1.0):
    x = wl.uniform_positions(N, L, seed)
    q = wl.uniform_charges(N, seed)
    return x, q


# ---------------------------------------------------------------- special functions

@pytest.mark.parametrize("z", [0.3, 1.9, 2.0, 2.5, 7.0, 30.0, 200.0])
def test_erfcx_matches_library(z):
    assert E.erfcx(z) == pytest.approx(sp.erfcx(z), rel=1e-14)


@pytest.mark.parametrize("x", [1e-6, 0.01, 0.7, 1.0, 1.0001, 3.0, 4.0, 4.0001, 12.0, 80.0])
def test_e1_and_ein_match_library(x):
    assert E.e1(x) == pytest.approx(sp.exp1(x), rel=1e-13)
    ein_ref = np.euler_gamma + math.log(x) + sp.exp1(x)
    assert E.ein(x) == pytest.approx(ein_ref, rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("a,b", [(0.154, 0.01), (0.154, 3.0), (0.154, 150.0), (2.0, 5.0),
                                 (0.6, 0.6), (9.0, 40.0), (39.0, 100.0)])
def test_incomplete_bessel_split_identity(a, b):
    """K0(a,b) + K0(b,a) = 2 K_0(2 sqrt(ab)): splitting int_0^inf e^{-at-b/t} dt/t
    at t = 1 (the full integral is the modified Bessel function)."""
    lhs = E.kinc(a, b) + E.kinc(b, a)
    assert lhs == pytest.approx(2.0 * sp.k0(2.0 * math.sqrt(a * b)), rel=1e-12)


@pytest.mark.parametrize("a", [0.05, 0.154, 1.0, 7.0])
def test_incomplete_bessel_b0_is_e1(a):
    """E1(x) = K0(x, 0) (Sec. 2, below Eq. 1p0)."""
    assert E.kinc(a, 0.0) == pytest.approx(sp.exp1(a), rel=1e-13)


def test_incomplete_bessel_b_derivative():
    for a, b in [(0.2, 1.0), (1.5, 4.0), (0.154, 60.0)]:
        hb = 1e-5 * max(b, 1.0)
        fd = (E.kinc(a, b + hb) - E.kinc(a, b - hb)) / (2 * hb)
        assert E.kinc_db(a, b) == pytest.approx(fd, rel=1e-7)


# ---------------------------------------------------------------- lattice sums

def test_madelung_constant_nacl():
    """NaCl: every ion of the 8x8x8 rock-salt cell (spacing a = 1/8) has
    q_i phi_i = -M / a with the textbook Madelung constant."""
    x, q = wl.nacl_cell(8, 1.0)
    a = 1.0 / 8
    phi, grad = E.total(3, x, q, 1.0, 8.0)
    mad = -(phi * q) * a
    assert np.allclose(mad, GOLDEN["madelung_nacl"]["value"], rtol=0, atol=2e-10)
    assert np.abs(grad).max() < 1e-9          # every ion sits at a symmetry point


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_total_potential_independent_of_xi(D):
    """phi^R + phi^F + phi^self does not depend on xi (Sec. 2)."""
    x, q = _system()
    ref = None
    for xi in (3.5, 6.0, 9.0):
        phi, grad = E.total(D, x, q, 1.0, xi, rc=7.0 / xi)
        if ref is None:
            ref = (phi, grad)
            continue
        assert np.abs(phi - ref[0]).max() < 1e-11 * np.abs(ref[0]).max()
        assert np.abs(grad - ref[1]).max() < 1e-10 * np.abs(ref[1]).max()


def test_free_space_total_is_coulomb():
    x, q = _system(60, 9)
    phi, grad = E.total(0, x, q, 1.0, 7.0)
    pc, gc = E.coulomb_0p(x, q)
    assert np.abs(phi - pc).max() < 1e-12 * np.abs(pc).max()
    assert np.abs(grad - gc).max() < 1e-11 * np.abs(gc).max()


@pytest.mark.parametrize("D", [2, 1])
def test_two_routes_to_the_fourier_part_agree(D):
    """Closed forms Eqs. (2pno0)+(2p0) / (1pno0)+(1p0) against the route through
    xi-independence (total at small xi2 minus the real-space part at xi)."""
    x, q = _system(50, 3)
    pf, gf = E.fourier(D, x, q, 1.0, 8.0)
    pr, gr = E.fourier_xi_route(D, x, q, 1.0, 8.0)
    assert np.abs(pf - pr).max() < 1e-11 * np.abs(pf).max()
    assert np.abs(gf - gr).max() < 1e-11 * np.abs(gf).max()


# ------------------------------------------------- the defining Fourier integrals

def _pair():
    """A neutral pair (+1, -1) and a target: the k = 0 Fourier integrals of the
    singly/doubly periodic sums are singular term by term but finite for a
    neutral set, so the quadratures below subtract the (zero) net charge."""
    xs = np.array([[0.21, 0.37, 0.44], [0.68, 0.52, 0.71]])
    qs = np.array([1.0, -1.0])
    xt = np.array([[0.33, 0.81, 0.15]])
    return xs, qs, xt


def test_free_space_fourier_integral_by_quadrature():
    """Eq. (fourier_space_explicit_0P) for one source: (4 pi/(2 pi)^3) int e^{-k^2/4xi^2}/k^2
    e^{ik.r} d^3k = (2/pi) int_0^inf e^{-k^2/4xi^2} sin(kr)/(kr) dk."""
    xi, r = 5.0, 0.37
    val, _ = integrate.quad(lambda k: 2 / math.pi * math.exp(-k * k / (4 * xi * xi)) * math.sin(k * r) / (k * r),
                            0, 80 * xi, limit=400)
    phi, _ = E.fourier(0, np.zeros((1, 3)), np.ones(1), 1.0, xi, xt=np.array([[r, 0, 0]]))
    assert phi[0] == pytest.approx(val, rel=1e-10)


def test_doubly_periodic_fourier_integral_by_quadrature():
    """Eq. (fourier_space_explicit_2P): (4 pi/(2 pi L^2)) sum_k int dkappa
    e^{-(k^2+kappa^2)/4xi^2}/(k^2+kappa^2) e^{i(k.v + kappa z)}, each kappa-integral
    by adaptive quadrature, against the closed forms Eqs. (2pno0), (2p0)."""
    xs, qs, xt = _pair()
    L, xi = 1.0, 4.0
    nmax = E.kmax_n(xi, L, 1e-16)
    tot = 0.0
    for n1 in range(-nmax, nmax + 1):
        for n2 in range(-nmax, nmax + 1):
            k1, k2 = 2 * math.pi * n1 / L, 2 * math.pi * n2 / L
            kk = k1 * k1 + k2 * k2
            if kk > (2 * math.pi * nmax / L) ** 2:
                continue
            d = xt[0] - xs

            def f(kap):
                ph = k1 * d[:, 0] + k2 * d[:, 1]
                s = np.sum(qs * (np.cos(ph + kap * d[:, 2]) - (1.0 if kk == 0 else 0.0)))
                den = kk + kap * kap
                return math.exp(-den / (4 * xi * xi)) * s / den if den > 0 else \
                    -0.5 * np.sum(qs * d[:, 2] ** 2)   # kappa -> 0 limit when k = 0
            val, _ = integrate.quad(f, -14 * xi, 14 * xi, limit=400, points=[0.0], epsabs=1e-14)
            tot += val
    tot *= 4 * math.pi / (2 * math.pi * L * L)
    phi, _ = E.fourier(2, xs, qs, L, xi, xt=xt)
    assert phi[0] == pytest.approx(tot, rel=1e-9, abs=1e-11)


def test_singly_periodic_fourier_integral_by_quadrature():
    """Eq. (fourier_space_explicit_1P) with the kappa-plane integral in polar
    form, int d^2kappa e^{i kappa.w} f(|kappa|) = 2 pi int kappa J0(kappa rho) f dkappa."""
    xs, qs, xt = _pair()
    L, xi = 1.0, 4.0
    nmax = E.kmax_n(xi, L, 1e-16)
    d = xt[0] - xs
    rho = np.hypot(d[:, 1], d[:, 2])
    tot = 0.0
    for n1 in range(-nmax, nmax + 1):
        k1 = 2 * math.pi * n1 / L

        def f(kap):
            s = np.sum(qs * np.cos(k1 * d[:, 0]) * (sp.j0(kap * rho) - (1.0 if n1 == 0 else 0.0)))
            den = k1 * k1 + kap * kap
            return math.exp(-den / (4 * xi * xi)) * s * kap / den if den > 0 else 0.0
        val, _ = integrate.quad(f, 0, 14 * xi, limit=800, epsabs=1e-14)
        tot += 2 * math.pi * val
    tot *= 4 * math.pi / ((2 * math.pi) ** 2 * L)
    phi, _ = E.fourier(1, xs, qs, L, xi, xt=xt)
    assert phi[0] == pytest.approx(tot, rel=1e-8, abs=1e-11)


# ---------------------------------------------------------------- gradients

@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_fourier_gradient_matches_finite_differences(D):
    x, q = _system(30, 11)
    xt = wl.uniform_positions(5, 1.0, 99) * 0.8 + 0.1
    _, g = E.fourier(D, x, q, 1.0, 6.0, xt=xt)
    hstep = 1e-5
    for a in range(3):
        e = np.zeros(3)
        e[a] = hstep
        pp, _ = E.fourier(D, x, q, 1.0, 6.0, xt=xt + e)
        pm, _ = E.fourier(D, x, q, 1.0, 6.0, xt=xt - e)
        fd = (pp - pm) / (2 * hstep)
        assert np.allclose(g[:, a], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


def test_uniform_charges_give_the_printed_Q():
    """Q = sum q^2 ~ N/3 for q ~ U[-1, 1] (values printed in Secs. 5.2, 7.1, 7.2)."""
    g = GOLDEN["q_uniform_charges"]
    for n, qv in zip(g["N"], g["Q"]):
        qs = wl.uniform_charges(n, seed=1, neutral=False)
        assert float(qs @ qs) == pytest.approx(qv, rel=0.12 if n == 100 else 0.02)


# ---------------------------------------------------------------- Poisson's equation

@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_fourier_part_solves_poisson_with_screened_charges(D):
    """phi^F is the potential of the Gaussian-screened charges (Eq. split_rhs with
    gamma of Eq. gamma), periodised along the D periodic axes:
    -Laplacian phi^F = 4 pi sum_n sum_p q_n gamma(x - x_n - p).  The Laplacian is
    taken by a fourth-order central difference of the oracle's closed forms
    (k-sums, the 2P/1P zero modes, the 0P erf sum), so a dropped term or a
    wrong sign in any of them fails; the charges are neutral (3P drops k = 0)."""
    L, xi, h = 1.0, 4.0, 2e-3
    x = wl.uniform_positions(6, L, 91)
    q = wl.uniform_charges(6, 91)
    pts = np.array([[0.37, 0.52, 0.61], [0.81, 0.13, 0.45], [0.5, 0.5, 0.2]])
    # fourth-order stencil along each axis: -f(2h) + 16 f(h) - 30 f(0) + 16 f(-h) - f(-2h)
    offs = [(a, s) for a in range(3) for s in (-2, -1, 1, 2)]
    xt = [pts]
    for a, s in offs:
        d = np.zeros(3)
        d[a] = s * h
        xt.append(pts + d)
    phi, _ = E.fourier(D, x, q, L, xi, xt=np.concatenate(xt))
    phi = phi.reshape(len(xt), len(pts))
    c = {(-2,): -1.0, (-1,): 16.0, (1,): 16.0, (2,): -1.0}
    lap = np.zeros(len(pts))
    for i, (a, s) in enumerate(offs):
        lap += c[(s,)] * phi[1 + i]
    lap = (lap - 3 * 30.0 * phi[0]) / (12.0 * h * h)
    # screened charge density, images along the periodic axes
    rho = np.zeros(len(pts))
    rng = range(-3, 4)
    for p0 in (rng if D >= 1 else [0]):
        for p1 in (rng if D >= 2 else [0]):
            for p2 in (rng if D >= 3 else [0]):
                shift = np.array([p0, p1, p2]) * L
                r2 = ((pts[:, None, :] - x[None, :, :] - shift) ** 2).sum(-1)
                rho += (q[None, :] * (xi / math.sqrt(math.pi)) ** 3 * np.exp(-xi * xi * r2)).sum(1)
    np.testing.assert_allclose(-lap, 4 * math.pi * rho, rtol=1e-7, atol=1e-7 * np.abs(4 * math.pi * rho).max())
