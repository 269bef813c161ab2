"""Pins of oracle B (the discrete SE algorithm), of the window functions and of
the parameter rules, against facts fixed outside them."""
import json
import math
import os

import numpy as np
import pytest
import scipy.special as sp
from scipy import integrate

from oracle import ewald as E
from oracle import params as prm
from oracle import se_discrete as S
from oracle import windows as W
from paper_1712_04732_gb300 import workloads as wl

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _system(N=300, seed=2):
    return wl.uniform_positions(N, 1.0, seed), wl.uniform_charges(N, seed)


def _rel(a, b):
    return float(np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(b ** 2)))


# ------------------------------------------------------------- parameter rules

def test_kp_fourier_estimate_printed_value():
    g = GOLDEN["kp_fourier_e5"]
    assert prm.kp_fourier(g["Q"], g["xi"], g["L"], g["M"]) == pytest.approx(g["value"], rel=0.01)


def test_kp_relative_truncation_printed_values():
    """Fig. error_pollution caption: relative truncation errors (abs / B)."""
    g = GOLDEN["kp_relative_pollution"]
    B = prm.scale_B(g["Q"], g["xi"], g["L"])
    for M, v in zip(g["M"], g["values"]):
        assert prm.kp_fourier(g["Q"], g["xi"], g["L"], M) / B == pytest.approx(v, rel=0.10)


def test_kp_inversions_round_trip():
    """Eqs. (KP_rc), (KP_kinf) invert Eqs. (KP_real_space), (KP_fourier_space)."""
    Q, xi, L = 3.32e4, 8.0, 1.0
    for eps in (1e-3, 1e-8, 1e-14):
        rc = prm.kp_rc(Q, xi, L, eps)
        assert prm.kp_real(Q, xi, L, rc) == pytest.approx(eps, rel=1e-9)
        kinf = prm.kp_kinf(Q, xi, L, eps)
        assert prm.kp_fourier(Q, xi, L, 2 * kinf) == pytest.approx(eps, rel=1e-9)


def test_lambda_table_matches_paper():
    for win in ("gaussian", "pkb"):
        for d, v in GOLDEN["lambda_table"][win].items():
            assert prm.LAMBDA[win][int(d)] == v


def test_degree_rule():
    """nu = min(P/2 + 2, 9) (Sec. 6)."""
    assert [prm.degree(P) for P in (4, 6, 8, 10, 12, 14, 16)] == [4, 5, 6, 7, 8, 9, 9]


# ------------------------------------------------------------- windows

@pytest.mark.parametrize("k", [0.0, 3.0, 17.0, 40.0])
def test_kaiser_transform_by_quadrature(k):
    """Eq. (kaiser_ft) against int_{-w}^{w} W_KB(x) cos(kx) dx."""
    w, beta = 0.2, 15.0
    val, _ = integrate.quad(lambda x: W.kaiser(x, w, beta) * math.cos(k * x), -w, w, limit=200,
                            epsabs=1e-15, epsrel=1e-13)
    assert W.kaiser_hat(k, w, beta) == pytest.approx(val, rel=1e-10, abs=1e-14)


def test_kaiser_transform_past_the_turning_point():
    w, beta, k = 0.2, 3.0, 40.0           # k w > beta: oscillatory branch
    val, _ = integrate.quad(lambda x: W.kaiser(x, w, beta) * math.cos(k * x), -w, w, limit=200)
    assert W.kaiser_hat(k, w, beta) == pytest.approx(val, rel=1e-9)


def test_gaussian_untruncated_transform():
    w, alpha = 0.2, 11.4
    for k in (0.0, 9.0, 30.0):
        val, _ = integrate.quad(lambda x: math.exp(-alpha * (x / w) ** 2) * math.cos(k * x), -np.inf, np.inf)
        assert W.gaussian_hat(k, w, alpha) == pytest.approx(val, rel=1e-10)


def test_window_derivatives_by_finite_differences():
    w = 0.1
    x = np.linspace(-0.099, 0.099, 37)
    for f, df, s in ((W.gaussian, W.gaussian_dx, 11.0), (W.kaiser, W.kaiser_dx, 20.0)):
        fd = (f(x + 1e-7, w, s) - f(x - 1e-7, w, s)) / 2e-7
        assert np.allclose(df(x, w, s), fd, rtol=1e-6, atol=1e-6)


def test_pkb_reproduces_polynomials_exactly():
    """The interpolation at nu + 1 Chebyshev points is exact for degree-nu targets."""
    P, h, nu = 6, 0.05, 5
    poly = np.polynomial.Polynomial([0.3, -1.2, 0.7, 2.0, -0.4, 0.9])
    p = W.PKB(P, h, 15.0, nu, target=poly)
    x = np.linspace(-P * h / 2, P * h / 2 * 0.999, 101)
    assert np.allclose(p(x), poly(x), rtol=1e-11, atol=1e-12)
    assert np.allclose(p.dx(x), poly.deriv()(x), rtol=1e-9, atol=1e-10)


def test_pkb_stencil_evaluation_matches_the_piecewise_polynomial():
    """Evaluating point k of the support in subinterval P-1-k at the common offset
    xbar = 2 frac - 1 (Sec. 4.1) agrees with evaluating the piecewise polynomial at
    the distance x_m - x_j = (frac + P/2 - 1 - k) h away from the joins."""
    P, h, nu = 8, 1.0 / 24, 6
    p = W.PKB(P, h, 2.5 * P, nu)
    frac = np.linspace(0.01, 0.99, 23)[:, None]
    k = np.arange(P)[None, :]
    assert np.allclose(p.stencil(frac, k), p((frac + P / 2 - 1 - k) * h), rtol=1e-13, atol=1e-15)
    assert np.allclose(p.stencil_dx(frac, k), p.dx((frac + P / 2 - 1 - k) * h), rtol=1e-11, atol=1e-12)


def test_pkb_vandermonde_condition_number_law():
    """Sec. 4.1: cond ~ 0.6 * 10^(0.38 nu), 1.6e3 at nu = 9."""
    g = GOLDEN["vandermonde_condition"]
    for nu in range(4, 13):
        c = W.PKB(8, 0.1, 20.0, nu).cond()
        law = g["law_coeff"] * 10 ** (g["law_base_exp"] * nu)
        assert 0.5 * law < c < 2.0 * law
    assert W.PKB(8, 0.1, 20.0, g["nu"]).cond() == pytest.approx(g["value_at_nu"], rel=0.1)


def test_pkb_fit_error_falls_with_degree():
    P, h = 8, 1.0 / 32
    beta = 2.5 * P
    x = np.linspace(-P * h / 2, P * h / 2, 2001)[:-1]
    errs = [np.abs(W.PKB(P, h, beta, nu)(x) - W.kaiser(x, P * h / 2, beta)).max() for nu in (3, 5, 7, 9)]
    assert all(b < a / 10 for a, b in zip(errs, errs[1:]))


# ------------------------------------------------------------- Green's functions

def test_green_functions_limits_at_zero():
    """The k -> 0 values of Eqs. (G_hat_0d), (G_hat_1d), (G_hat_2d) and App. A."""
    R = 1.7
    tiny = 1e-5
    assert S.green(0, R, 0.0, tiny) == pytest.approx(R * R / 2, rel=1e-8)
    # 1 - J0 cancels at small kappa; kappa = 1e-3 keeps 6 digits and a (R kappa)^2 bias
    assert S.green(1, R, 0.0, 1e-3) == pytest.approx(R * R / 4 * (1 - 2 * math.log(R)), rel=2e-5)
    assert S.green(2, R, 0.0, 1e-3) == pytest.approx(-R * R / 2, rel=2e-5)
    assert S.green(3, R, 0.0, 0.0) == 0.0


@pytest.mark.parametrize("kap", [0.5, 3.0, 11.0, 37.0])
def test_green_functions_by_quadrature_of_truncated_kernels(kap):
    """Transforms of the truncated free-space Green's functions (Sec. 3.1, App. A):
    1D G = -|z|/2, 2D G = -log(r)/(2 pi), 3D G = 1/(4 pi r), each cut at R."""
    R = 1.3
    g2, _ = integrate.quad(lambda z: -abs(z) / 2 * math.cos(kap * z), -R, R, limit=400)
    assert S.green(2, R, 0.0, kap) == pytest.approx(g2, rel=1e-9, abs=1e-12)
    g1, _ = integrate.quad(lambda r: -math.log(r) / (2 * math.pi) * sp.j0(kap * r) * 2 * math.pi * r, 0, R, limit=400)
    assert S.green(1, R, 0.0, kap) == pytest.approx(g1, rel=1e-9, abs=1e-12)
    g0, _ = integrate.quad(lambda r: 1 / (4 * math.pi * r) * math.sin(kap * r) / (kap * r) * 4 * math.pi * r * r,
                           0, R, limit=400)
    assert S.green(0, R, 0.0, kap) == pytest.approx(g0, rel=1e-9, abs=1e-12)


# ------------------------------------------------------------- the discrete algorithm

@pytest.mark.parametrize("D", [3, 2, 1, 0])
@pytest.mark.parametrize("window", ["gaussian", "pkb", "kb"])
def test_se_oracle_follows_the_error_estimates(D, window):
    """Sec. 5.2: relative error about 2 e^{-(pi/2) P c} (Gaussian) and
    10 e^{-2.5 P} (PKB/KB) once other errors are negligible (M = 32, xi = 8, P = 8)."""
    x, q = _system()
    pa, ga = E.fourier(D, x, q, 1.0, 8.0)
    o = S.SEOracle(D, 1.0, 8.0, 32, 8, window)
    pb, gb = o.potential(x, q, grad=True)
    est = prm.approx_error("gaussian" if window == "gaussian" else "pkb", 8, 1.0)
    err = _rel(pb, pa)
    assert est / 10 < err < 2 * est
    assert _rel(gb, ga) < 100 * est           # method 1 forces lose about one P-step


@pytest.mark.parametrize("D,M,lam", [(3, 48, None), (2, 48, None), (1, 48, None), (0, 48, 2.5)])
def test_se_oracle_reaches_machine_precision(D, M, lam):
    """PKB with P = 16 (Sec. 7.1: machine precision from P ~ 14)."""
    x, q = _system(200, 4)
    pa, ga = E.fourier(D, x, q, 1.0, 8.0)
    o = S.SEOracle(D, 1.0, 8.0, M, 16, "pkb", eps_rel=1e-16, lam=lam)
    pb, gb = o.potential(x, q, grad=True)
    assert _rel(pb, pa) < 5e-14
    assert _rel(gb, ga) < 5e-12


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_se_operator_is_symmetric(D):
    """phi = A q with A = S^T G S symmetric (G real and even in k):
    q2 . A q1 = q1 . A q2 for two charge sets on the same positions."""
    x, q1 = _system(120, 6)
    q2 = wl.uniform_charges(120, 77)
    o = S.SEOracle(D, 1.0, 6.0, 24, 6, "pkb")
    p1, _ = o.potential(x, q1)
    p2, _ = o.potential(x, q2)
    assert float(q2 @ p1) == pytest.approx(float(q1 @ p2), rel=1e-12)


@pytest.mark.parametrize("D", [3, 1])
def test_se_oracle_gradient_is_derivative_of_potential(D):
    """The gather gradient with the exact derivative of the piecewise polynomial
    equals the finite-difference derivative of the gathered potential (targets
    away from subinterval joins, where the PKB may jump)."""
    x, q = _system(100, 8)
    o = S.SEOracle(D, 1.0, 6.0, 24, 8, "pkb")
    H = o.grid_charges(x, q)
    Ht = o.convolve(H)
    xt = wl.uniform_positions(40, 1.0, 31) * 0.9 + 0.05
    frac = (xt + np.array(o.off)) / o.h % 1.0
    keep = np.all((frac > 0.01) & (frac < 0.99), axis=1)
    xt = xt[keep]
    _, g = o.gather(Ht, xt, grad=True)
    st = 1e-7
    for a in range(3):
        e = np.zeros(3)
        e[a] = st
        fd = (o.gather(Ht, xt + e)[0] - o.gather(Ht, xt - e)[0]) / (2 * st)
        assert np.allclose(g[:, a], fd, rtol=1e-5, atol=1e-5 * np.abs(fd).max())


def test_se_oracle_linear_and_translation_covariant_3p():
    """3P: shifting all particles by a whole number of grid cells leaves phi
    unchanged (the discrete method is exactly shift-invariant on its grid)."""
    x, q = _system(150, 12)
    o = S.SEOracle(3, 1.0, 7.0, 24, 6, "pkb")
    p0, _ = o.potential(x, q)
    p1, _ = o.potential((x + 5 * o.h) % 1.0, q)
    assert np.allclose(p0, p1, rtol=1e-12, atol=1e-12 * np.abs(p0).max())


# ------------------------------------------------------ forces by method 2 (Sec. 7.2)

def test_ik_factor_differentiates_pure_modes():
    """i k on an n-point grid: d/dx of sin(2 pi m x / L) is (2 pi m / L) cos(2 pi m x / L)
    for |m| < n/2; the Nyquist mode (sampled as cos(pi j)) has no derivative."""
    n, L = 12, 0.75
    d = L / n
    xs = np.arange(n) * d
    for m in range(1, n // 2):
        f = np.sin(2 * np.pi * m * xs / L)
        df = np.fft.ifft(S.ik_factor(n, d) * np.fft.fft(f))
        np.testing.assert_allclose(df.real, 2 * np.pi * m / L * np.cos(2 * np.pi * m * xs / L), atol=1e-12)
        assert np.max(np.abs(df.imag)) < 1e-12
    nyq = np.cos(np.pi * np.arange(n))
    assert np.max(np.abs(np.fft.ifft(S.ik_factor(n, d) * np.fft.fft(nyq)))) < 1e-14


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_method2_force_matches_continuum(D):
    """Method 2 (i k in the scaling) against oracle A's analytic gradients."""
    x, q = _system(N=80, seed=5)
    o = S.SEOracle(D, 1.0, 4.0, 32, 16, "pkb")
    _, g2 = o.potential(x, q, grad=True, force_method=2)
    _, ga = E.fourier(D, x, q, 1.0, 4.0)
    assert _rel(g2, ga) < (1e-6 if D == 0 else 1e-9)


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_method2_conserves_momentum(D):
    """With the same window for gridding and gathering and an odd, purely
    imaginary multiplier, sum_m F_m = -sum_j H_j (dH~)_j vanishes: the operator
    of i k sigma is antisymmetric.  Method 1 has no such identity."""
    x, q = _system(N=100, seed=6)
    o = S.SEOracle(D, 1.0, 6.0, 24, 6, "pkb")
    _, g2 = o.potential(x, q, grad=True, force_method=2)
    _, g1 = o.potential(x, q, grad=True, force_method=1)
    F2, F1 = -q[:, None] * g2, -q[:, None] * g1
    assert np.max(np.abs(F2.sum(axis=0))) < 1e-13 * np.abs(F2).sum()
    assert np.max(np.abs(F1.sum(axis=0))) > 1e-9 * np.abs(F1).sum()


def test_method2_error_tracks_the_potential_and_method1_needs_two_more_points():
    """Sec. 7.2 (Fig. force, 3P, PKB, xi = 8, M = 64): method 2 has the error
    curve of the potential; method 1 is offset and needs P + 2 to reach the
    error of method 2 at P."""
    x, q = _system(N=200, seed=2)
    _, ga = E.fourier(3, x, q, 1.0, 8.0)
    pa, _ = E.fourier(3, x, q, 1.0, 8.0)
    err = {}
    for P in (4, 6, 8, 10):
        o = S.SEOracle(3, 1.0, 8.0, 64, P, "pkb")
        phi, g1 = o.potential(x, q, grad=True, force_method=1)
        _, g2 = o.potential(x, q, grad=True, force_method=2)
        err[P] = (_rel(phi, pa), _rel(g1, ga), _rel(g2, ga))
    for P in (4, 6, 8, 10):
        ephi, e1, e2 = err[P]
        assert e2 < 2.0 * ephi and ephi < 2.0 * e2
        assert e1 > 10.0 * e2
    for P in (4, 6, 8):
        assert err[P + 2][1] < err[P][2]
