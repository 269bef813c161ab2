"""Pins of the parameter selection of Sec. 6 (oracle/params.py): the grid size
from Eq. (KP_kinf), the support from the approximation-error estimates of
Sec. 5.2, the error-pollution correction of Eq. (error_pollution), and the
AFT sizes of Eqs. (estimate-s), (estimate-nl).

Each rule is checked against what it promises, measured with the discrete SE
algorithm (oracle B) against the direct Ewald sums (oracle A): parameters from
a tolerance meet that tolerance, the pollution case of Fig. error_pollution
misses it without the correction and meets it with it, and the AFT upsampling
rule reaches the requested error while one mode less in the set I does not.
The AFT sizes of the 2P and 1P workloads are also compared with the values
worked out by hand from Sec. 6."""
import json
import math
import os

import numpy as np
import pytest

from oracle import ewald as E
from oracle import params as prm
from oracle import se_discrete as S
from paper_1712_04732_gb300 import workloads as wl

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _rms(a):
    return float(np.sqrt(np.mean(np.asarray(a) ** 2)))


def _abs_err(D, L, xi, M, P, win, x, q, idx, pa, eps_rel=1e-10):
    o = S.SEOracle(D, L, xi, M, P, win, eps_rel=eps_rel)
    pb, _ = o.potential(x, q, xt=x[idx])
    return _rms(pb - pa)


@pytest.mark.parametrize("D", [3, 2, 1, 0])
@pytest.mark.parametrize("window", ["pkb", "gaussian"])
@pytest.mark.parametrize("eps_rel", [1e-5, 1e-8])
def test_from_tolerance_meets_the_tolerance(D, window, eps_rel):
    """Sec. 6: (M, P) from eps = eps_rel B reach an rms error <= eps against the
    continuum sums (the AFT parameters for the same eps_rel)."""
    N, L, xi = 300, 1.0, 8.0
    x, q = wl.uniform_positions(N, L, 5), wl.uniform_charges(N, 5)
    Q = prm.q_sum_sq(q)
    B = prm.scale_B(Q, xi, L)
    idx = np.arange(0, N, 3)
    pa, _ = E.fourier(D, x, q, L, xi, xt=x[idx])
    M, P = prm.from_tolerance(eps_rel * B, xi, L, Q, window)
    err = _abs_err(D, L, xi, M, P, window, x, q, idx, pa, eps_rel=eps_rel)
    assert err <= eps_rel * B


def _pollution_case():
    g = GOLDEN["kp_relative_pollution"]
    N, L, xi = 1000, g["L"], g["xi"]
    x, q = wl.uniform_positions(N, L, 11), wl.uniform_charges(N, 11)
    Q = prm.q_sum_sq(q)
    # the tolerance at which Eq. (KP_kinf) gives M = 70, the first grid of the figure
    eps = prm.kp_fourier(Q, xi, L, g["M"][0]) * 1.0001
    idx = np.arange(0, N, 5)
    pa, _ = E.fourier(3, x, q, L, xi, xt=x[idx])
    return N, L, xi, x, q, Q, eps, idx, pa


@pytest.fixture(scope="module")
def pollution_case():
    return _pollution_case()


@pytest.mark.parametrize("window", ["pkb", "gaussian"])
def test_pollution_correction_fig_error_pollution(pollution_case, window):
    """Fig. error_pollution (3P, N = 1000, L = 5, xi = 6, M = 70): the support
    from the approximation estimate exceeds f_W(M / (xi L)), and with those
    (M, P) the error misses the tolerance several times over; with M raised by
    5 % and P + 4 (Sec. 6) it meets it (within 2x, the spread of the estimates
    in Fig. AB_test)."""
    N, L, xi, x, q, Q, eps, idx, pa = pollution_case
    B = prm.scale_B(Q, xi, L)
    M0 = 2 * math.ceil(prm.kp_kinf(Q, xi, L, eps))
    assert M0 == 70
    if window == "gaussian":
        P0 = prm.even_up(math.log(2.0 * B / eps) / ((math.pi / 2.0) * math.sqrt(prm.GAUSS_C2)))
    else:
        P0 = prm.even_up(math.log(10.0 * B / eps) / 2.5)
    assert P0 > prm.pollution_limit(window, M0 / (xi * L))
    M1, P1 = prm.from_tolerance(eps, xi, L, Q, window)
    assert (M1, P1) == (prm.even_up(1.05 * M0), P0 + 4)
    e_uncorrected = _abs_err(3, L, xi, M0, P0, window, x, q, idx, pa)
    e_corrected = _abs_err(3, L, xi, M1, P1, window, x, q, idx, pa)
    assert e_uncorrected > 5.0 * eps
    assert e_corrected < 2.0 * eps


def test_pollution_rule_not_applied_below_the_limit():
    """xi = 3, L = 1, eps = 1e-5 B: P = 6 from the estimate is below f_W(M /
    (xi L)), so (M, P) stay as the estimates give them, and they meet the
    tolerance in 3P."""
    N, L, xi = 300, 1.0, 3.0
    x, q = wl.uniform_positions(N, L, 5), wl.uniform_charges(N, 5)
    Q = prm.q_sum_sq(q)
    B = prm.scale_B(Q, xi, L)
    eps = 1e-5 * B
    M0 = 2 * math.ceil(prm.kp_kinf(Q, xi, L, eps))
    M, P = prm.from_tolerance(eps, xi, L, Q, "pkb")
    assert M == M0 and P <= prm.pollution_limit("pkb", M / (xi * L))
    idx = np.arange(0, N, 3)
    pa, _ = E.fourier(3, x, q, L, xi, xt=x[idx])
    assert _abs_err(3, L, xi, M, P, "pkb", x, q, idx, pa) <= eps


def test_aft_sizes_of_the_workloads():
    """Sec. 6 worked out by hand for the slab (D = 2, M = 64, PKB P = 6) and the
    wire (D = 1, M = 128, PKB P = 8) at eps_rel = 1e-5, and the free-space grid
    (D = 0, M = 48, P = 8): (M~, s M~, n_l, s0 M~)."""
    g = prm.grid(2, 1.0, 64, 6, "pkb", eps_rel=1e-5)
    assert (g["Mt"], g["sMt"], g["nl"], g["s0Mt"]) == (80, 176, 6, 160)
    g = prm.grid(1, 1.0, 128, 8, "pkb", eps_rel=1e-5)
    assert (g["Mt"], g["sMt"], g["nl"], g["s0Mt"]) == (148, 350, 11, 370)
    g = prm.grid(0, 1.0, 48, 8, "pkb")
    assert (g["Mt"], g["sMt"], g["s0Mt"]) == (60, 120, 168)


@pytest.mark.parametrize("D", [2, 1])
@pytest.mark.parametrize("eps_rel", [1e-10, 1e-8, 1e-6])
def test_aft_upsampling_reaches_the_tolerance(D, eps_rel):
    """Eqs. (estimate-s), (estimate-nl) with M = 40, PKB P = 16 (every other
    error far below eps_rel): the relative error against the continuum sums is
    within 2 eps_rel."""
    N, L, xi = 300, 1.0, 8.0
    x, q = wl.uniform_positions(N, L, 5), wl.uniform_charges(N, 5)
    idx = np.arange(0, N, 3)
    pa, _ = E.fourier(D, x, q, L, xi, xt=x[idx])
    err = _abs_err(D, L, xi, 40, 16, "pkb", x, q, idx, pa, eps_rel=eps_rel) / _rms(pa)
    assert err <= 2.0 * eps_rel


@pytest.mark.parametrize("D", [2, 1])
def test_aft_set_I_is_not_oversized(D):
    """At eps_rel = 1e-8 (M = 40, P = 16) the set I of Eq. (estimate-nl) is as
    small as it can be: one mode less along each periodic direction misses the
    tolerance by more than 10x."""
    N, L, xi = 300, 1.0, 8.0
    x, q = wl.uniform_positions(N, L, 5), wl.uniform_charges(N, 5)
    idx = np.arange(0, N, 3)
    pa, _ = E.fourier(D, x, q, L, xi, xt=x[idx])
    o = S.SEOracle(D, L, xi, 40, 16, "pkb", eps_rel=1e-8)
    nl = o.g["nl"]
    o2 = S.SEOracle(D, L, xi, 40, 16, "pkb", eps_rel=1e-8, nl=nl - 1)
    pb, _ = o2.potential(x, q, xt=x[idx])
    assert _rms(pb - pa) / _rms(pa) > 10 * 1e-8
