"""Pins of the oracles in non-cubic boxes (Sec. 2: the domain need not be a
cube).  Oracle A is pinned by lattice identities and by the independence of
the total potential from the splitting parameter; oracle B (the discrete SE
algorithm with per-axis grids) is pinned against oracle A."""
import json
import os

import numpy as np
import pytest

from oracle import ewald as E
from oracle import params as prm
from oracle import se_discrete as S
from paper_1712_04732_gb300 import workloads as wl

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def _system(N, seed, box):
    x = wl.uniform_positions(N, 1.0, seed) * np.asarray(box)
    return x, wl.uniform_charges(N, seed)


@pytest.mark.parametrize("D,axis", [(3, 0), (3, 1), (3, 2), (2, 0), (2, 1), (1, 0)])
def test_replicated_cell_along_a_periodic_axis(D, axis):
    """Two copies of a periodic cell side by side along a periodic direction,
    in a box twice as long there, form the same infinite lattice, so every
    particle sees the same Fourier-space part."""
    box = np.array([1.0, 0.8, 1.2])
    x, q = _system(60, 3 + axis, box)
    shift = np.zeros(3)
    shift[axis] = box[axis]
    x2 = np.vstack([x, x + shift])
    q2 = np.concatenate([q, q])
    box2 = box.copy()
    box2[axis] *= 2
    p1, g1 = E.fourier(D, x, q, box, 5.0)
    p2, g2 = E.fourier(D, x2, q2, box2, 5.0, xt=x)
    assert _rel(p2, p1) < 1e-12
    assert _rel(g2, g1) < 1e-11


@pytest.mark.parametrize("D", [3, 2, 1])
def test_total_potential_independent_of_xi_in_a_box(D):
    """Eq. (potential_split): phi^R + phi^F + phi^self does not depend on xi."""
    box = np.array([1.0, 0.75, 1.5])
    x, q = _system(40, 11 + D, box)
    t1, g1 = E.total(D, x, q, box, 4.0, rc=8.0 / 4.0)
    t2, g2 = E.total(D, x, q, box, 6.0, rc=8.0 / 6.0)
    assert _rel(t1, t2) < 1e-10
    assert _rel(g1, g2) < 1e-9


def test_madelung_constant_in_a_supercell():
    """The NaCl cell stacked twice along z (box 1 x 1 x 2) gives the Madelung
    constant at every ion."""
    x, q = wl.nacl_cell(8, 1.0)
    x2 = np.vstack([x, x + np.array([0.0, 0.0, 1.0])])
    q2 = np.concatenate([q, q])
    a = 1.0 / 8
    phi, _ = E.total(3, x2, q2, (1.0, 1.0, 2.0), 14.0, rc=0.49)
    mad = -q2 * phi * a
    assert np.allclose(mad, GOLDEN["madelung_nacl"]["value"], rtol=0, atol=2e-10)


def test_box_grid_rules():
    Lv, h, Mv = prm.box_grid((1.0, 0.75, 1.25), 32)
    assert h == 1.0 / 32 and Mv == [32, 24, 40]
    with pytest.raises(ValueError):
        prm.box_grid((1.0, 0.7, 1.0), 32)                  # 22.4 h
    g = prm.grid(2, (1.0, 1.0, 1.0), 32, 8, "pkb")
    c = prm.grid(2, 1.0, 32, 8, "pkb")
    assert (g["Mt"], g["s0Mt"], g["sMt"], g["nl"], g["R"]) == (c["Mt"], c["s0Mt"], c["sMt"], c["nl"], c["R"])
    assert g["nI"][:2] == [c["nl"], c["nl"]]
    # the oversampled free grid holds the truncated kernel: s0 L~_i >= L~_i + R
    for D in (0, 1, 2):
        g = prm.grid(D, (1.0, 0.5, 2.0), 32, 8, "pkb")
        for i in range(D, 3):
            assert g["s0Mt_v"][i] * g["h"] >= g["Lt_v"][i] + g["R"] - 1e-12


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_se_oracle_in_a_box_matches_the_direct_sums(D):
    """Oracle B with per-axis grids against oracle A, PKB P = 14, in a
    1 x 0.75 x 1.25 box."""
    box = np.array([1.0, 0.75, 1.25])
    x, q = _system(80, 21 + D, box)
    o = S.SEOracle(D, box, 5.0, 32, 14, "pkb", eps_rel=1e-13)
    assert o.n[:D] == [32, 24, 40][:D]
    phi, g = o.potential(x, q, grad=True)
    pa, ga = E.fourier(D, x, q, box, 5.0)
    tol = 2e-8 if D == 0 else 1e-9
    assert _rel(phi, pa) < tol
    assert _rel(g, ga) < 20 * tol
    _, g2 = o.potential(x, q, grad=True, force_method=2)
    assert _rel(g2, ga) < 2 * tol
