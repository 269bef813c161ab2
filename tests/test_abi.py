"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every
function declared in include/se_gb300.h, and validates arguments on the host."""
import ctypes
import os
import re

import pytest

from oracle import params as prm
from paper_1712_04732_gb300 import _native as nat
from paper_1712_04732_gb300 import build as bld

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "se_gb300.h")


@pytest.fixture(scope="module")
def lib():
    bld.build()
    return nat.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(se_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "se_potential" in names and "se_force" in names and "se_plan_create" in names
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(nat.EXPORTS) == names


def test_status_names(lib):
    for code, name in nat.STATUS.items():
        assert lib.se_status_str(code).decode() == name


@pytest.mark.parametrize("D,M,P,xi,box", [
    (4, 32, 8, 8.0, 1.0),       # D out of range
    (3, 31, 8, 8.0, 1.0),       # M odd
    (3, 32, 7, 8.0, 1.0),       # P odd
    (3, 8, 10, 8.0, 1.0),       # P > M
    (3, 64, 18, 8.0, 1.0),      # P > 16
    (3, 32, 8, -1.0, 1.0),      # xi <= 0
    (3, 32, 8, 8.0, 0.0),       # empty box
])
def test_plan_create_rejects_bad_arguments(lib, D, M, P, xi, box):
    h = ctypes.c_void_p()
    b = (ctypes.c_double * 3)(box, box, box)
    st = lib.se_plan_create(ctypes.byref(h), b, D, xi, M, P, nat.SE_WIN_PKB, nat.SE_F32, None)
    assert st == 1 and not h.value
    assert lib.se_last_error()


@pytest.mark.parametrize("sides", [(1.0, 1.0, 1.03), (1.0, 1.0 + 1.0 / 32, 1.0), (1.0, 1.0, -1.0),
                                   (1.0, 0.125, 1.0)])
def test_plan_create_rejects_sides_off_the_grid(lib, sides):
    """Non-cubic boxes share h = L_x / M: every side must be an even multiple of
    h (33 h and 32.96 h are not), positive, and long enough for the support of
    a periodic direction (4 h < P = 8)."""
    h = ctypes.c_void_p()
    b = (ctypes.c_double * 3)(*sides)
    assert lib.se_plan_create(ctypes.byref(h), b, 3, 8.0, 32, 8, 1, 0, None) == 1
    assert not h.value


def test_calls_reject_null_plan(lib):
    assert lib.se_potential(None, 10, None, None, None, 0) == 1
    assert lib.se_force(None, 10, None, None, None, None, None, 0) == 1
    assert lib.se_plan_destroy(None) == 0


@pytest.mark.parametrize("eps_rel,xi,L,Q,win", [
    (1e-5, 8.0, 1.0, 3.32e4, "pkb"), (1e-10, 8.0, 1.0, 3.32e4, "pkb"), (1e-3, 3.0, 10.0, 3.32e4, "pkb"),
    (1.6e-8, 6.0, 5.0, 334.0, "gaussian"), (1e-12, 17.0, 3.0, 3.32e4, "pkb"), (1e-5, 2.0, 1.0, 100.0, "pkb"),
])
@pytest.mark.parametrize("D", [3, 0])
def test_parameter_rules_agree_with_the_oracle(lib, eps_rel, xi, L, Q, win, D):
    """se_params_from_tolerance (C++) and the oracle's Sec. 6 rules (Python) are
    written independently; they must give the same (M, P) for the absolute
    tolerance eps_rel B (the rules do not depend on D)."""
    M, P = ctypes.c_int(), ctypes.c_int()
    w = nat.SE_WIN_GAUSSIAN if win == "gaussian" else nat.SE_WIN_PKB
    box = (ctypes.c_double * 3)(L, L, L)
    assert lib.se_params_from_tolerance(eps_rel, xi, 0, Q, box, D, w, ctypes.byref(M), ctypes.byref(P)) == 0
    eps = eps_rel * prm.scale_B(Q, xi, L)
    assert (M.value, P.value) == prm.from_tolerance(eps, xi, L, Q, win)


def test_parameter_rules_take_Q_from_N(lib):
    """Q <= 0: Q = N / 3, the mean of sum q^2 for charges uniform in [-1, 1]."""
    M, P = ctypes.c_int(), ctypes.c_int()
    box = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    assert lib.se_params_from_tolerance(1e-6, 8.0, 30000, 0.0, box, 2, nat.SE_WIN_PKB,
                                        ctypes.byref(M), ctypes.byref(P)) == 0
    Q = 30000 / 3.0
    assert (M.value, P.value) == prm.from_tolerance(1e-6 * prm.scale_B(Q, 8.0, 1.0), 8.0, 1.0, Q, "pkb")


@pytest.mark.parametrize("sides", [(1.0, 0.75, 1.5), (1.0, 1.0, 2.0), (2.0, 1.0, 1.0), (1.0, 0.6, 1.2)])
def test_parameter_rules_fit_the_box(lib, sides):
    """A box that is not a cube: M is the smallest even value at or above the
    cube's rule for which every side is an even multiple of h = L_x / M (the
    oracle's box_grid accepts it, and it rejects every smaller even M)."""
    M, P = ctypes.c_int(), ctypes.c_int()
    box = (ctypes.c_double * 3)(*sides)
    Q, xi, eps_rel = 3000.0, 8.0, 1e-5
    assert lib.se_params_from_tolerance(eps_rel, xi, 0, Q, box, 3, nat.SE_WIN_PKB,
                                        ctypes.byref(M), ctypes.byref(P)) == 0
    M0, P0 = prm.from_tolerance(eps_rel * prm.scale_B(Q, xi, sides[0]), xi, sides[0], Q, "pkb")
    assert P.value == P0 and M.value >= M0 and M.value % 2 == 0
    prm.box_grid(sides, M.value)
    for m in range(M0 + (M0 & 1), M.value, 2):
        with pytest.raises(ValueError):
            prm.box_grid(sides, m)


@pytest.mark.parametrize("args", [
    dict(eps_rel=0.0), dict(eps_rel=1.5), dict(xi=-1.0), dict(D=4), dict(D=-1), dict(win=7),
    dict(Q=0.0, N=0), dict(box=(1.0, 0.0, 1.0)), dict(box=(1.0, 1.0 / 3.0 + 1e-7, 1.0)),
])
def test_parameter_rules_reject_bad_arguments(lib, args):
    a = dict(eps_rel=1e-5, xi=8.0, N=100, Q=30.0, box=(1.0, 1.0, 1.0), D=3, win=nat.SE_WIN_PKB)
    a.update(args)
    M, P = ctypes.c_int(), ctypes.c_int()
    box = (ctypes.c_double * 3)(*a["box"])
    assert lib.se_params_from_tolerance(a["eps_rel"], a["xi"], a["N"], a["Q"], box, a["D"], a["win"],
                                        ctypes.byref(M), ctypes.byref(P)) == 1
    assert lib.se_last_error()


def test_allocation_failure_hook_is_host_only(lib):
    """Arming and disarming the injected allocation failure touches no GPU."""
    assert lib.se_debug_fail_alloc(3) == 0
    assert lib.se_debug_fail_alloc(0) == 0


@pytest.mark.parametrize("field,value", [("fft_mode", 3), ("gather_mode", 5), ("force_method", 3)])
def test_plan_create_rejects_bad_options(lib, field, value):
    """Options out of range are refused on the host, before any device work:
    fft_mode 0 (default), 1 (cuFFT everywhere) or 2 (D = 1 line transforms);
    gather_mode up to 4; force_method 1 or 2."""
    o = nat.Opts()
    lib.se_opts_default(ctypes.byref(o))
    setattr(o, field, value)
    h = ctypes.c_void_p()
    b = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    assert lib.se_plan_create(ctypes.byref(h), b, 1, 8.0, 32, 8, nat.SE_WIN_PKB, nat.SE_F32, ctypes.byref(o)) == 1
    assert not h.value
    assert field.split("_")[0] in lib.se_last_error().decode()


def test_batch_form_flags_are_distinct_bits():
    flags = [nat.SE_BATCH_NO_AUTOTUNE, nat.SE_BATCH_BRANCHES, nat.SE_BATCH_FUSED, nat.SE_BATCH_LINES]
    assert flags == [1, 2, 4, 8]
    src = open(HEADER).read()
    for name, v in zip(("SE_BATCH_NO_AUTOTUNE", "SE_BATCH_BRANCHES", "SE_BATCH_FUSED", "SE_BATCH_LINES"), flags):
        assert re.search(rf"#define {name}\s+{v}u", src), name
