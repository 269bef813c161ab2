"""Non-cubic boxes (Sec. 2: the domain need not be a cube) on the GPU path:
parity with the oracle's per-axis discrete algorithm, accuracy against the
direct sums, the real-space part and the Madelung constant of a supercell."""
import numpy as np
import pytest
import torch

from oracle import ewald as E
from oracle import se_discrete as S
from paper_1712_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {torch.float64: (1e-11, 1e-10), torch.float32: (2e-6, 1e-5)}   # (phi, F) relative rms
BOX = (1.0, 0.75, 1.25)


def _se():
    import paper_1712_04732_gb300 as se
    return se


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def _system(N, seed, box):
    return wl.uniform_positions(N, 1.0, seed) * np.asarray(box), wl.uniform_charges(N, seed)


def _oracle_for(plan, **kw):
    info = plan.info()
    o = S.SEOracle(plan.D, plan.box, plan.xi, plan.M, plan.P, plan.window, s_mt=list(info["s_mt_v"]),
                   nl=list(info["n_I"]), **kw)
    assert o.n == list(info["grid"])
    if plan.D < 3:
        assert list(o.g["s0Mt_v"][plan.D:]) == list(info["s0_mt_v"][plan.D:])
    return o


def _run(plan, x, q):
    xt = torch.tensor(x, dtype=plan.dtype, device=plan.device)
    qt = torch.tensor(q, dtype=plan.dtype, device=plan.device)
    F, phi, En = plan.force(xt, qt, energy=True)
    torch.cuda.synchronize()
    return F.double().cpu().numpy(), phi.double().cpu().numpy(), En.item()


@pytest.mark.parametrize("force_method", [1, 2])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("window", ["pkb", "gaussian"])
@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_box_matches_discrete_oracle(D, window, dtype, force_method):
    se = _se()
    x, q = _system(800, 71 + D, BOX)
    plan = se.Plan(D, BOX, 6.0, 24, 8, window, dtype=dtype, force_method=force_method)
    assert plan.info()["M_v"] == (24, 18, 30)
    F, phi, En = _run(plan, x, q)
    pb, gb = _oracle_for(plan).potential(x, q, grad=True, force_method=force_method)
    tp, tf = TOL[dtype]
    assert _rel(phi, pb) < tp
    assert _rel(F, -q[:, None] * gb) < tf
    assert En == pytest.approx(0.5 * float(q @ pb), rel=10 * tp)


@pytest.mark.parametrize("force_method", [1, 2])
def test_free_space_box_with_the_column_stage(force_method):
    """D = 0 in a 1 x 0.75 x 1.5 box with M~_z = 32: the fused z-column kernel."""
    se = _se()
    box = (1.0, 0.75, 1.5)
    x, q = _system(700, 5, box)
    plan = se.Plan(0, box, 6.0, 16, 6, "pkb", dtype=torch.float64, force_method=force_method)
    info = plan.info()
    assert info["column_fft"] == 1 and info["Mt_v"] == (24, 20, 32)
    F, phi, _ = _run(plan, x, q)
    pb, gb = _oracle_for(plan).potential(x, q, grad=True, force_method=force_method)
    assert _rel(phi, pb) < 1e-11
    assert _rel(F, -q[:, None] * gb) < 1e-10


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_box_accuracy_against_direct_sums(D):
    """FP64, PKB P = 14, 1 x 0.75 x 1.25 box: the GPU result against oracle A."""
    se = _se()
    x, q = _system(400, 81 + D, BOX)
    plan = se.Plan(D, BOX, 5.0, 32, 14, "pkb", dtype=torch.float64, aft_eps=1e-13)
    F, phi, _ = _run(plan, x, q)
    pa, ga = E.fourier(D, x, q, BOX, 5.0)
    tol = 2e-8 if D == 0 else 1e-9
    assert _rel(phi, pa) < tol
    assert _rel(F, -q[:, None] * ga) < 20 * tol


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_box_real_space(D):
    se = _se()
    x, q = _system(2000, 91 + D, BOX)
    plan = se.Plan(D, BOX, 14.0, 24, 6, "pkb", dtype=torch.float64)
    phi, F = plan.real_space(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"), 0.3)
    torch.cuda.synchronize()
    pr, gr = E.real(D, x, q, BOX, 14.0, 0.3)
    assert _rel(phi.cpu().numpy(), pr) < 1e-12
    assert _rel(F.cpu().numpy(), -q[:, None] * gr) < 1e-11


def test_madelung_constant_in_a_supercell():
    """NaCl cell stacked twice along z (box 1 x 1 x 2): GPU Fourier part +
    real-space part + self term give the Madelung constant at every ion."""
    se = _se()
    x, q = wl.nacl_cell(8, 1.0)
    x2 = np.vstack([x, x + np.array([0.0, 0.0, 1.0])])
    q2 = np.concatenate([q, q])
    plan = se.Plan(3, (1.0, 1.0, 2.0), 14.0, 64, 16, "pkb", dtype=torch.float64)
    phi, F = plan.total(torch.tensor(x2, device="cuda"), torch.tensor(q2, device="cuda"), 0.49)
    torch.cuda.synchronize()
    mad = -(phi.cpu().numpy() * q2) / 8.0
    assert np.allclose(mad, 1.7475645946, atol=1e-9)
    assert np.abs(F.cpu().numpy()).max() < 1e-8
