"""Real-space part on the GPU (se_real_space) against the direct sum of the
oracle, and the full Ewald potential on the GPU against the Madelung constant."""
import numpy as np
import pytest
import torch

from oracle import ewald as E
from paper_1712_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-5)])
@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_real_space_matches_direct_sum(D, dtype, tol):
    import paper_1712_04732_gb300 as se
    N, xi, rc = 3000, 14.0, 0.3
    x = wl.uniform_positions(N, 1.0, 50 + D)
    q = wl.uniform_charges(N, 50 + D)
    plan = se.Plan(D, 1.0, xi, 32, 6, "pkb", dtype=dtype)
    xt = torch.tensor(x, dtype=dtype, device="cuda")
    qt = torch.tensor(q, dtype=dtype, device="cuda")
    phi, F = plan.real_space(xt, qt, rc)
    torch.cuda.synchronize()
    pr, gr = E.real(D, x, q, 1.0, xi, rc)
    assert _rel(phi.double().cpu().numpy(), pr) < tol
    assert _rel(F.double().cpu().numpy(), -q[:, None] * gr) < 10 * tol


def test_real_space_single_cell_per_axis():
    """rc close to L/2: one cell per periodic axis, the images enumerated by shifts."""
    import paper_1712_04732_gb300 as se
    x = wl.uniform_positions(500, 1.0, 7)
    q = wl.uniform_charges(500, 7)
    plan = se.Plan(3, 1.0, 9.0, 24, 6, "pkb", dtype=torch.float64)
    phi, F = plan.real_space(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"), 0.49)
    pr, gr = E.real(3, x, q, 1.0, 9.0, 0.49)
    assert _rel(phi.cpu().numpy(), pr) < 1e-12


def test_full_ewald_potential_gives_the_madelung_constant():
    """NaCl cell: GPU Fourier part (PKB P = 16) + GPU real-space part + self term."""
    import paper_1712_04732_gb300 as se
    x, q = wl.nacl_cell(8, 1.0)
    plan = se.Plan(3, 1.0, 14.0, 64, 16, "pkb", dtype=torch.float64)
    phi, F = plan.total(torch.tensor(x, device="cuda"), torch.tensor(q, device="cuda"), 0.49)
    torch.cuda.synchronize()
    mad = -(phi.cpu().numpy() * q) / 8.0
    assert np.allclose(mad, 1.7475645946, atol=1e-9)
    assert np.abs(F.cpu().numpy()).max() < 1e-8
