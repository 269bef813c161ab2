"""Batched evaluation of independent systems (se_batch_*): every system of the
batch matches a standalone plan with the same parameters, the CUDA-graph form
matches the per-system launches, and the Sec. 6 parameter choice meets the
requested tolerance against the direct sums."""
import numpy as np
import pytest
import torch

from oracle import ewald as E
from paper_1712_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def _systems(n_sys=10, seed=3):
    sysl = wl.batch_systems(n_sys, seed=seed, n_min=400, n_max=6000)
    specs = [(len(q), D, 1.0, 8.0 * (len(q) / 1e4) ** (1.0 / 3.0)) for x, q, D in sysl]
    x = np.concatenate([s[0] for s in sysl])
    q = np.concatenate([s[1] for s in sysl])
    return sysl, specs, x, q


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_standalone_plans(autotune):
    import paper_1712_04732_gb300 as se
    sysl, specs, x, q = _systems()
    b = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, autotune=autotune)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    qt = torch.tensor(q, dtype=torch.float32, device="cuda")
    F, phi, En = b.force(xt, qt)
    F2, phi2, En2 = b.force(xt, qt)                 # graph replay
    Fe, phie, Ene = b.force(xt, qt, each=True)      # one se_force per system
    torch.cuda.synchronize()
    assert _rel(phi2.cpu().numpy(), phi.cpu().numpy()) < 1e-6
    assert _rel(F2.cpu().numpy(), F.cpu().numpy()) < 1e-6
    off = 0
    for i, (xs, qs, D) in enumerate(sysl):
        n = len(qs)
        info = b.system_info(i)
        plan = se.Plan(D, 1.0, specs[i][3], info["M"], info["P"], "pkb", dtype=torch.float32)
        Fp, pp, Ep = plan.force(xt[off:off + n], qt[off:off + n], energy=True)
        torch.cuda.synchronize()
        assert _rel(phi[off:off + n].cpu().numpy(), pp.cpu().numpy()) < 1e-5
        assert _rel(F[off:off + n].cpu().numpy(), Fp.cpu().numpy()) < 1e-5
        assert _rel(phie[off:off + n].cpu().numpy(), pp.cpu().numpy()) < 1e-5
        assert En[i].item() == pytest.approx(Ep.item(), rel=1e-5)
        off += n
        plan.close()
    b.close()


def test_batch_parameters_meet_the_tolerance():
    """M_i, P_i from Sec. 6 for eps_rms = 1e-5 B_i: the potential of each system
    against the direct sums (3P k-sum, 2P closed forms)."""
    import paper_1712_04732_gb300 as se
    sysl, specs, x, q = _systems(6, seed=9)
    b = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, autotune=False)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    qt = torch.tensor(q, dtype=torch.float32, device="cuda")
    F, phi, _ = b.force(xt, qt)
    torch.cuda.synchronize()
    off = 0
    for i, (xs, qs, D) in enumerate(sysl):
        n = len(qs)
        idx = np.arange(0, n, max(1, n // 200))
        pa, _ = E.fourier(D, xs, qs, 1.0, specs[i][3], xt=xs[idx])
        assert _rel(phi[off:off + n].cpu().numpy()[idx], pa) < 5e-5
        off += n
    b.close()
