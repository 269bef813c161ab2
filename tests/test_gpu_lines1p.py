"""D = 1 plans with the free-direction transforms as line transforms
(se_opts.fft_mode = 2): the padded transforms of the zero mode and the set I
(Alg. 1, Alg. 2) and the scaling run as three line-transform launches.  The
results must match oracle B (the same discrete algorithm) and the cuFFT path of
the same plan to rounding."""
import numpy as np
import pytest
import torch

from oracle import se_discrete as S
from paper_1712_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def _run(plan, x, q):
    xt = torch.tensor(x, dtype=plan.dtype, device=plan.device)
    qt = torch.tensor(q, dtype=plan.dtype, device=plan.device)
    F, phi, En = plan.force(xt, qt, energy=True)
    torch.cuda.synchronize()
    return F.double().cpu().numpy(), phi.double().cpu().numpy(), En.item()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("window", ["pkb", "gaussian"])
@pytest.mark.parametrize("N,M,P", [(700, 20, 8), (900, 24, 6), (300, 12, 4)])
def test_line_transforms_match_oracle_and_cufft(N, M, P, window, dtype):
    import paper_1712_04732_gb300 as se
    x = wl.uniform_positions(N, 1.0, 31 + M)
    q = wl.uniform_charges(N, 31 + M)
    pl = se.Plan(1, 1.0, 6.0, M, P, window, dtype=dtype, fft_mode=2)
    pc = se.Plan(1, 1.0, 6.0, M, P, window, dtype=dtype)
    assert pl.info()["column_fft"] == 2 and pc.info()["column_fft"] == 0
    F, phi, En = _run(pl, x, q)
    Fc, phic, Enc = _run(pc, x, q)
    info = pl.info()
    o = S.SEOracle(1, 1.0, 6.0, M, P, window, s_mt=info["s_mt"], nl=info["n_l"])
    pb, gb = o.potential(x, q, grad=True)
    tp, tf = (1e-11, 1e-10) if dtype == torch.float64 else (2e-6, 1e-5)
    assert _rel(phi, pb) < tp
    assert _rel(F, -q[:, None] * gb) < tf
    rc = 1e-12 if dtype == torch.float64 else 1e-6
    assert _rel(phi, phic) < rc
    assert _rel(F, Fc) < rc
    assert En == pytest.approx(Enc, rel=10 * rc)
    pl.close()
    pc.close()


def test_line_transforms_on_the_wire_workload():
    """The wire workload (N = 1.2e6, M = 128, P = 8, 2-3-5-7-smooth lengths:
    J lines of 150, set I padded to 350, zero mode to 378): line transforms
    against cuFFT on every particle, FP32."""
    import paper_1712_04732_gb300 as se
    x, q, spec = wl.make("wire_1p", seed=1)
    kw = dict(dtype=torch.float32, fft_sizes=1)
    pl = se.Plan(1, 1.0, spec["xi"], spec["M"], spec["P"], "pkb", fft_mode=2, **kw)
    pc = se.Plan(1, 1.0, spec["xi"], spec["M"], spec["P"], "pkb", **kw)
    assert pl.info()["column_fft"] == 2
    F, phi, _ = _run(pl, x, q)
    Fc, phic, _ = _run(pc, x, q)
    assert _rel(phi, phic) < 1e-6
    assert _rel(F, Fc) < 1e-6
    assert np.max(np.abs(phi - phic)) < 1e-5 * np.sqrt(np.mean(phic ** 2))
    pl.close()
    pc.close()
