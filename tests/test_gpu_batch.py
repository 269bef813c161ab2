"""Batched evaluation of independent systems (se_batch_*): every system of the
batch matches a standalone plan with the same parameters, the CUDA-graph form
matches the per-system launches, and the Sec. 6 parameter choice meets the
requested tolerance against the direct sums."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import ewald as E
from oracle import params as prm
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
        plan = se.Plan(D, 1.0, specs[i][3], info["M"], info["P"], "pkb", dtype=torch.float32, aft_eps=1e-5 / 4)
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
    """Without autotuning, M_i and P_i + 2 from Sec. 6 for eps_rms = 1e-5 B_i (the
    AFT at a quarter of it): the potential and forces of each system against
    the direct sums (3P k-sum, 2P closed forms), rms error within 1e-5 B_i and
    relative errors within 1e-5."""
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
        pa, ga = E.fourier(D, xs, qs, 1.0, specs[i][3], xt=xs[idx])
        ph = phi[off:off + n].cpu().numpy()[idx]
        assert _rel(ph, pa) < 1e-5
        assert _rel(F[off:off + n].cpu().numpy()[idx], -qs[idx, None] * ga) < 1e-5
        B = prm.scale_B(prm.q_sum_sq(qs), specs[i][3], 1.0)
        assert float(np.sqrt(np.mean((ph - pa) ** 2))) <= 1e-5 * B
        off += n
    b.close()


def test_autotuned_parameters_meet_the_tolerance_for_phi_and_F():
    """The autotuner picks (M, P) per system from candidates around the Sec. 6
    rule by errors measured against an FP64 reference on the first call's
    inputs (each within eps_rel / 2): every system's phi and F then meet 1e-5
    against the direct sums (3P k-sum, 2P closed forms), and the errors the
    tuner reports agree with them."""
    import paper_1712_04732_gb300 as se
    sysl, specs, x, q = _systems(6, seed=9)
    b = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, autotune=True)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    qt = torch.tensor(q, dtype=torch.float32, device="cuda")
    F, phi, _ = b.force(xt, qt)
    torch.cuda.synchronize()
    off = 0
    for i, (xs, qs, D) in enumerate(sysl):
        n = len(qs)
        idx = np.arange(0, n, max(1, n // 200))
        pa, ga = E.fourier(D, xs, qs, 1.0, specs[i][3], xt=xs[idx])
        ep, ef = b.accuracy(i)
        assert 0 <= ep <= 0.5e-5 and 0 <= ef <= 0.5e-5
        assert _rel(phi[off:off + n].cpu().numpy()[idx], pa) < 1e-5
        assert _rel(F[off:off + n].cpu().numpy()[idx], -qs[idx, None] * ga) < 1e-5
        off += n
    b.close()


def _mixed_systems(n_sys, seed, n_min=300, n_max=4000):
    """Systems of every periodicity (D = 3, 2, 1, 0 in turn), N log-uniform."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_sys):
        n = int(10 ** rng.uniform(np.log10(n_min), np.log10(n_max)))
        x = wl.uniform_positions(n, 1.0, seed * 1000 + i)
        q = wl.uniform_charges(n, seed * 1000 + i)
        out.append((x, q, (3, 2, 1, 0)[i % 4]))
    specs = [(len(q), D, 1.0, 8.0 * (len(q) / 1e4) ** (1.0 / 3.0)) for x, q, D in out]
    return out, specs, np.concatenate([s[0] for s in out]), np.concatenate([s[1] for s in out])


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_fused_form_matches_per_system_calls(dtype):
    """The multi-system form (one launch per stage over all systems) against one
    plain se_force per system on the same plans.  The gridding blocks are
    fixed-point sums (exact in any order) and the merge order is fixed.  In
    FP64 the gathering is the same code in both, so potentials and forces are
    bitwise equal; an FP32 se_force of a system with 32 or more particles per
    tile takes the tile-staged gathering, which sums the same products in
    another order, so FP32 agrees to rounding.  Graph replays are bitwise
    equal; the energy sums per-CTA partials over the sorted records, whose order
    inside a tile follows the atomic ranks of the binning, so it agrees to
    rounding."""
    import paper_1712_04732_gb300 as se
    sysl, specs, x, q = _mixed_systems(12, seed=5)
    b = se.Batch(specs, eps_rel=1e-5, dtype=dtype, autotune=False, form="fused")
    Ps = sorted({b.system_info(i)["P"] for i in range(len(specs))})
    assert len(Ps) >= 2, Ps                          # more than one support class
    xt = torch.tensor(x, dtype=dtype, device="cuda")
    qt = torch.tensor(q, dtype=dtype, device="cuda")
    F, phi, En = b.force(xt, qt)
    F2, phi2, En2 = b.force(xt, qt)                 # graph replay
    Fe, phie, Ene = b.force(xt, qt, each=True)
    torch.cuda.synchronize()
    assert b.form()[0] == "fused"
    assert torch.equal(phi, phi2) and torch.equal(F, F2)
    if dtype == torch.float64:
        assert torch.equal(phi, phie) and torch.equal(F, Fe)
    else:
        assert _rel(phi.cpu().numpy(), phie.cpu().numpy()) < 1e-6
        assert _rel(F.cpu().numpy(), Fe.cpu().numpy()) < 1e-6
    rt = 1e-13 if dtype == torch.float64 else 1e-6
    np.testing.assert_allclose(En.cpu().numpy(), Ene.cpu().numpy(), rtol=rt)
    np.testing.assert_allclose(En2.cpu().numpy(), Ene.cpu().numpy(), rtol=rt)
    # every system against the discrete oracle of its own parameters
    from oracle import se_discrete
    off = 0
    for i, (xs, qs, D) in enumerate(sysl):
        n = len(qs)
        info = b.system_info(i)
        ref = se_discrete.SEOracle(D, 1.0, specs[i][3], info["M"], info["P"], "pkb", s_mt=info["s_mt"],
                                   nl=info["n_l"])
        pb, gb = ref.potential(xs, qs, grad=True)
        tol = 1e-10 if dtype == torch.float64 else 2e-5
        assert _rel(phi[off:off + n].double().cpu().numpy(), pb) < tol
        assert _rel(F[off:off + n].double().cpu().numpy(), -qs[:, None] * gb) < 10 * tol
        off += n
    b.close()


def test_fused_form_on_the_batched_workload():
    """The 64-system workload of the benchmark (more than 1024 tiles, so the
    tile-count scan runs several rounds): the multi-system graph against the
    per-system graph and against one se_force per system."""
    import paper_1712_04732_gb300 as se
    sysl = wl.batch_systems(64, seed=1)
    specs = [(len(q), D, 1.0, 8.0 * (len(q) / 1e4) ** (1.0 / 3.0)) for x, q, D in sysl]
    xt = torch.tensor(np.concatenate([s[0] for s in sysl]), dtype=torch.float32, device="cuda")
    qt = torch.tensor(np.concatenate([s[1] for s in sysl]), dtype=torch.float32, device="cuda")
    bf = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, autotune=False, form="fused")
    bb = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, autotune=False, form="branches")
    F, phi, En = bf.force(xt, qt)
    Fb, phib, Enb = bb.force(xt, qt)
    Fe, phie, Ene = bf.force(xt, qt, each=True)
    torch.cuda.synchronize()
    assert sum(bf.system_info(i)["n_tiles"] for i in range(64)) > 1024
    assert bf.form()[0] == "fused" and bb.form()[0] == "branches"
    assert bf.form()[1] < bb.form()[1]               # fewer library launches per call
    for a, c in ((phi, phib), (phi, phie), (F, Fb), (F, Fe)):
        assert _rel(a.cpu().numpy(), c.cpu().numpy()) < 1e-6
    np.testing.assert_allclose(En.cpu().numpy(), Ene.cpu().numpy(), rtol=1e-6)
    bf.close()
    bb.close()


def _systems_3p2p(n_sys, seed, n_min=300, n_max=6000):
    sysl = wl.batch_systems(n_sys, seed=seed, n_min=n_min, n_max=n_max)
    specs = [(len(q), D, 1.0, 8.0 * (len(q) / 1e4) ** (1.0 / 3.0)) for x, q, D in sysl]
    return sysl, specs, np.concatenate([s[0] for s in sysl]), np.concatenate([s[1] for s in sysl])


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_lines_form_matches_per_system_calls(dtype):
    """The single-pipeline form (the transforms of all systems as line transforms
    in five launches, the adaptive transform of the 2P systems included) against
    one se_force per system on the same plans (cuFFT transforms) and against the
    discrete oracle of each system's parameters.  The two transforms round
    differently, so the forms agree to rounding: 1e-12 in FP64, 2e-6 in FP32."""
    import paper_1712_04732_gb300 as se
    sysl, specs, x, q = _systems_3p2p(12, seed=7)
    b = se.Batch(specs, eps_rel=1e-5, dtype=dtype, autotune=False, form="lines")
    xt = torch.tensor(x, dtype=dtype, device="cuda")
    qt = torch.tensor(q, dtype=dtype, device="cuda")
    F, phi, En = b.force(xt, qt)
    F2, phi2, En2 = b.force(xt, qt)                 # graph replay
    Fe, phie, Ene = b.force(xt, qt, each=True)
    torch.cuda.synchronize()
    assert b.form()[0] == "lines"
    assert torch.equal(phi, phi2) and torch.equal(F, F2)
    rt = 1e-12 if dtype == torch.float64 else 2e-6
    off = 0
    for i, (xs, qs, D) in enumerate(sysl):
        n = len(qs)
        assert _rel(phi[off:off + n].cpu().numpy(), phie[off:off + n].cpu().numpy()) < rt
        assert _rel(F[off:off + n].cpu().numpy(), Fe[off:off + n].cpu().numpy()) < rt
        off += n
    np.testing.assert_allclose(En.cpu().numpy(), Ene.cpu().numpy(), rtol=10 * rt)
    from oracle import se_discrete
    off = 0
    for i, (xs, qs, D) in enumerate(sysl):
        n = len(qs)
        info = b.system_info(i)
        if D == 2:
            assert info["s0_mt"] > info["Mt"]            # the zero mode is transformed padded
        ref = se_discrete.SEOracle(D, 1.0, specs[i][3], info["M"], info["P"], "pkb", s_mt=info["s_mt"],
                                   nl=info["n_l"])
        pb, gb = ref.potential(xs, qs, grad=True)
        tol = 1e-10 if dtype == torch.float64 else 2e-5
        assert _rel(phi[off:off + n].double().cpu().numpy(), pb) < tol
        assert _rel(F[off:off + n].double().cpu().numpy(), -qs[:, None] * gb) < 10 * tol
        off += n
    b.close()


def test_lines_form_on_the_batched_workload():
    """The 64-system workload of the benchmark in the single-pipeline form: at
    most 50 kernel launches per call (no cuFFT), results equal to the
    multi-system form with cuFFT transforms to FP32 rounding."""
    import paper_1712_04732_gb300 as se
    sysl, specs, x, q = _systems_3p2p(64, seed=1, n_min=1e3, n_max=1e5)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    qt = torch.tensor(q, dtype=torch.float32, device="cuda")
    bl = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, autotune=False, form="lines")
    bf = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, autotune=False, form="fused")
    F, phi, En = bl.force(xt, qt)
    Ff, phif, Enf = bf.force(xt, qt)
    torch.cuda.synchronize()
    form, kernels = bl.form()
    assert form == "lines" and kernels <= 50, (form, kernels)
    assert _rel(phi.cpu().numpy(), phif.cpu().numpy()) < 2e-6
    assert _rel(F.cpu().numpy(), Ff.cpu().numpy()) < 2e-6
    np.testing.assert_allclose(En.cpu().numpy(), Enf.cpu().numpy(), rtol=2e-5)
    bl.close()
    bf.close()


def test_lines_form_needs_3p_or_2p_systems():
    """A batch with a 1P or free-space system cannot take the single-pipeline
    form: the call reports SE_EINVAL; the autotuner then picks another form."""
    import paper_1712_04732_gb300 as se
    from paper_1712_04732_gb300 import _native as nat
    sysl, specs, x, q = _mixed_systems(4, seed=9)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    qt = torch.tensor(q, dtype=torch.float32, device="cuda")
    b = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, autotune=False, form="lines")
    with pytest.raises(nat.SEError) as ei:
        b.force(xt, qt)
    assert ei.value.name == "SE_EINVAL" and "D = 3 and 2" in str(ei.value)
    b.close()
    bt = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, autotune=True)
    F, phi, En = bt.force(xt, qt)
    torch.cuda.synchronize()
    assert bt.form()[0] in ("fused", "branches")
    assert torch.isfinite(F).all()
    bt.close()


def test_batch_form_flags_exclude_each_other():
    import paper_1712_04732_gb300 as se
    from paper_1712_04732_gb300 import _native as nat
    lib = nat.load()
    h = ctypes.c_void_p()
    n = (ctypes.c_int64 * 1)(1000)
    D = (ctypes.c_int * 1)(3)
    L = (ctypes.c_double * 1)(1.0)
    xi = (ctypes.c_double * 1)(8.0)
    for flags in (nat.SE_BATCH_FUSED | nat.SE_BATCH_BRANCHES, nat.SE_BATCH_LINES | nat.SE_BATCH_FUSED,
                  nat.SE_BATCH_LINES | nat.SE_BATCH_BRANCHES):
        code = lib.se_batch_create(ctypes.byref(h), 1, n, D, L, xi, None, 1e-5, nat.SE_WIN_PKB, nat.SE_F32, flags)
        assert nat.STATUS[code] == "SE_EINVAL"
        assert not h.value
    del se
