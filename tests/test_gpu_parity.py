"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Oracle B runs the same discrete algorithm (Alg. 4) with the same parameters,
so the FP64 path must agree with it to rounding; the FP32 path to its own
rounding.  Sizes span several gridding tiles with ragged edges.
"""
import numpy as np
import pytest
import torch

from oracle import ewald as E
from oracle import se_discrete as S
from paper_1712_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {torch.float64: (1e-11, 1e-10), torch.float32: (2e-6, 1e-5)}   # (phi, F) relative rms


def _se():
    import paper_1712_04732_gb300 as se
    return se


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def _oracle_for(plan, **kw):
    info = plan.info()
    o = S.SEOracle(plan.D, plan.L, plan.xi, plan.M, plan.P, plan.window, s_mt=info["s_mt"], nl=info["n_l"], **kw)
    assert o.Mt == info["Mt"]
    if plan.D < 3:
        assert o.g["s0Mt"] == info["s0_mt"]
    return o


def _run(plan, x, q, **kw):
    dev = plan.device
    xt = torch.tensor(x, dtype=plan.dtype, device=dev)
    qt = torch.tensor(q, dtype=plan.dtype, device=dev)
    F, phi, En = plan.force(xt, qt, energy=True, **kw)
    torch.cuda.synchronize()
    return F.double().cpu().numpy(), phi.double().cpu().numpy(), En.item()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("window", ["pkb", "gaussian"])
@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_force_and_potential_match_discrete_oracle(D, window, dtype):
    se = _se()
    N, M, P = 700, 20, 8
    x = wl.uniform_positions(N, 1.0, 11 + D)
    q = wl.uniform_charges(N, 11 + D)
    plan = se.Plan(D, 1.0, 6.0, M, P, window, dtype=dtype)
    F, phi, En = _run(plan, x, q)
    o = _oracle_for(plan)
    pb, gb = o.potential(x, q, grad=True)
    tp, tf = TOL[dtype]
    assert _rel(phi, pb) < tp
    assert _rel(F, -q[:, None] * gb) < tf
    assert En == pytest.approx(0.5 * float(q @ pb), rel=10 * tp)


@pytest.mark.parametrize("spread_mode,gather_mode,split", [
    (1, 1, 1), (2, 1, 2), (2, 1, 4), (2, 2, 8), (3, 1, 1), (3, 2, 1), (1, 2, 3), (2, 3, 2), (2, 0, 1), (2, 4, 1)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_every_kernel_variant(spread_mode, gather_mode, split, dtype):
    """Gridding variants (shared atomics, cluster-split atomics, per-warp private
    blocks) and gathering variants (staged with split CTAs, direct reads, the
    staged block over chunks with four particles or one particle per warp --
    the FP32 defaults at 111 particles per tile) give the same potential and
    forces."""
    se = _se()
    N, M = 3000, 24
    x = wl.uniform_positions(N, 1.0, 41)
    q = wl.uniform_charges(N, 41)
    for D in (3, 2):
        plan = se.Plan(D, 1.0, 6.0, M, 8, "pkb", dtype=dtype, spread_mode=spread_mode,
                       gather_mode=gather_mode, split=split)
        F, phi, En = _run(plan, x, q)
        pb, gb = _oracle_for(plan).potential(x, q, grad=True)
        tp, tf = TOL[dtype]
        assert _rel(phi, pb) < tp
        assert _rel(F, -q[:, None] * gb) < tf
        assert En == pytest.approx(0.5 * float(q @ pb), rel=10 * tp)


@pytest.mark.parametrize("P", [2, 4, 6, 10, 12, 14, 16])
def test_every_compiled_support(P):
    se = _se()
    D = [3, 2, 1, 0][P // 2 % 4]
    N, M = 300, max(16, P + 4)
    x = wl.uniform_positions(N, 1.0, 100 + P)
    q = wl.uniform_charges(N, 100 + P)
    pb = gb = None
    for fm in (1, 2):
        plan = se.Plan(D, 1.0, 5.0, M, P, "pkb", dtype=torch.float64, force_method=fm)
        F, phi, _ = _run(plan, x, q)
        pb, gb = _oracle_for(plan).potential(x, q, grad=True, force_method=fm)
        assert _rel(phi, pb) < 1e-11
        assert _rel(F, -q[:, None] * gb) < 1e-10


@pytest.mark.parametrize("D", [3, 1])
def test_grid_not_divisible_by_the_tile(D):
    """M = 28: the periodic tile edge becomes 7 (a divisor of M); free axes end ragged."""
    se = _se()
    x = wl.uniform_positions(500, 1.0, 5)
    q = wl.uniform_charges(500, 5)
    plan = se.Plan(D, 1.0, 6.5, 28, 6, "pkb", dtype=torch.float64)
    assert 28 % plan.info()["tile"][0] == 0
    F, phi, _ = _run(plan, x, q)
    pb, gb = _oracle_for(plan).potential(x, q, grad=True)
    assert _rel(phi, pb) < 1e-11
    assert _rel(F, -q[:, None] * gb) < 1e-10


@pytest.mark.parametrize("tile", [4, 16])
def test_tile_edges(tile):
    se = _se()
    x = wl.uniform_positions(800, 1.0, 6)
    q = wl.uniform_charges(800, 6)
    plan = se.Plan(2, 1.0, 6.0, 32, 8, "pkb", dtype=torch.float64, tile=tile)
    F, phi, _ = _run(plan, x, q)
    pb, gb = _oracle_for(plan).potential(x, q, grad=True)
    assert _rel(phi, pb) < 1e-11
    assert _rel(F, -q[:, None] * gb) < 1e-10


def test_positions_on_grid_lines_and_box_faces():
    """Particles exactly on grid nodes, on tile boundaries and at x = 0.  With a
    dyadic spacing (M = 32) x / h is exact in both the kernel and the oracle, so
    both place the support identically and agree to rounding."""
    se = _se()
    M = 32
    h = 1.0 / M
    rng = np.random.default_rng(4)
    x = rng.integers(0, M, size=(200, 3)) * h
    x[:10] = 0.0
    x[10:20, 0] = 8 * h
    q = wl.uniform_charges(200, 9)
    for D in (3, 2, 0):
        plan = se.Plan(D, 1.0, 6.0, M, 6, "pkb", dtype=torch.float64)
        F, phi, _ = _run(plan, x, q)
        pb, gb = _oracle_for(plan).potential(x, q, grad=True)
        assert _rel(phi, pb) < 1e-11


def test_positions_on_grid_lines_non_dyadic_spacing():
    """With h = 1/24 a node coordinate x / h may round to either side of the
    integer, which moves the support by one point; the truncated window's edge
    value W(w) = 1/I0(beta) bounds the difference (Sec. 4: the KB window does
    not vanish at |x| = w)."""
    se = _se()
    M = 24
    rng = np.random.default_rng(4)
    x = rng.integers(0, M, size=(200, 3)) / M
    q = wl.uniform_charges(200, 9)
    plan = se.Plan(3, 1.0, 6.0, M, 6, "pkb", dtype=torch.float64)
    F, phi, _ = _run(plan, x, q)
    pb, _ = _oracle_for(plan).potential(x, q, grad=True)
    from scipy.special import i0
    assert _rel(phi, pb) < 20.0 / i0(2.5 * 6)


def test_periodic_coordinates_are_wrapped():
    se = _se()
    x = wl.uniform_positions(300, 1.0, 8)
    q = wl.uniform_charges(300, 8)
    plan = se.Plan(2, 1.0, 6.0, 24, 6, "pkb", dtype=torch.float64)
    _, phi0, _ = _run(plan, x, q)
    xs = x.copy()
    xs[:, 0] += np.where(np.arange(300) % 2, 3.0, -2.0)
    xs[:, 1] -= 1.0
    _, phi1, _ = _run(plan, xs, q)
    assert _rel(phi1, phi0) < 1e-12


def test_all_particles_in_one_tile():
    se = _se()
    rng = np.random.default_rng(2)
    x = 0.5 + 0.01 * rng.random((2000, 3))
    q = wl.uniform_charges(2000, 2)
    plan = se.Plan(0, 1.0, 6.0, 24, 8, "pkb", dtype=torch.float64)
    F, phi, _ = _run(plan, x, q)
    pb, gb = _oracle_for(plan).potential(x, q, grad=True)
    assert _rel(phi, pb) < 1e-11
    assert _rel(F, -q[:, None] * gb) < 1e-10


def test_single_particle_and_empty_input():
    se = _se()
    plan = se.Plan(3, 1.0, 6.0, 16, 6, "pkb", dtype=torch.float64)
    x = np.array([[0.3, 0.6, 0.9]])
    q = np.array([1.0])
    F, phi, _ = _run(plan, x, q)
    pb, gb = _oracle_for(plan).potential(x, q, grad=True)
    assert _rel(phi, pb) < 1e-12
    e = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    out = plan.potential(e, torch.empty(0, dtype=torch.float64, device="cuda"))
    assert out.shape == (0,)


def test_self_term_flag():
    se = _se()
    x = wl.uniform_positions(200, 1.0, 1)
    q = wl.uniform_charges(200, 1)
    plan = se.Plan(3, 1.0, 6.0, 16, 6, "pkb", dtype=torch.float64)
    _, p0, _ = _run(plan, x, q)
    _, p1, _ = _run(plan, x, q, add_self=True)
    assert np.allclose(p1 - p0, -2 * 6.0 / np.sqrt(np.pi) * q, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("D,M,P", [(2, 24, 8), (1, 24, 8), (0, 36, 6)])
def test_fft_friendly_sizes_match_discrete_oracle(D, M, P):
    """fft_sizes = 1 rounds the free-direction lengths M~, s0 M~ and s M~ up to
    2-3-5-7-smooth sizes (here M~ = 44 -> 48): the discrete oracle given the
    same extension and upsampling (lambda = (M~ - M) / P, s0 = s0 M~ / M~, the
    same s M~ and n_l) agrees to FP64 rounding, and the result stays within the
    method's error of the default plan's."""
    se = _se()
    N = 500
    x = wl.uniform_positions(N, 1.0, 41)
    q = wl.uniform_charges(N, 41)
    plan = se.Plan(D, 1.0, 6.0, M, P, "pkb", dtype=torch.float64, fft_sizes=1)
    base = se.Plan(D, 1.0, 6.0, M, P, "pkb", dtype=torch.float64)
    info, binfo = plan.info(), base.info()
    assert info["Mt"] == 48 and binfo["Mt"] == 44
    for n in (info["Mt"], info["s0_mt"], info["s_mt"]):
        if n == 0:                                  # no set-I transform (D = 0)
            continue
        r = n
        for f in (2, 3, 5, 7):
            while r % f == 0:
                r //= f
        assert r == 1 and n % 2 == 0
    F, phi, _ = _run(plan, x, q)
    o = S.SEOracle(D, 1.0, 6.0, M, P, "pkb", lam=(info["Mt"] - M) / P, s0=info["s0_mt"] / info["Mt"],
                   s_mt=info["s_mt"], nl=info["n_l"])
    assert o.Mt == info["Mt"] and o.g["s0Mt"] == info["s0_mt"]
    pb, gb = o.potential(x, q, grad=True)
    assert _rel(phi, pb) < 1e-11
    assert _rel(F, -q[:, None] * gb) < 1e-10
    F0, phi0, _ = _run(base, x, q)
    assert _rel(phi, phi0) < 1e-4


def test_host_io_path_equals_device_path():
    se = _se()
    x = wl.uniform_positions(1000, 1.0, 12)
    q = wl.uniform_charges(1000, 12)
    plan = se.Plan(1, 1.0, 6.0, 20, 6, "pkb", dtype=torch.float32)
    F, phi, En = _run(plan, x, q)
    xh = torch.tensor(x, dtype=torch.float32).pin_memory()
    qh = torch.tensor(q, dtype=torch.float32).pin_memory()
    Fh = torch.empty((1000, 3), dtype=torch.float32).pin_memory()
    ph = torch.empty(1000, dtype=torch.float32).pin_memory()
    eh = torch.empty((), dtype=torch.float64).pin_memory()
    plan.force_host(xh, qh, Fh, ph, eh)
    assert _rel(ph.double().numpy(), phi) < 1e-6
    assert _rel(Fh.double().numpy(), F) < 1e-6
    assert eh.item() == pytest.approx(En, rel=1e-6)


@pytest.mark.parametrize("D", [3, 1])
def test_host_io_page_locked_inputs_read_in_place_fp64(D):
    """FP64 SE_HOST_IO calls with page-locked x and q (read in place by the
    counting pass, which writes the device copies) against the device path:
    the same kernels on the same values, so the results agree to the last bits
    of the energy's summation order."""
    se = _se()
    N = 2000
    x = wl.uniform_positions(N, 1.0, 40 + D)
    q = wl.uniform_charges(N, 40 + D)
    plan = se.Plan(D, 1.0, 6.0, 24, 8, "pkb", dtype=torch.float64)
    F, phi, En = _run(plan, x, q)
    xh = torch.tensor(x, dtype=torch.float64).pin_memory()
    qh = torch.tensor(q, dtype=torch.float64).pin_memory()
    Fh = torch.empty((N, 3), dtype=torch.float64).pin_memory()
    ph = torch.empty(N, dtype=torch.float64).pin_memory()
    eh = torch.empty((), dtype=torch.float64).pin_memory()
    for _ in range(2):                               # eager capture, then the replayed graph
        plan.force_host(xh, qh, Fh, ph, eh)
        assert np.array_equal(ph.numpy(), phi) and np.array_equal(Fh.numpy(), F)
        assert eh.item() == pytest.approx(En, rel=1e-13)


def test_host_io_graph_replay_follows_new_contents_and_buffers():
    """Repeated SE_HOST_IO calls on the same page-locked buffers replay a captured
    graph: new contents written into the buffers between calls must be read
    again; new buffers, pageable buffers and a potential-only call (other
    flags) must give the same results as the device path."""
    se = _se()
    N = 1500
    plan = se.Plan(0, 1.0, 6.0, 24, 8, "pkb", dtype=torch.float32)
    xh = torch.empty((N, 3), dtype=torch.float32).pin_memory()
    qh = torch.empty(N, dtype=torch.float32).pin_memory()
    Fh = torch.empty((N, 3), dtype=torch.float32).pin_memory()
    ph = torch.empty(N, dtype=torch.float32).pin_memory()
    eh = torch.empty((), dtype=torch.float64).pin_memory()
    for seed in (31, 32, 33):                       # same buffers, new contents
        x = wl.uniform_positions(N, 1.0, seed)
        q = wl.uniform_charges(N, seed)
        xh.copy_(torch.tensor(x, dtype=torch.float32))
        qh.copy_(torch.tensor(q, dtype=torch.float32))
        plan.force_host(xh, qh, Fh, ph, eh)
        F, phi, En = _run(plan, x, q)
        assert _rel(ph.double().numpy(), phi) < 1e-6
        assert _rel(Fh.double().numpy(), F) < 1e-6
        assert eh.item() == pytest.approx(En, rel=1e-6)
    # other buffers (pinned and pageable), then the potential alone
    x = wl.uniform_positions(N, 1.0, 34)
    q = wl.uniform_charges(N, 34)
    F, phi, En = _run(plan, x, q)
    for pin in (True, False):
        mk = (lambda t: t.pin_memory()) if pin else (lambda t: t)
        xh2, qh2 = mk(torch.tensor(x, dtype=torch.float32)), mk(torch.tensor(q, dtype=torch.float32))
        Fh2, ph2 = mk(torch.empty((N, 3), dtype=torch.float32)), mk(torch.empty(N, dtype=torch.float32))
        eh2 = mk(torch.empty((), dtype=torch.float64))
        plan.force_host(xh2, qh2, Fh2, ph2, eh2)
        assert _rel(ph2.double().numpy(), phi) < 1e-6 and _rel(Fh2.double().numpy(), F) < 1e-6
        assert eh2.item() == pytest.approx(En, rel=1e-6)
        pp = mk(torch.empty(N, dtype=torch.float32))
        plan.potential_host(xh2, qh2, pp)
        assert _rel(pp.double().numpy(), phi) < 1e-6


def test_vjp_matches_oracle_and_linearity():
    """g_q = A g and g_x = g grad(A q) + q grad(A g) (operator symmetry)."""
    se = _se()
    N = 500
    x = wl.uniform_positions(N, 1.0, 21)
    q = wl.uniform_charges(N, 21)
    g = wl.uniform_charges(N, 22)
    for D in (3, 1):
        plan = se.Plan(D, 1.0, 6.0, 20, 8, "pkb", dtype=torch.float64)
        xt, qt, gt = (torch.tensor(a, device="cuda") for a in (x, q, g))
        gx, gq = plan.vjp(xt, qt, gt)
        o = _oracle_for(plan)
        pg, dg = o.potential(x, g, grad=True)
        _, dq = o.potential(x, q, grad=True)
        assert _rel(gq.cpu().numpy(), pg) < 1e-11
        ref = g[:, None] * dq + q[:, None] * dg
        assert _rel(gx.cpu().numpy(), ref) < 1e-10


def test_energy_autograd_against_finite_differences():
    """E = 1/2 q.phi; dE/dx = -F and dE/dq = phi versus central differences (FP64,
    h = 1e-6, 32 particles kept away from grid lines where the window shifts)."""
    se = _se()
    plan = se.Plan(0, 1.0, 6.0, 24, 8, "pkb", dtype=torch.float64)
    h = 1.0 / 24
    info = plan.info()
    off = info["delta_L"] / 2
    rng = np.random.default_rng(3)
    x = []
    while len(x) < 32:
        c = rng.random(3)
        fr = ((c + off) / h) % 1.0
        if np.all((fr > 1e-3) & (fr < 1 - 1e-3)):
            x.append(c)
    x = torch.tensor(np.array(x), device="cuda", requires_grad=True)
    q = torch.tensor(wl.uniform_charges(32, 3), device="cuda", requires_grad=True)
    En = se.energy(plan, x, q)
    En.backward()
    eps = 1e-6
    xd = x.detach()
    for idx in [(0, 0), (5, 1), (17, 2), (31, 0)]:
        xp = xd.clone(); xp[idx] += eps
        xm = xd.clone(); xm[idx] -= eps
        fd = (se.energy(plan, xp, q.detach()).item() - se.energy(plan, xm, q.detach()).item()) / (2 * eps)
        assert x.grad[idx].item() == pytest.approx(fd, rel=1e-6, abs=1e-8)
    for i in [0, 9, 30]:
        qp = q.detach().clone(); qp[i] += eps
        qm = q.detach().clone(); qm[i] -= eps
        fd = (se.energy(plan, xd, qp).item() - se.energy(plan, xd, qm).item()) / (2 * eps)
        assert q.grad[i].item() == pytest.approx(fd, rel=1e-6, abs=1e-8)


def test_potential_autograd_gradcheck():
    se = _se()
    plan = se.Plan(3, 1.0, 5.0, 16, 6, "pkb", dtype=torch.float64)
    rng = np.random.default_rng(5)
    x = []
    while len(x) < 12:
        c = rng.random(3)
        fr = (c * 16) % 1.0
        if np.all((fr > 1e-2) & (fr < 1 - 1e-2)):
            x.append(c)
    x = torch.tensor(np.array(x), device="cuda", requires_grad=True)
    q = torch.tensor(wl.uniform_charges(12, 5), device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda a, b: se.potential(plan, a, b), (x, q), eps=1e-6, atol=1e-5, rtol=1e-4)


def test_neutrality_and_box_errors():
    se = _se()
    plan = se.Plan(2, 1.0, 6.0, 16, 6, "pkb", dtype=torch.float64)
    x = torch.tensor(wl.uniform_positions(50, 1.0, 1), device="cuda")
    q = torch.ones(50, dtype=torch.float64, device="cuda")
    with pytest.raises(se.SEError) as ei:
        plan.potential(x, q, check_neutral=True)
    assert ei.value.name == "SE_ENONNEUTRAL"
    xb = x.clone()
    xb[3, 2] = 1.5                      # free direction, outside [0, L)
    with pytest.raises(se.SEError) as ei:
        plan.potential(xb, q - q.mean(), sync_check=True)
    assert ei.value.name == "SE_EOUTOFBOX"
    xn = x.clone()
    xn[7, 0] = float("nan")
    with pytest.raises(se.SEError) as ei:
        plan.potential(xn, q - q.mean(), sync_check=True)
    assert ei.value.name == "SE_ENOTFINITE"
    plan.potential(x, q - q.mean(), sync_check=True)     # the plan stays usable


def test_streams_and_repeatability():
    se = _se()
    x = torch.tensor(wl.uniform_positions(4000, 1.0, 1), device="cuda", dtype=torch.float32)
    q = torch.tensor(wl.uniform_charges(4000, 1), device="cuda", dtype=torch.float32)
    plan = se.Plan(3, 1.0, 8.0, 32, 8, "pkb", dtype=torch.float32)
    p0 = plan.potential(x, q)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        p1 = plan.potential(x, q)
    s.synchronize()
    assert torch.allclose(p0, p1, rtol=1e-5, atol=1e-6 * p0.abs().max().item())


# ----------------------------------------------------- the named workloads at full size

def _sample(n, k, seed=0):
    return np.sort(np.random.default_rng(seed).choice(n, size=min(k, n), replace=False))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_free_space_workload_full_size(dtype):
    """0P, N = 20000, M = 48, lambda = 2, PKB P = 8, xi = 8 (the benchmark workload): the
    GPU against the direct sum (oracle A) on 400 sampled targets (rms relative
    error <= 1e-5 for phi and F) and against oracle B (same discretisation)."""
    se = _se()
    x, q, spec = wl.make("free_0p", seed=1)
    plan = se.Plan(0, 1.0, 8.0, 48, 8, "pkb", dtype=dtype, lam=spec["lam"])
    F, phi, En = _run(plan, x, q)
    idx = _sample(len(q), 400)
    pa, ga = E.fourier(0, x, q, 1.0, 8.0, xt=x[idx])
    assert _rel(phi[idx], pa) < 1e-5
    assert _rel(F[idx], -q[idx, None] * ga) < 1e-5
    o = _oracle_for(plan, lam=spec["lam"])
    pb, gb = o.potential(x, q, xt=x[idx], grad=True)
    tp, tf = TOL[dtype]
    assert _rel(phi[idx], pb) < tp
    assert _rel(F[idx], -q[idx, None] * gb) < tf


def test_lattice_workload_madelung():
    """3P, NaCl cell (512 ions): SE k-space part (Gaussian P = 8 is accurate to
    ~1e-5; P = 16 PKB to ~1e-14) plus the oracle's real-space and self terms
    reproduces the Madelung constant."""
    se = _se()
    x, q = wl.nacl_cell(8, 1.0)
    plan = se.Plan(3, 1.0, 8.0, 48, 16, "pkb", dtype=torch.float64)
    _, phi, _ = _run(plan, x, q)
    pr, _ = E.real(3, x, q, 1.0, 8.0, 6.5 / 8.0)
    tot = phi + pr + E.self_term(q, 8.0)
    assert np.allclose(-(tot * q) / 8.0, 1.7475645946, atol=1e-9)


def test_lattice_workload_gaussian():
    se = _se()
    x, q, spec = wl.make("lattice_3p", seed=1)
    plan = se.Plan(3, 1.0, 8.0, 32, 8, "gaussian", dtype=torch.float64)
    F, phi, _ = _run(plan, x, q)
    pa, ga = E.fourier(3, x, q, 1.0, 8.0)
    assert _rel(phi, pa) < 3 * 2 * np.exp(-(np.pi / 2) * 8 * np.sqrt(0.91))   # Sec. 5.2 estimate
    pb, gb = _oracle_for(plan).potential(x, q, grad=True)
    assert _rel(phi, pb) < 1e-11


def _tile_ids(plan, x):
    """Gridding tile of each particle: the tile holding its lowest support point
    floor(t) - P/2 + 1 (t = (x + offset)/h, wrapped along periodic axes)."""
    info = plan.info()
    h, D, P = info["h"], plan.D, plan.P
    n = np.array(info["grid"])
    T = np.array(info["tile"])
    off = np.array([0.0 if a < D else (info["Mt_v"][a] - info["M_v"][a]) * h / 2 for a in range(3)])
    anc = np.floor((x + off) / h).astype(np.int64) - P // 2 + 1
    for a in range(D):
        anc[:, a] %= n[a]
    t = anc // T
    nt = -(-n // T)
    return (t[:, 2] * nt[1] + t[:, 1]) * nt[0] + t[:, 0]


def _stratified(plan, x, k_random, seed):
    """One target in every non-empty gridding tile, plus k_random drawn at random."""
    _, first = np.unique(_tile_ids(plan, x), return_index=True)
    extra = np.random.default_rng(seed).choice(len(x), size=min(k_random, len(x)), replace=False)
    return np.unique(np.concatenate([first, extra]))


def _assert_elementwise(a, b, tol):
    """Every element within tol times the rms of the reference."""
    err = np.abs(np.asarray(a) - b).max()
    assert err <= tol * np.sqrt(np.mean(np.asarray(b) ** 2)), err


@pytest.mark.parametrize("dtype,P", [(torch.float32, 6), (torch.float32, 8), (torch.float64, 10)])
def test_slab_workload_full_size(dtype, P):
    """2P, N = 100000, M = 64, xi = 16, PKB P = 6, 8 (FP32) / 10 (FP64): the GPU
    against oracle B (same discretisation) at full size, on one target in every
    non-empty gridding tile plus 300 at random: rms and element-wise."""
    se = _se()
    x, q, spec = wl.make("slab_2p", seed=1)
    plan = se.Plan(2, 1.0, spec["xi"], spec["M"], P, "pkb", dtype=dtype)
    F, phi, _ = _run(plan, x, q)
    idx = _stratified(plan, x, 300, 1)
    assert len(idx) >= plan.info()["n_tiles"] // 2
    pb, gb = _oracle_for(plan).potential(x, q, xt=x[idx], grad=True)
    tp, tf = TOL[dtype]
    assert _rel(phi[idx], pb) < tp
    assert _rel(F[idx], -q[idx, None] * gb) < tf
    _assert_elementwise(phi[idx], pb, 10 * tp)
    _assert_elementwise(F[idx], -q[idx, None] * gb, 10 * tf)


@pytest.mark.parametrize("dtype,P,tol_phi,tol_F", [(torch.float32, 6, 1e-5, 3e-4), (torch.float32, 8, 1e-5, 1e-5),
                                                   (torch.float64, 10, 1e-9, 2e-8)])
def test_slab_parameters_accuracy_against_direct_sum(dtype, P, tol_phi, tol_F):
    """The slab grid (M = 64, xi = 16) against the closed forms Eqs. (2pno0), (2p0)
    on 2000 particles (200 sampled targets); forces need P + 2 for the
    potential's accuracy (Sec. 7.2)."""
    se = _se()
    x, q, spec = wl.make("slab_2p", seed=3, N=2000)
    plan = se.Plan(2, 1.0, spec["xi"], spec["M"], P, "pkb", dtype=dtype)
    F, phi, _ = _run(plan, x, q)
    idx = _sample(len(q), 200, 4)
    pa, ga = E.fourier(2, x, q, 1.0, spec["xi"], xt=x[idx])
    assert _rel(phi[idx], pa) < tol_phi
    assert _rel(F[idx], -q[idx, None] * ga) < tol_F


@pytest.mark.parametrize("fft_sizes", [0, 1])
def test_wire_workload_full_size(fft_sizes):
    """1P, N = 1.2e6 (a sixth of them in ten Gaussian clouds), M = 128, xi = 32,
    PKB P = 8, FP32, with the paper's minimal transform lengths and with the
    2-3-5-7-smooth lengths the benchmark times (fft_sizes = 1; the oracle given
    the same extension and upsampling): the GPU against oracle B at full size on
    one target in every non-empty gridding tile (every tile of the clouds
    included) plus 200 at random, rms and element-wise."""
    se = _se()
    x, q, spec = wl.make("wire_1p", seed=1)
    plan = se.Plan(1, 1.0, spec["xi"], spec["M"], spec["P"], "pkb", dtype=torch.float32, fft_sizes=fft_sizes)
    F, phi, _ = _run(plan, x, q)
    idx = _stratified(plan, x, 200, 2)
    info = plan.info()
    assert len(idx) >= info["n_tiles"] // 4
    if fft_sizes:
        o = S.SEOracle(1, 1.0, spec["xi"], spec["M"], spec["P"], "pkb", lam=(info["Mt"] - spec["M"]) / spec["P"],
                       s0=info["s0_mt"] / info["Mt"], s_mt=info["s_mt"], nl=info["n_l"])
        assert o.Mt == info["Mt"] and o.g["s0Mt"] == info["s0_mt"]
    else:
        o = _oracle_for(plan)
    pb, gb = o.potential(x, q, xt=x[idx], grad=True)
    tp, tf = TOL[torch.float32]
    assert _rel(phi[idx], pb) < tp
    assert _rel(F[idx], -q[idx, None] * gb) < tf
    _assert_elementwise(phi[idx], pb, 10 * tp)
    _assert_elementwise(F[idx], -q[idx, None] * gb, 10 * tf)


def test_fp32_tile_beyond_the_fixed_point_limit():
    """FP32 gridding accumulates fixed-point integers in tiles of up to 65 536
    particles and float atomics beyond: 70 000 particles packed into one tile
    (3P, M = 32, tile edge 8: every lowest support point in cells 0..7) take the
    float path, against oracle B."""
    se = _se()
    N = 70000
    x = 3.0 / 32 + (8.0 / 32) * wl.uniform_positions(N, 1.0, 91) * (1 - 1e-7)
    q = wl.uniform_charges(N, 91)
    plan = se.Plan(3, 1.0, 6.0, 32, 8, "pkb", dtype=torch.float32, tile=8)
    assert len(np.unique(_tile_ids(plan, x))) == 1
    F, phi, _ = _run(plan, x, q)
    idx = _sample(N, 300, 3)
    pb, gb = _oracle_for(plan).potential(x, q, xt=x[idx], grad=True)
    assert _rel(phi[idx], pb) < 1e-5
    assert _rel(F[idx], -q[idx, None] * gb) < 3e-5


def test_wire_parameters_accuracy_against_direct_sum():
    """The wire grid (M = 128, xi = 32, P = 8) against the 1P sum through
    xi-independence (Sec. 2) on 3000 particles (clouds included)."""
    se = _se()
    x, q, spec = wl.make("wire_1p", seed=5, N=3000)
    plan = se.Plan(1, 1.0, spec["xi"], spec["M"], spec["P"], "pkb", dtype=torch.float32)
    F, phi, _ = _run(plan, x, q)
    pa, ga = E.fourier_xi_route(1, x, q, 1.0, spec["xi"])
    assert _rel(phi, pa) < 1e-5
    assert _rel(F, -q[:, None] * ga) < 1e-5


@pytest.mark.parametrize("M,P,lam,fused", [(20, 8, None, 1), (10, 4, 1.3, 1), (20, 6, 1.3, 0), (16, 4, 1.3, 0)])
@pytest.mark.parametrize("force_method", [1, 2])
def test_free_space_column_stage_and_cufft_agree(M, P, lam, fused, force_method):
    """D = 0: the fused column kernel (2 M~ = 64, 32) and the cuFFT stages
    (fft_mode = 1, or 2 M~ = 56, 44 that are not powers of two) both match the
    oracle, for both force methods."""
    se = _se()
    N = 900
    x = wl.uniform_positions(N, 1.0, 61 + M + P)
    q = wl.uniform_charges(N, 61 + M + P)
    pb = gb = None
    for mode in (0, 1):
        plan = se.Plan(0, 1.0, 6.0, M, P, "pkb", dtype=torch.float64, lam=lam, force_method=force_method,
                       fft_mode=mode)
        assert plan.info()["column_fft"] == (fused if mode == 0 else 0)
        F, phi, _ = _run(plan, x, q)
        if pb is None:
            pb, gb = _oracle_for(plan, lam=lam).potential(x, q, grad=True, force_method=force_method)
        assert _rel(phi, pb) < 1e-11
        assert _rel(F, -q[:, None] * gb) < 1e-10


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("D", [3, 0])
def test_results_are_bit_reproducible(D, dtype):
    """Gridding accumulates integers (fixed point with a power-of-two scale per
    tile), the merge runs in a fixed order and the transforms and the gathering
    are deterministic, so two calls on the same input give identical bits of
    phi and F.  The FP64 energy sum follows the order of the particles within a
    tile, which the binning's atomics decide: equal to rounding."""
    se = _se()
    N = 5000
    x = torch.tensor(wl.uniform_positions(N, 1.0, 77), dtype=dtype, device="cuda")
    q = torch.tensor(wl.uniform_charges(N, 77), dtype=dtype, device="cuda")
    plan = se.Plan(D, 1.0, 6.0, 24, 8, "pkb", dtype=dtype)
    F1, p1, E1 = plan.force(x, q, energy=True)
    F2, p2, E2 = plan.force(x, q, energy=True)
    torch.cuda.synchronize()
    assert torch.equal(F1, F2) and torch.equal(p1, p2)
    assert abs(E1.item() - E2.item()) <= 1e-13 * abs(E1.item())


def test_fixed_point_gridding_extreme_charge_scales():
    """The per-tile scale follows the charges' magnitude: scaling q by 1e-12 or
    1e+12 scales phi by that factor and F by its square."""
    se = _se()
    N = 2000
    x = torch.tensor(wl.uniform_positions(N, 1.0, 78), dtype=torch.float32, device="cuda")
    q = torch.tensor(wl.uniform_charges(N, 78), dtype=torch.float32, device="cuda")
    plan = se.Plan(3, 1.0, 6.0, 24, 8, "pkb", dtype=torch.float32)
    F, phi, _ = plan.force(x, q, energy=True)
    for f in (1e-12, 1e12):
        Fs, ps, _ = plan.force(x, q * f, energy=True)
        torch.cuda.synchronize()
        assert _rel((ps / f).double().cpu().numpy(), phi.double().cpu().numpy()) < 1e-6
        assert _rel((Fs / (f * f)).double().cpu().numpy(), F.double().cpu().numpy()) < 1e-6
