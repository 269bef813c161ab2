"""Allocation failures, injected on the host (se_debug_fail_alloc): every device
allocation the library makes can fail, and each failure must come back as
SE_ENOMEM, leak nothing, and leave the library (and a plan whose call failed)
usable.  No GPU fault is involved: the armed allocation returns the error
without calling cudaMalloc."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1712_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SE_ENOMEM = 4


@pytest.fixture
def lib():
    from paper_1712_04732_gb300 import _native as nat
    lib = nat.load()
    yield lib
    lib.se_debug_fail_alloc(0)


def _create(lib, D, M=24, P=8, dt=0):
    from paper_1712_04732_gb300 import _native as nat
    h = ctypes.c_void_p()
    box = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    st = lib.se_plan_create(ctypes.byref(h), box, D, 8.0, M, P, nat.SE_WIN_PKB, dt, None)
    return st, h


@pytest.mark.parametrize("D", [3, 2, 1, 0])
def test_plan_create_reports_every_failed_allocation(lib, D):
    """For k = 1, 2, ...: the k-th allocation of se_plan_create fails ->
    SE_ENOMEM, no plan, and no device memory kept; once k exceeds the number of
    allocations the plan is created."""
    torch.cuda.init()
    torch.cuda.synchronize()
    st, h = _create(lib, D)                 # warm the context, cuFFT and module loads
    assert st == 0
    lib.se_plan_destroy(h)
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(1, 80):
        lib.se_debug_fail_alloc(k)
        st, h = _create(lib, D)
        lib.se_debug_fail_alloc(0)
        if st == 0:
            lib.se_plan_destroy(h)
            break
        assert st == SE_ENOMEM, lib.se_last_error().decode()
        assert not h.value
        assert b"injected" in lib.se_last_error()
        failures += 1
    assert 3 <= failures < 79
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= (16 << 20)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_call_after_a_failed_workspace_growth(lib, dtype):
    """A force call that must grow the particle workspace fails with SE_ENOMEM
    when that allocation fails; the next call (allocation disarmed) succeeds on
    the same plan and gives the result of a fresh plan."""
    import paper_1712_04732_gb300 as se
    plan = se.Plan(3, 1.0, 8.0, 24, 8, "pkb", dtype=dtype)
    N = 2000
    x = torch.tensor(wl.uniform_positions(N, 1.0, 8), dtype=dtype, device="cuda")
    q = torch.tensor(wl.uniform_charges(N, 8), dtype=dtype, device="cuda")
    lib.se_debug_fail_alloc(1)
    with pytest.raises(se.SEError) as ei:
        plan.force(x, q)
    lib.se_debug_fail_alloc(0)
    assert ei.value.code == SE_ENOMEM
    F, phi, _ = plan.force(x, q)
    ref = se.Plan(3, 1.0, 8.0, 24, 8, "pkb", dtype=dtype)
    F2, phi2, _ = ref.force(x, q)
    torch.cuda.synchronize()
    assert torch.equal(phi, phi2) and torch.equal(F, F2)
    plan.close()
    ref.close()


def test_batch_reports_a_failed_allocation(lib):
    """The batch path (per-system plans and the multi-system workspace): an
    allocation failing at set-up or at the first call surfaces as SE_ENOMEM,
    the batch can be destroyed, and an unarmed batch works."""
    import paper_1712_04732_gb300 as se
    sysl = wl.batch_systems(4, seed=2, n_min=300, n_max=2000)
    specs = [(len(q), D, 1.0, 8.0 * (len(q) / 1e4) ** (1.0 / 3.0)) for x, q, D in sysl]
    x = torch.tensor(np.concatenate([s[0] for s in sysl]), dtype=torch.float32, device="cuda")
    q = torch.tensor(np.concatenate([s[1] for s in sysl]), dtype=torch.float32, device="cuda")
    seen = 0
    for k in (1, 5, 20, 60, 120):
        lib.se_debug_fail_alloc(k)
        try:
            b = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, autotune=False, form="fused")
            b.force(x, q)
            torch.cuda.synchronize()
            b.close()
        except se.SEError as exc:
            assert exc.code == SE_ENOMEM
            seen += 1
        finally:
            lib.se_debug_fail_alloc(0)
    assert seen >= 2
    b = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, autotune=False, form="fused")
    F, phi, E = b.force(x, q)
    torch.cuda.synchronize()
    assert torch.isfinite(phi).all() and torch.isfinite(F).all()
    b.close()
