"""se_potential_noalloc: the potential without device allocation in the call.

Callers that may not allocate device memory while they run (a fixed memory
budget handed out at start-up, no implicit cudaMalloc synchronisation inside a
time step) create and reserve the plan once, then use this entry point.  It
must give the same potential as se_potential, call after call, although the
fixed gridding scratch keeps the previous call's contents.  This file is
collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1712_04732_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _positions(kind, N, seed):
    """Uniform in the unit box, or packed into the corner cube [0, 0.3)^3 so that
    most gridding tiles are empty (their blocks in the fixed scratch then still
    hold the previous call's values, which must not be read)."""
    x = wl.uniform_positions(N, 1.0, seed)
    return x if kind == "uniform" else 0.3 * x


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
@pytest.mark.parametrize("D", [3, 2, 1, 0])
@pytest.mark.parametrize("sequence", [("uniform", "uniform"), ("uniform", "corner")])
def test_noalloc_potential_matches_se_potential_on_two_calls(D, dtype, tol, sequence):
    import paper_1712_04732_gb300 as se
    from paper_1712_04732_gb300 import _native as nat
    lib = nat.load()
    N = 3000
    plan = se.Plan(D, 1.0, 6.0, 24, 8, "pkb", dtype=dtype)
    plan.reserve(N)
    for call, (kind, seed) in enumerate(zip(sequence, (31, 32))):   # two calls in a row, different systems
        x = torch.tensor(_positions(kind, N, seed), dtype=dtype, device="cuda")
        q = torch.tensor(wl.uniform_charges(N, seed), dtype=dtype, device="cuda")
        ref = plan.potential(x, q)
        out = torch.full_like(ref, float("nan"))
        plan._sync_stream()
        st = lib.se_potential_noalloc(plan.handle, N, _ptr(x), _ptr(q), _ptr(out), 0)
        assert st == 0, lib.se_last_error().decode()
        torch.cuda.synchronize()
        r, o = ref.double().cpu().numpy(), out.double().cpu().numpy()
        assert np.all(np.isfinite(o)), f"call {call}"
        assert np.linalg.norm(o - r) / np.linalg.norm(r) < tol, f"call {call}"
    plan.close()


def test_noalloc_rejects_what_it_cannot_do_without_allocating():
    import paper_1712_04732_gb300 as se
    from paper_1712_04732_gb300 import _native as nat
    lib = nat.load()
    plan = se.Plan(3, 1.0, 6.0, 16, 6, "pkb", dtype=torch.float32)
    plan.reserve(100)
    cap = plan.info()["capacity"]
    x = torch.rand((cap + 1, 3), device="cuda")
    q = torch.zeros(cap + 1, device="cuda")
    phi = torch.empty(cap + 1, device="cuda")
    plan._sync_stream()
    assert lib.se_potential_noalloc(plan.handle, cap + 1, _ptr(x), _ptr(q), _ptr(phi), 0) == 9   # SE_ECAPACITY
    assert lib.se_potential_noalloc(plan.handle, 10, _ptr(x), _ptr(q), _ptr(phi), nat.SE_HOST_IO) == 1
    assert lib.se_potential_noalloc(plan.handle, 10, _ptr(x), _ptr(q), _ptr(phi), 0) == 0
    torch.cuda.synchronize()
    plan.close()


def test_noalloc_rejects_blocks_beyond_the_fixed_scratch():
    """An FP64 3P plan with M = 128 and P = 8 needs 4096 tiles x 15^3 x 8 bytes =
    110 MB of gridding blocks, more than the 32 MiB array: SE_ECAPACITY before
    anything is launched, and the plan still works through se_potential."""
    import paper_1712_04732_gb300 as se
    from paper_1712_04732_gb300 import _native as nat
    lib = nat.load()
    plan = se.Plan(3, 1.0, 8.0, 128, 8, "pkb", dtype=torch.float64)
    plan.reserve(1000)
    info = plan.info()
    blk = (info["tile"][0] + 7) * (info["tile"][1] + 7) * (info["tile"][2] + 7)
    assert info["n_tiles"] * blk * 8 > (32 << 20)
    x = torch.tensor(wl.uniform_positions(1000, 1.0, 5), device="cuda")
    q = torch.tensor(wl.uniform_charges(1000, 5), device="cuda")
    phi = torch.empty(1000, dtype=torch.float64, device="cuda")
    plan._sync_stream()
    assert lib.se_potential_noalloc(plan.handle, 1000, _ptr(x), _ptr(q), _ptr(phi), 0) == 9   # SE_ECAPACITY
    assert b"fixed scratch" in lib.se_last_error()
    ref = plan.potential(x, q)
    torch.cuda.synchronize()
    assert torch.isfinite(ref).all()
    plan.close()
