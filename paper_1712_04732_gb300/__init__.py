"""GB300-native Spectral Ewald k-space library (sm_103a CUDA behind a C ABI).

Computes the Fourier-space part of the Ewald potential, and its forces, for
point charges with periodicity in 3, 2, 1 or 0 directions by the unified
Spectral Ewald method of Shamshirgar, Bagge & Tornberg (Alg. 4).  PyTorch is
used here only for device memory and streams; every step of the computation
runs in the CUDA library ``_build/libse_gb300.so`` (see ``include/se_gb300.h``).

    plan = Plan(D=0, L=1.0, xi=8.0, M=48, P=8, window="pkb", dtype=torch.float32)
    phi = plan.potential(x, q)                # x (N, 3), q (N,) CUDA tensors
    F, phi, E = plan.force(x, q, energy=True)
    E = energy(plan, x, q); E.backward()      # dE/dx = -F, dE/dq = phi
"""
from __future__ import annotations

import ctypes

import torch

from . import _native as nat
from ._native import SEError

__all__ = ["Plan", "Batch", "SEError", "potential", "energy", "params_from_tolerance", "measure_peak"]

_WINDOWS = {"gaussian": nat.SE_WIN_GAUSSIAN, "pkb": nat.SE_WIN_PKB}
_DTYPES = {torch.float32: nat.SE_F32, torch.float64: nat.SE_F64}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Plan:
    """One Spectral Ewald configuration on one GPU (``se_plan_create``).

    D: periodic directions (the first D axes); L: box side, or the three sides
    of a non-cubic box (each an even multiple of h = L_x / M); xi: Ewald
    splitting parameter; M: grid intervals along x; P: window support;
    window: "pkb" or "gaussian"; dtype: torch.float32 or torch.float64.
    Keyword overrides (Sec. 6 defaults otherwise): lam, s0, s_mt, n_l, nu,
    shape, aft_eps, tile, spread_mode, gather_mode, split (kernel variants),
    force_method (1: gradient of the window, 2: i k in the scaling; Sec. 7.2),
    fft_mode (1: cuFFT for every transform stage; 2: D = 1 free-direction transforms
    as line transforms), fft_sizes (1: free-direction
    transform lengths rounded up to 2-3-5-7-smooth sizes).
    """

    def __init__(self, D: int, L, xi: float, M: int, P: int, window: str = "pkb",
                 dtype=torch.float32, device=None, lam=None, s0=None, s_mt=None, n_l=None, nu=None,
                 shape=None, aft_eps=None, tile=None, spread_mode=None, gather_mode=None, split=None,
                 force_method=None, fft_mode=None, fft_sizes=None):
        self._lib = nat.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("the Spectral Ewald library runs on CUDA devices only")
        self.dtype = dtype
        sides = [float(v) for v in (L if hasattr(L, "__len__") else (L, L, L))]
        if len(sides) != 3:
            raise ValueError("L is one side or three sides")
        self.box = tuple(sides)
        self.L = sides[0] if sides[0] == sides[1] == sides[2] else self.box
        self.D, self.xi, self.M, self.P, self.window = D, float(xi), M, P, window
        o = nat.Opts()
        self._lib.se_opts_default(ctypes.byref(o))
        if lam is not None: o.lambda_ = lam
        if s0 is not None: o.s0 = s0
        if s_mt is not None: o.s_mt = s_mt
        if n_l is not None: o.n_l = n_l
        if nu is not None: o.nu = nu
        if shape is not None: o.shape = shape
        if aft_eps is not None: o.aft_eps = aft_eps
        if tile is not None: o.tile = tile
        if spread_mode is not None: o.spread_mode = spread_mode
        if gather_mode is not None: o.gather_mode = gather_mode
        if split is not None: o.split = split
        if force_method is not None: o.force_method = force_method
        if fft_mode is not None: o.fft_mode = fft_mode
        if fft_sizes is not None: o.fft_sizes = fft_sizes
        box = (ctypes.c_double * 3)(*self.box)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            nat.check(self._lib.se_plan_create(ctypes.byref(h), box, D, float(xi), M, P, _WINDOWS[window],
                                               _DTYPES[dtype], ctypes.byref(o)))
        self._h = h
        self._stream = None

    # ------------------------------------------------------------------ admin
    def close(self):
        if getattr(self, "_h", None):
            self._lib.se_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        i = nat.Info()
        nat.check(self._lib.se_plan_get_info(self._h, ctypes.byref(i)))
        out = {f: getattr(i, f) for f, _ in nat.Info._fields_}
        out["grid"] = tuple(i.grid)
        out["tile"] = tuple(i.tile)
        for f in ("M_v", "Mt_v", "s0_mt_v", "s_mt_v", "n_I", "L_v"):
            out[f] = tuple(getattr(i, f))
        return out

    def set_profiling(self, enable: bool = True):
        nat.check(self._lib.se_plan_set_profiling(self._h, int(bool(enable))))

    def profile(self) -> dict:
        """Accumulated per-stage milliseconds, profiled calls, library kernel launches."""
        ms = (ctypes.c_double * nat.SE_N_STAGES)()
        calls, launches = ctypes.c_int64(), ctypes.c_int64()
        nat.check(self._lib.se_plan_get_profile(self._h, ms, ctypes.byref(calls), ctypes.byref(launches)))
        return {"ms": dict(zip(nat.STAGES, list(ms))), "calls": calls.value, "launches": launches.value}

    def reserve(self, n: int):
        nat.check(self._lib.se_plan_reserve(self._h, int(n)))

    def check(self):
        nat.check(self._lib.se_plan_check(self._h))

    def _sync_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        if s != self._stream:
            nat.check(self._lib.se_plan_set_stream(self._h, ctypes.c_void_p(s)))
            self._stream = s

    def _args(self, x, q):
        if x.device != self.device or q.device != self.device:
            raise ValueError("x and q must live on the plan's device")
        if x.dtype != self.dtype or q.dtype != self.dtype:
            raise TypeError(f"x and q must be {self.dtype}")
        x = x.contiguous()
        q = q.contiguous()
        if x.dim() != 2 or x.shape[1] != 3 or q.shape != (x.shape[0],):
            raise ValueError("expected x of shape (N, 3) and q of shape (N,)")
        self._sync_stream()
        return x, q

    @staticmethod
    def _flags(add_self, check_neutral, sync_check):
        return ((nat.SE_ADD_SELF if add_self else 0) | (nat.SE_CHECK_NEUTRAL if check_neutral else 0)
                | (nat.SE_SYNC_CHECK if sync_check else 0))

    # ------------------------------------------------------------------ compute
    def potential(self, x, q, add_self=False, check_neutral=False, sync_check=False):
        """phi~^{DP,F} at the particles (``se_potential``)."""
        x, q = self._args(x, q)
        phi = torch.empty(x.shape[0], dtype=self.dtype, device=self.device)
        nat.check(self._lib.se_potential(self._h, x.shape[0], _ptr(x), _ptr(q), _ptr(phi),
                                         self._flags(add_self, check_neutral, sync_check)))
        return phi

    def force(self, x, q, add_self=False, energy=False, want_phi=True, check_neutral=False, sync_check=False,
              out=None):
        """(F, phi, E): F = -q grad phi (``se_force``); E = 1/2 sum q phi (FP64) or None.
        ``out`` = (F, phi, E) preallocated outputs (phi, E may be None)."""
        x, q = self._args(x, q)
        n = x.shape[0]
        if out is not None:
            F, phi, E = out
        else:
            F = torch.empty((n, 3), dtype=self.dtype, device=self.device)
            phi = torch.empty(n, dtype=self.dtype, device=self.device) if want_phi else None
            E = torch.empty((), dtype=torch.float64, device=self.device) if energy else None
        nat.check(self._lib.se_force(self._h, n, _ptr(x), _ptr(q), _ptr(F), _ptr(phi), _ptr(E),
                                     self._flags(add_self, check_neutral, sync_check)))
        return F, phi, E

    def vjp(self, x, q, g):
        """(dL/dx, dL/dq) for phi = A(x) q and cotangent g (``se_vjp``)."""
        x, q = self._args(x, q)
        g = g.to(self.dtype).contiguous()
        gx = torch.empty((x.shape[0], 3), dtype=self.dtype, device=self.device)
        gq = torch.empty(x.shape[0], dtype=self.dtype, device=self.device)
        nat.check(self._lib.se_vjp(self._h, x.shape[0], _ptr(x), _ptr(q), _ptr(g), _ptr(gx), _ptr(gq)))
        return gx, gq

    def real_space(self, x, q, rc, phi=None, F=None, accumulate=False):
        """Real-space part phi^R (and F^R) with cut-off rc (``se_real_space``)."""
        x, q = self._args(x, q)
        n = x.shape[0]
        if phi is None and F is None:
            phi = torch.empty(n, dtype=self.dtype, device=self.device)
            F = torch.empty((n, 3), dtype=self.dtype, device=self.device)
        nat.check(self._lib.se_real_space(self._h, n, _ptr(x), _ptr(q), float(rc), _ptr(phi), _ptr(F),
                                          nat.SE_ACCUMULATE if accumulate else 0))
        return phi, F

    def total(self, x, q, rc):
        """Full Ewald potential and force, Eq. (potential_split): Fourier part with
        the self term (se_force) plus the real-space part (se_real_space)."""
        F, phi, _ = self.force(x, q, add_self=True)
        self.real_space(x, q, rc, phi, F, accumulate=True)
        return phi, F

    def force_host(self, x, q, F, phi=None, energy=None, add_self=False):
        """``se_force`` with SE_HOST_IO on host tensors (copies inside the call;
        with page-locked tensors a repeated call replays a captured graph)."""
        self._sync_stream()
        flags = nat.SE_HOST_IO | (nat.SE_ADD_SELF if add_self else 0)
        nat.check(self._lib.se_force(self._h, x.shape[0], _ptr(x), _ptr(q), _ptr(F), _ptr(phi), _ptr(energy),
                                     flags))

    def potential_host(self, x, q, phi, add_self=False):
        """``se_potential`` with SE_HOST_IO on host tensors."""
        self._sync_stream()
        flags = nat.SE_HOST_IO | (nat.SE_ADD_SELF if add_self else 0)
        nat.check(self._lib.se_potential(self._h, x.shape[0], _ptr(x), _ptr(q), _ptr(phi), flags))


class Batch:
    """Many independent systems evaluated together (``se_batch_create``): per-system
    M and P from the rules of Sec. 6 for relative tolerance ``eps_rel``, autotuned
    kernel variants and one CUDA graph per call.  ``systems`` is a list of
    (N, D, L, xi) tuples; ``Q`` optional per-system sums of q^2.  ``form``:
    "auto" (the tuner chooses), "lines" (binning, gridding, merge and gathering
    of all systems in one launch per stage and support class, and the
    transforms of all systems in five launches; D = 3 and 2 only), "fused"
    (the same stages, each system's transforms in parallel graph branches) or
    "branches" (every system's own pipeline in parallel graph branches)."""

    _FORMS = {"auto": 0, "branches": nat.SE_BATCH_BRANCHES, "fused": nat.SE_BATCH_FUSED,
              "lines": nat.SE_BATCH_LINES}
    _FORM_NAMES = {1: "branches", 2: "fused", 3: "lines"}

    def __init__(self, systems, eps_rel=1e-5, window="pkb", dtype=torch.float32, device=None, Q=None,
                 autotune=True, form="auto"):
        self._lib = nat.load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.dtype = dtype
        n = len(systems)
        self.N = [int(s[0]) for s in systems]
        Na = (ctypes.c_int64 * n)(*self.N)
        Da = (ctypes.c_int * n)(*[int(s[1]) for s in systems])
        La = (ctypes.c_double * n)(*[float(s[2]) for s in systems])
        Xa = (ctypes.c_double * n)(*[float(s[3]) for s in systems])
        Qa = (ctypes.c_double * n)(*Q) if Q is not None else None
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            flags = (0 if autotune else nat.SE_BATCH_NO_AUTOTUNE) | self._FORMS[form]
            nat.check(self._lib.se_batch_create(ctypes.byref(h), n, Na, Da, La, Xa, Qa, float(eps_rel),
                                                _WINDOWS[window], _DTYPES[dtype], flags))
        self._h = h
        self._stream = None

    def close(self):
        if getattr(self, "_h", None):
            self._lib.se_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def form(self):
        """("lines" | "fused" | "branches", library kernels per call) of the captured graph."""
        f = ctypes.c_int()
        k = ctypes.c_int64()
        nat.check(self._lib.se_batch_get_form(self._h, ctypes.byref(f), ctypes.byref(k)))
        return self._FORM_NAMES[f.value], int(k.value)

    def system_info(self, i):
        inf = nat.Info()
        nat.check(self._lib.se_batch_get_system(self._h, i, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in nat.Info._fields_}

    def accuracy(self, i):
        """(phi, F) relative rms errors the autotuner measured for system i (-1: not measured)."""
        ep, ef = ctypes.c_double(), ctypes.c_double()
        nat.check(self._lib.se_batch_get_accuracy(self._h, i, ctypes.byref(ep), ctypes.byref(ef)))
        return ep.value, ef.value

    def _sync_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        if s != self._stream:
            nat.check(self._lib.se_batch_set_stream(self._h, ctypes.c_void_p(s)))
            self._stream = s

    def force(self, x, q, out=None, each=False):
        """(F, phi, E[nsys]) for the concatenated systems; ``each`` runs one plain
        se_force per system instead of the batched graph."""
        self._sync_stream()
        x = x.contiguous()
        q = q.contiguous()
        n = x.shape[0]
        if out is None:
            out = (torch.empty((n, 3), dtype=self.dtype, device=self.device),
                   torch.empty(n, dtype=self.dtype, device=self.device),
                   torch.empty(len(self.N), dtype=torch.float64, device=self.device))
        F, phi, E = out
        fn = self._lib.se_batch_force_each if each else self._lib.se_batch_force
        nat.check(fn(self._h, _ptr(x), _ptr(q), _ptr(F), _ptr(phi), _ptr(E)))
        return F, phi, E


class _PotentialFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, x, q):
        ctx.plan = plan
        ctx.save_for_backward(x, q)
        return plan.potential(x, q)

    @staticmethod
    def backward(ctx, g):
        x, q = ctx.saved_tensors
        gx, gq = ctx.plan.vjp(x, q, g)
        return None, gx, gq


class _EnergyFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, plan, x, q, add_self):
        F, phi, E = plan.force(x, q, add_self=add_self, energy=True)
        ctx.save_for_backward(F, phi)
        return E

    @staticmethod
    def backward(ctx, gE):
        F, phi = ctx.saved_tensors
        s = gE.to(F.dtype)
        return None, -F * s, phi * s, None


def potential(plan: Plan, x, q):
    """Differentiable phi~^{DP,F}(x; q): backward runs the adjoint kernel ``se_vjp``."""
    return _PotentialFn.apply(plan, x, q)


def energy(plan: Plan, x, q, add_self: bool = False):
    """Differentiable E = 1/2 sum q_m phi_m (FP64): dE/dx = -F, dE/dq = phi."""
    return _EnergyFn.apply(plan, x, q, add_self)


def params_from_tolerance(eps_rel: float, xi: float, L, Q: float = 0.0, window: str = "pkb", N: int = 0,
                          D: int = 3):
    """(M, P) from the rules of Sec. 6 for the relative rms tolerance eps_rel
    (``se_params_from_tolerance``).  ``L`` is the box side or the three sides;
    ``Q`` = sum q^2 (0: N / 3)."""
    lib = nat.load()
    box = (ctypes.c_double * 3)(*([float(L)] * 3 if isinstance(L, (int, float)) else [float(v) for v in L]))
    M, P = ctypes.c_int(), ctypes.c_int()
    nat.check(lib.se_params_from_tolerance(eps_rel, xi, int(N), Q, box, int(D), _WINDOWS[window], ctypes.byref(M),
                                           ctypes.byref(P)))
    return M.value, P.value


_PEAK_KINDS = {"fp32_fma": 0, "fp64_fma": 1, "smem_atomic_i32": 2, "smem_atomic_f32": 3}


def measure_peak(kind: str, iters: int):
    """Measured ceiling on the current device (``se_measure_peak``): flop/s for
    "fp32_fma" / "fp64_fma", shared-memory atomic updates/s for
    "smem_atomic_i32" / "smem_atomic_f32"; returns (rate, kernel ms)."""
    lib = nat.load()
    r, ms = ctypes.c_double(), ctypes.c_double()
    nat.check(lib.se_measure_peak(_PEAK_KINDS[kind], int(iters), ctypes.byref(r), ctypes.byref(ms)))
    return r.value, ms.value
