#!/usr/bin/env python
"""Benchmark of the Spectral Ewald k-space path on GB300.

One step = one pass of the whole path (binning, gridding, FFT / AFT, scaling,
inverse FFT / AIFT, gathering of phi and F, FP64 energy) over the headline
workload, the largest single-GPU one: the singly periodic wire, D = 1,
N = 1.2e6 charges (1e6 uniform in the unit box plus 2e5 in ten Gaussian clouds
of sigma 0.03), q ~ U(-1,1) neutralised, xi = 32, M = 128, PKB window P = 8,
free-direction transform lengths rounded up to 2-3-5-7-smooth sizes
(M~ = 150, s0 M~ = 378, s M~ = 350).
`value` is the FP32 form (FP32 gridding/FFT/gathering, FP64 scaling tables and
energy); the FP64 form of the same plan is reported beside it.  Inputs are
resident on the device when timing starts; L2 is flushed (256 MB write) before
every timed step and only the step is inside the CUDA events.  Each timed step
replays a captured CUDA graph of se_force.  The free-space workload (D = 0,
N = 20000, M = 48) follows as a second line in `free_0p`, the slab and the
batch of 64 systems after it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank runs its own copy of the workload (independent
replicas; the path has no exchange step) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particles/s (phi+F) at rms rel err <=1e-5, FP32 vs FP64 form; spread/gather GB/s"
WORKLOAD = "wire_1p"
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of the tile kernels on the
# headline workload, from one ncu capture of this benchmark's FP32 step
# (profiles/wire_1p_tile_kernels.md); the gridding stage is two launches (light
# tiles 39.00 MB, heavy tiles 4.81 MB).  Set to None when a kernel changes.
NCU_TRAFFIC = {"spread": 43.818e6, "gather": 61.208e6}
# l1tex__data_pipe_lsu_wavefronts_mem_shared.sum of the same capture: shared-memory
# wavefronts per stage (gridding: light 33.686e6 + heavy 4.746e6 tiles; gathering
# 53.781e6), the unit both tile kernels are bound by
NCU_SMEM_WAVEFRONTS = {"spread": 38.432e6, "gather": 53.781e6}
# targets of the oracle's sample on the headline workload (about 20 s of the
# host's cores through the xi route of oracle A)
CPU_TARGETS = 128


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-form", choices=["auto", "lines", "fused", "branches"], default="auto",
                    help="execution form of the batched systems (auto: the autotuner's choice)")
    ap.add_argument("--only", choices=["batch", "slab_2p", "wire_1p", "free_0p"], default=None,
                    help="time only the batched form or one workload's FP32 step (profiling aid; "
                         "prints its own JSON line)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(v: float, device) -> float:
    """Largest value of v over the ranks of the default process group (v itself
    without one): the timing rule takes the slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(n_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job particles per second: every rank processes its own replica."""
    return world * n_per_rank / seconds


def algorithmic_counts(P: int, nu: int):
    """Per-particle FMA counts of the tile kernels (PKB: Horner of degree nu):
    gridding P^3 + P^2 + 3 P nu (P^3 products w_xy w_z, P^2 products q w_x w_y,
    3 P window values); gathering phi + grad phi by the separable contraction
    2 P^3 (x with W and W') + 3 P^2 (y) + 4 P (z) + 6 P nu (W and W' on three
    axes).  The naive per-point count of the gathering, 4 P^3 + 3 P^2 + 6 P nu,
    is reported beside it."""
    return {"spread": P ** 3 + P ** 2 + 3 * P * nu,
            "gather": 2 * P ** 3 + 3 * P ** 2 + 4 * P + 6 * P * nu,
            "gather_naive": 4 * P ** 3 + 3 * P ** 2 + 6 * P * nu,
            "spread_updates": P ** 3}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.12)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                c = [s.strip() for s in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    rows.append((float(c[1]), float(c[2]), c[5:9]))
                except ValueError:
                    continue
        os.unlink(self.f.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for _, _, r in rows for n, v in zip(names, r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm implementer
    and part codes), else the platform's processor string."""
    import platform
    try:
        info = {}
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if ":" in line:
                    k, v = line.split(":", 1)
                    info.setdefault(k.strip(), v.strip())
        if info.get("model name"):
            return info["model name"]
        if info.get("CPU implementer"):
            return f"implementer {info['CPU implementer']} part {info.get('CPU part', '?')} ({platform.machine()})"
    except OSError:
        pass
    return platform.processor() or platform.machine()


def oracle_sample_targets(x, spec, k, seed=7):
    """A fixed sample of k targets: half drawn from the uniform particles, half
    from the clustered ones (the last sixth of a clustered workload)."""
    import numpy as np
    g = np.random.default_rng(seed)
    n = len(x)
    if spec.get("clustered"):
        nb = n // 6
        a = g.choice(n - nb, size=k // 2, replace=False)
        b = (n - nb) + g.choice(nb, size=k - k // 2, replace=False)
        return np.sort(np.concatenate([a, b]))
    return np.sort(g.choice(n, size=min(k, n), replace=False))


def cpu_oracle(spec, x, q, targets):
    """Oracle A (FP64, plain C on the host cores) at the given targets: the 1P
    and 2P sums through the splitting-parameter independence of the total
    potential (Sec. 2), the 0P direct sum, the 3P k-sum."""
    from oracle import ewald
    if spec["D"] in (1, 2):
        return ewald.fourier_xi_route(spec["D"], x, q, spec["L"], spec["xi"], xt=x[targets])
    return ewald.fourier(spec["D"], x, q, spec["L"], spec["xi"], xt=x[targets])


def run_reference(a):
    """The oracle, as it stands, on the host cores, on the headline workload:
    each step evaluates phi and F at a sample of targets against all 1.2e6
    sources (oracle A, xi route)."""
    from paper_1712_04732_gb300 import workloads as wl
    rank, world, _ = dist_env()
    if rank != 0:
        return
    x, q, spec = wl.make(WORKLOAD, seed=1)
    nt = max(1, min(8, 1200 // max(1, a.steps + a.warmup)))
    idx = oracle_sample_targets(x, spec, nt, seed=11)
    for _ in range(a.warmup):
        cpu_oracle(spec, x, q, idx)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        cpu_oracle(spec, x, q, idx)
    dt = (time.perf_counter() - t0) / a.steps
    v = nt / dt
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "particles/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(spec),
            "cpu_baseline": {"value": v, "unit": "particles/s", "cores": cores, "kind": "oracle",
                             "cpu": cpu_model(),
                             "sample": f"phi+F at {nt} of {spec['N']} targets (half of them in the clouds) "
                                       f"per step against all sources, oracle A through xi-independence, FP64"},
            "e2e": {"value": v, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(spec):
    return {"workload": f"{WORKLOAD}: D={spec['D']} (x periodic), N={spec['N']} (1e6 uniform in [0,1)^3 + 2e5 in 10 "
                        f"Gaussian clouds, sigma 0.03), q~U(-1,1) neutralised, xi={spec['xi']}, M={spec['M']}, "
                        f"PKB P={spec['P']}, transform lengths 2-3-5-7-smooth (M~=150, s0M~=378, sM~=350), "
                        f"phi+F+energy",
            "l2": "flushed (256 MB write) before every timed step", "timing": "CUDA graph replay, CUDA events"}


def measure_peaks(se, dev, local):
    """FP32 / FP64 FMA and shared-memory atomic ceilings measured on this GPU
    (about a third of a second each), with the SM clock sampled meanwhile."""
    import torch
    clocks = Clocks(local)
    out = {}
    for kind, iters in (("fp32_fma", 300000), ("fp64_fma", 6000), ("smem_atomic_i32", 250000),
                        ("smem_atomic_f32", 100000)):
        rate, ms = se.measure_peak(kind, iters)
        out[kind] = {"value": rate / 1e12, "unit": "TFLOP/s" if "fma" in kind else "Tupdates/s", "kernel_ms": ms}
    torch.cuda.synchronize(dev)
    out["clocks"] = clocks.stop()
    out["how"] = ("se_measure_peak: every SM filled with resident warps; FMA: 8 independent chains a = a b + c "
                  "per thread; atomics: each lane adds to its own shared-memory word, 32 banks per warp")
    return out


def time_graph_steps(g, flush, steps, warmup, dev, world):
    import torch
    for _ in range(warmup):
        flush.zero_()
        g.replay()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for e0, e1 in ev:
        flush.zero_()
        e0.record()
        g.replay()
        e1.record()
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    ms = max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps, dev)
    if world > 1:
        torch.distributed.barrier()
    return ms, wall


class Form:
    """One plan of a workload with device-resident inputs and outputs, and its
    se_force call captured in a CUDA graph."""

    def __init__(self, se, spec, x_np, q_np, dtype, dev, **kw):
        import torch
        self.N = len(q_np)
        self.plan = se.Plan(spec["D"], spec["L"], spec["xi"], spec["M"], kw.pop("P", spec["P"]), spec["window"],
                            dtype=dtype, device=dev, lam=spec.get("lam"), **kw)
        self.plan.reserve(self.N)
        self.x = torch.tensor(x_np, dtype=dtype, device=dev)
        self.q = torch.tensor(q_np, dtype=dtype, device=dev)
        self.out = (torch.empty((self.N, 3), dtype=dtype, device=dev), torch.empty(self.N, dtype=dtype, device=dev),
                    torch.empty((), dtype=torch.float64, device=dev))
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            for _ in range(3):
                self.step_eager()
        torch.cuda.current_stream(dev).wait_stream(s)
        self.g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.g, capture_error_mode="thread_local"):
            self.step_eager()

    def step_eager(self):
        self.plan.force(self.x, self.q, energy=True, out=self.out)

    def stage_profile(self, flush, calls, dev):
        """Per-stage milliseconds from CUDA events on the plan's stream (eager
        calls of the same kernels, same launch configuration), and the library
        kernels launched per call."""
        import torch
        self.plan.set_profiling(True)
        l0 = self.plan.profile()["launches"]
        for _ in range(calls):
            flush.zero_()
            self.step_eager()
        torch.cuda.synchronize(dev)
        pr = self.plan.profile()
        self.plan.set_profiling(False)
        return {k: v / pr["calls"] for k, v in pr["ms"].items()}, (pr["launches"] - l0) / calls

    def e2e(self, x_np, q_np, calls, warmup, dev, world):
        """particles/s through se_force with SE_HOST_IO on page-locked host
        buffers: copies of x, q in and phi, F, E out inside every call."""
        import torch
        dt = self.x.dtype
        xh = torch.tensor(x_np, dtype=dt).pin_memory()
        qh = torch.tensor(q_np, dtype=dt).pin_memory()
        Fh = torch.empty((self.N, 3), dtype=dt).pin_memory()
        ph = torch.empty(self.N, dtype=dt).pin_memory()
        eh = torch.empty((), dtype=torch.float64).pin_memory()
        for _ in range(warmup):
            self.plan.force_host(xh, qh, Fh, ph, eh)
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(calls):
            self.plan.force_host(xh, qh, Fh, ph, eh)
        sec = max_over_ranks((time.perf_counter() - t0) / calls, dev)
        es = dt.itemsize
        return {"value": aggregate_throughput(self.N, world, sec), "unit": "particles/s",
                "h2d_bytes_per_step": self.N * 4 * es, "d2h_bytes_per_step": self.N * 4 * es + 8,
                "api": "se_force with SE_HOST_IO (page-locked host buffers)", "calls": calls}

    def result(self):
        F = self.out[0].double().cpu().numpy()
        phi = self.out[1].double().cpu().numpy()
        return F, phi

    def close(self):
        self.plan.close()


def rooflines(stage_ms, N, P, nu, peaks, traffic):
    """Roofline entries of the gridding and gathering kernels: algorithmic FLOP
    per launch over the launch's CUDA-event time against the measured FP32 FMA
    ceiling; for gridding also the P^3 shared-memory updates per particle against
    the measured integer-atomic ceiling."""
    cnt = algorithmic_counts(P, nu)
    fp32 = peaks["fp32_fma"]["value"]
    out = {}
    for k, kern in (("spread", f"k_spread_cl_f32fast<{P},{nu}>"), ("gather", f"k_gather_tile_f32fast<{P},{nu},true>")):
        sec = stage_ms[k] * 1e-3
        flop = 2.0 * cnt[k] * N
        ach = flop / sec / 1e12
        e = {"kernel": kern, "bound": "alu", "achieved": ach, "peak": fp32, "unit": "TFLOP/s", "frac": ach / fp32,
             "traffic": traffic.get(k), "launch_ms": stage_ms[k],
             "traffic_what": "bytes per stage, dram read + write, one cold-cache ncu capture"
                             + (" (two launches: light and heavy tiles)" if k == "spread" else ""),
             "per_launch": f"{flop:.4e} flop ({cnt[k]} FMA/particle x {N})",
             "peak_source": "measured: se_measure_peak FP32 FMA chains on this GPU (of measured)"}
        wf = NCU_SMEM_WAVEFRONTS.get(k)
        if wf:
            # one wavefront per clock per SM: the measured integer-atomic ceiling
            # (32 distinct-bank updates = one wavefront) divided by 32
            pk = peaks["smem_atomic_i32"]["value"] * 1e12 / 32.0
            e["smem_pipe"] = {"achieved": wf / sec, "peak": pk, "unit": "wavefronts/s", "frac": wf / sec / pk,
                              "wavefronts_per_stage": wf,
                              "what": "shared-memory wavefronts (ncu, same kernels) over the stage time, against "
                                      "one wavefront per clock per SM (measured atomic ceiling / 32)"}
        if k == "spread":
            upd = cnt["spread_updates"] * N / sec / 1e12
            e["atomic_updates"] = {"achieved": upd, "peak": peaks["smem_atomic_i32"]["value"], "unit": "Tupdates/s",
                                   "frac": upd / peaks["smem_atomic_i32"]["value"],
                                   "what": "P^3 fixed-point shared-memory atomic adds per particle"}
        else:
            e["naive_count"] = {"fma_per_particle": cnt["gather_naive"],
                                "achieved": 2.0 * cnt["gather_naive"] * N / sec / 1e12}
        out[k] = e
    return out


def accuracy(F, phi, q, idx, pa, ga):
    import numpy as np
    Fa = -q[idx, None] * ga
    return {"phi": float(np.linalg.norm(phi[idx] - pa) / np.linalg.norm(pa)),
            "F": float(np.linalg.norm(F[idx] - Fa) / np.linalg.norm(Fa)),
            "phi_max_abs_over_rms": float(np.abs(phi[idx] - pa).max() / np.sqrt(np.mean(pa ** 2))),
            "targets": int(len(idx))}


def run_free_space(se, wl, dev, flush, steps, warmup, world, rank, with_cpu):
    """The free-space workload (D = 0, N = 20000, M = 48, lambda = 2, PKB P = 8):
    FP32 form, FP64 form, FP32 with forces by method 2 of Sec. 7.2, e2e, and the
    direct sum on all targets (oracle A) for accuracy and the CPU baseline."""
    import numpy as np
    import torch
    x_np, q_np, spec = wl.make("free_0p", seed=rank + 1)
    N = spec["N"]
    out = {"workload": f"free_0p: D=0, N={N} uniform, q~U(-1,1) neutralised, xi={spec['xi']}, M={spec['M']}, "
                       f"lambda={spec['lam']} (M~=64, FFT 128^3), PKB P={spec['P']}, phi+F+energy"}
    forms = {}
    for name, dt, kw in (("fp32", torch.float32, {}), ("fp64", torch.float64, {}),
                         ("fp32_method2", torch.float32, {"force_method": 2})):
        f = Form(se, spec, x_np, q_np, dt, dev, **kw)
        ms, _ = time_graph_steps(f.g, flush, steps, warmup, dev, world)
        out[name] = {"value": aggregate_throughput(N, world, ms * 1e-3), "unit": "particles/s", "ms_per_step": ms,
                     "steps": steps}
        forms[name] = f
    out["speedup_fp32_over_fp64"] = out["fp64"]["ms_per_step"] / out["fp32"]["ms_per_step"]
    st, lps = forms["fp32"].stage_profile(flush, 50, dev)
    out["stage_ms"] = st
    out["library_kernels_per_step"] = lps
    out["e2e"] = forms["fp32"].e2e(x_np, q_np, 100, 5, dev, world)
    if with_cpu:
        idx = np.arange(N)
        t0 = time.perf_counter()
        pa, ga = cpu_oracle(spec, x_np, q_np, idx)
        tc = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": N / tc, "unit": "particles/s", "cores": len(os.sched_getaffinity(0)),
                               "kind": "oracle", "cpu": cpu_model(),
                               "sample": f"phi+F at all {N} targets, one pass of the direct FP64 sum (oracle A)"}
        out["accuracy_vs_oracle"] = {k: accuracy(*forms[k].result(), q_np, idx, pa, ga) for k in forms}
    for f in forms.values():
        f.close()
    return out


def run_slab(se, wl, dev, flush, steps, warmup, world):
    """The slab (D = 2, N = 1e5, M = 64, xi = 16) in FP32 at P = 8, the support
    whose forces meet 1e-5 against the direct sum (P + 2 rule of Sec. 7.2)."""
    import torch
    x_np, q_np, spec = wl.make("slab_2p", seed=1)
    f = Form(se, spec, x_np, q_np, torch.float32, dev, P=8, fft_sizes=1)
    ms, _ = time_graph_steps(f.g, flush, steps, warmup, dev, world)
    st, lps = f.stage_profile(flush, 20, dev)
    inf = f.plan.info()
    f.close()
    return {"particles": spec["N"], "P": 8, "ms_per_step": ms, "value": aggregate_throughput(spec["N"], world, ms * 1e-3),
            "unit": "particles/s", "stage_ms": st,
            "transform_lengths": {"Mt": list(inf["Mt_v"]), "s0Mt": list(inf["s0_mt_v"]), "sMt": list(inf["s_mt_v"])}}


def run_batch(se, wl, dev, flush, steps, form="auto"):
    """64 independent systems, N log-uniform in [1e3, 1e5], D alternating 3, 2,
    xi = 8 (N/1e4)^(1/3), PKB, per-system M and P from the Sec. 6 rules at
    relative tolerance 1e-5, FP32, phi + F: the autotuned batched graph against
    one plain se_force call per system, both timed with CUDA events after an L2
    flush; the two graph forms are also timed side by side without tuning."""
    import numpy as np
    import torch
    sysl = wl.batch_systems(64, seed=1)
    specs = [(len(q), D, 1.0, 8.0 * (len(q) / 1e4) ** (1.0 / 3.0)) for x, q, D in sysl]
    x = torch.tensor(np.concatenate([s[0] for s in sysl]), dtype=torch.float32, device=dev)
    q = torch.tensor(np.concatenate([s[1] for s in sysl]), dtype=torch.float32, device=dev)
    ntot = x.shape[0]
    t0 = time.perf_counter()
    b = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, device=dev, form=form)
    out = (torch.empty((ntot, 3), device=dev), torch.empty(ntot, device=dev),
           torch.empty(len(specs), dtype=torch.float64, device=dev))
    b.force(x, q, out=out)                          # autotune + capture
    torch.cuda.synchronize(dev)
    setup_s = time.perf_counter() - t0
    res = {}
    for name, each in (("graph", False), ("per_system", True)):
        for _ in range(3):
            b.force(x, q, out=out, each=each)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize(dev)
        with torch.cuda.nvtx.range(f"batch_{name}"):          # lets a profiler select these launches
            for e0, e1 in ev:
                flush.zero_()
                e0.record()
                b.force(x, q, out=out, each=each)
                e1.record()
            torch.cuda.synchronize(dev)
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
        res[name] = {"ms_per_step": ms, "value": ntot / (ms * 1e-3), "unit": "particles/s"}
    Ms = [b.system_info(i)["M"] for i in range(len(specs))]
    Ps = [b.system_info(i)["P"] for i in range(len(specs))]
    form, kernels = b.form()
    b.close()
    res.update({"systems": len(specs), "particles": ntot, "M_range": [min(Ms), max(Ms)],
                "P_range": [min(Ps), max(Ps)], "setup_s_incl_autotune": setup_s,
                "form": form, "library_kernels_per_call": kernels,
                "speedup_graph_over_per_system": res["per_system"]["ms_per_step"] / res["graph"]["ms_per_step"]})
    return res


def run_ours(a):
    import numpy as np
    import torch

    import paper_1712_04732_gb300 as se
    from paper_1712_04732_gb300 import build as bld
    from paper_1712_04732_gb300 import workloads as wl

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    bld.build()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    if a.only is not None:
        if a.only == "batch":
            res = {"batch_form": run_batch(se, wl, dev, flush, a.steps, a.batch_form)}
        elif a.only == "slab_2p":
            res = {"slab_2p": run_slab(se, wl, dev, flush, a.steps, a.warmup, world)}
        elif a.only == "free_0p":
            x_np, q_np, spec = wl.make("free_0p", seed=rank + 1)
            f = Form(se, spec, x_np, q_np, torch.float32, dev)
            ms, _ = time_graph_steps(f.g, flush, a.steps, a.warmup, dev, world)
            stage_ms, _ = f.stage_profile(flush, max(3, min(a.steps, 20)), dev)
            res = {"free_0p": {"ms_per_step": ms, "value": spec["N"] / (ms * 1e-3), "stage_ms": stage_ms}}
            f.close()
        else:
            x_np, q_np, spec = wl.make(WORKLOAD, seed=rank + 1)
            f = Form(se, spec, x_np, q_np, torch.float32, dev, fft_sizes=1)
            ms, _ = time_graph_steps(f.g, flush, a.steps, a.warmup, dev, world)
            stage_ms, _ = f.stage_profile(flush, max(3, min(a.steps, 20)), dev)
            res = {"wire_1p": {"ms_per_step": ms, "value": spec["N"] / (ms * 1e-3), "stage_ms": stage_ms}}
            f.close()
        if rank == 0:
            print(json.dumps(res), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    peaks = measure_peaks(se, dev, local)

    # ---- headline: the wire workload, FP32 form ------------------------------------
    x_np, q_np, spec = wl.make(WORKLOAD, seed=rank + 1)
    N = spec["N"]
    f32 = Form(se, spec, x_np, q_np, torch.float32, dev, fft_sizes=1)
    clocks = Clocks(local)
    ms32, wall32 = time_graph_steps(f32.g, flush, a.steps, a.warmup, dev, world)
    clk = clocks.stop()
    value = aggregate_throughput(N, world, ms32 * 1e-3)

    # ---- FP64 form of the same plan --------------------------------------------------
    f64 = Form(se, spec, x_np, q_np, torch.float64, dev, fft_sizes=1)
    k64 = max(3, min(a.steps, 50))
    ms64, _ = time_graph_steps(f64.g, flush, k64, min(a.warmup, 5), dev, world)

    # ---- stage profile and roofline of the FP32 form -----------------------------------
    kp = max(3, min(a.steps, 50))
    stage_ms, launches_per_step = f32.stage_profile(flush, kp, dev)
    info = f32.plan.info()
    roofs = rooflines(stage_ms, N, spec["P"], info["nu"], peaks, NCU_TRAFFIC)
    dom = "gather" if stage_ms["gather"] >= stage_ms["spread"] else "spread"
    # spread/gather GB/s on algorithmic bytes (16 B in per particle, 16 B out, the
    # grid written once and read once), against the measured copy bandwidth
    grid_bytes = 4 * info["grid"][0] * info["grid"][1] * info["grid"][2]
    sg_bytes = N * (16 + 16) + 2 * grid_bytes
    sg_gbs = sg_bytes / ((stage_ms["spread"] + stage_ms["merge"] + stage_ms["gather"]) * 1e-3) / 1e9
    hbm_gbs, hbm_src = 6800.0, "fallback 6800 GB/s"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            hbm_gbs, hbm_src = float(json.load(fh)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (copy), of measured"
    except (OSError, KeyError, ValueError):
        pass

    # ---- end to end through the C ABI with host buffers ---------------------------
    e2e = f32.e2e(x_np, q_np, max(3, min(a.steps, 30)), 3, dev, world)

    line = {"metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config(spec),
            "fp64_form": {"value": aggregate_throughput(N, world, ms64 * 1e-3), "unit": "particles/s",
                          "ms_per_step": ms64, "steps": k64, "speedup_fp32_over_fp64": ms64 / ms32},
            "roofline": dict(roofs[dom], dominant=dom),
            "roofline_other": roofs["spread" if dom == "gather" else "gather"],
            "measured_peaks": peaks,
            "stage_ms": stage_ms,
            "spread_gather_gbs": sg_gbs,
            "spread_gather_hbm_frac": {"value": sg_gbs / hbm_gbs, "peak_gbs": hbm_gbs, "peak_source": hbm_src},
            "e2e": e2e,
            "gpu_launches": int(round(launches_per_step * a.steps)),
            "gpu_launches_per_step": launches_per_step,
            "clocks": clk, "wall_s_timed_region": wall32}

    # ---- CPU baseline and accuracy on the headline workload (rank 0, one GPU) ------
    with_cpu = rank == 0 and world == 1 and not a.no_cpu_baseline
    if with_cpu:
        idx = oracle_sample_targets(x_np, spec, CPU_TARGETS)
        t0 = time.perf_counter()
        pa, ga = cpu_oracle(spec, x_np, q_np, idx)
        tc = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(idx) / tc, "unit": "particles/s",
                                "cores": len(os.sched_getaffinity(0)), "kind": "oracle", "cpu": cpu_model(),
                                "sample": f"phi+F at {len(idx)} of {N} targets (half in the clouds) against all "
                                          f"sources, oracle A through xi-independence (Sec. 2), FP64, one pass"}
        line["accuracy_vs_oracle"] = {"fp32": accuracy(*f32.result(), q_np, idx, pa, ga),
                                      "fp64": accuracy(*f64.result(), q_np, idx, pa, ga)}
    f32.close()
    f64.close()

    # ---- the other workloads ----------------------------------------------------------
    if not a.no_batch:
        line["free_0p"] = run_free_space(se, wl, dev, flush, min(a.steps, 200), min(a.warmup, 10), world, rank,
                                         with_cpu)
        line["slab_2p"] = run_slab(se, wl, dev, flush, min(a.steps, 50), min(a.warmup, 5), world)
        line["batch_form"] = run_batch(se, wl, dev, flush, min(a.steps, 50), a.batch_form)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
