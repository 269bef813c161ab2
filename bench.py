#!/usr/bin/env python
"""Benchmark of the Spectral Ewald k-space path on GB300.

One step = one pass of the whole path (binning, gridding, FFT, scaling,
inverse FFT, gathering of phi and F, FP64 energy) over the free-space
workload: D = 0, N = 20000 charges uniform in [0,1)^3, q ~ U(-1,1) shifted to
zero sum, xi = 8, M = 48, extension lambda = 2 (M~ = 64, FFT (2 M~)^3 = 128^3),
PKB window P = 8.
`value` is the FP32 form (FP32 gridding/FFT/gathering, FP64 scaling tables and
energy); the FP64 form is reported beside it.  Inputs are resident on the
device when timing starts; L2 is flushed (256 MB write) before every timed step
and only the step is inside the CUDA events.  Each timed step replays a
captured CUDA graph of se_force.

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
WORKLOAD = "free_0p"
L2_FLUSH_BYTES = 256 << 20
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# FP32 FMA peak from unit counts and the maximum SM clock: 152 SMs x 128 lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the tile kernels on this workload,
# from one ncu --set full capture of this benchmark's FP32 step; reset to None whenever the
# kernel changes
NCU_TRAFFIC = {"spread": 664576, "gather": 1436160}


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--only", choices=["batch", "slab_2p", "wire_1p"], default=None,
                    help="time only the batched form or one of the larger workloads (profiling aid; "
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


def algorithmic_counts(P: int, nu: int, window: str):
    """Per-particle FMA counts of the tile kernels (PKB: Horner of degree nu for
    3P weights, their derivatives for the gradient):
    gridding P^3 + P^2 + 3 P nu, gathering phi + grad phi 4 P^3 + 3 P^2 + 6 P nu."""
    return {"spread": P ** 3 + P ** 2 + 3 * P * nu, "gather": 4 * P ** 3 + 3 * P ** 2 + 6 * P * nu}


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


def cpu_oracle_sample(x, q, targets, L, xi):
    """The FP64 oracle (direct free-space Ewald sum with forces) on the given targets."""
    from oracle import ewald
    phi, grad = ewald.fourier(0, x, q, L, xi, xt=x[targets])
    return phi, grad


def run_reference(a):
    """The oracle, as it stands, on the host cores: each step evaluates phi and F
    at a sample of 2000 targets of the workload (all 20000 sources)."""
    import numpy as np
    from paper_1712_04732_gb300 import workloads as wl
    rank, world, _ = dist_env()
    if rank != 0:
        return
    x, q, spec = wl.make(WORKLOAD, seed=1)
    ns = 2000
    idx = np.arange(ns)
    for _ in range(a.warmup):
        cpu_oracle_sample(x, q, idx, spec["L"], spec["xi"])
    t0 = time.perf_counter()
    for _ in range(a.steps):
        cpu_oracle_sample(x, q, idx, spec["L"], spec["xi"])
    dt = (time.perf_counter() - t0) / a.steps
    v = ns / dt
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "particles/s", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(spec),
            "cpu_baseline": {"value": v, "unit": "particles/s", "cores": cores, "kind": "oracle",
                             "cpu": cpu_model(),
                             "sample": f"phi+F at {ns} of {spec['N']} targets (all sources) per step, direct FP64 sum"},
            "e2e": {"value": v, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(spec):
    return {"workload": f"{WORKLOAD}: D={spec['D']} free space, N={spec['N']} uniform in [0,1)^3, "
                        f"q~U(-1,1) neutralised, xi={spec['xi']}, M={spec['M']}, lambda={spec['lam']} (M~=64, FFT 128^3), "
                        f"PKB P={spec['P']}, phi+F+energy",
            "l2": "flushed (256 MB write) before every timed step", "timing": "CUDA graph replay, CUDA events"}


def run_batch(se, wl, dev, flush, steps):
    """64 independent systems, N log-uniform in [1e3, 1e5], D alternating 3, 2,
    xi = 8 (N/1e4)^(1/3), PKB, per-system M and P from the Sec. 6 rules at
    relative tolerance 1e-5, FP32, phi + F: the autotuned batched graph (the
    tuner picks the multi-system or the per-system-branches form) against one
    plain se_force call per system, both timed with CUDA events after an L2
    flush; the two graph forms are also timed side by side without tuning."""
    import numpy as np
    import torch
    sysl = wl.batch_systems(64, seed=1)
    specs = [(len(q), D, 1.0, 8.0 * (len(q) / 1e4) ** (1.0 / 3.0)) for x, q, D in sysl]
    x = torch.tensor(np.concatenate([s[0] for s in sysl]), dtype=torch.float32, device=dev)
    q = torch.tensor(np.concatenate([s[1] for s in sysl]), dtype=torch.float32, device=dev)
    ntot = x.shape[0]
    t0 = time.perf_counter()
    b = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, device=dev)
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
    # the two graph forms side by side, default kernel variants
    for fname in ("fused", "branches"):
        bf = se.Batch(specs, eps_rel=1e-5, dtype=torch.float32, device=dev, autotune=False, form=fname)
        for _ in range(3):
            bf.force(x, q, out=out)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize(dev)
        for e0, e1 in ev:
            flush.zero_()
            e0.record()
            bf.force(x, q, out=out)
            e1.record()
        torch.cuda.synchronize(dev)
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
        res[f"untuned_{fname}"] = {"ms_per_step": ms, "value": ntot / (ms * 1e-3), "unit": "particles/s",
                                   "library_kernels_per_call": bf.form()[1]}
        bf.close()
    return res


def run_other_workloads(se, wl, dev, flush, steps, names=("slab_2p", "wire_1p")):
    """The FP32 step on the larger workloads (slab 1e5 and wire 1.2e6 particles),
    with the free-direction transform lengths rounded up to 2-3-5-7-smooth sizes
    (plan option fft_sizes): particles/s from graph replays after an L2 flush,
    and the gridding and gathering stages' algorithmic FLOP rate against the
    derived FP32 peak."""
    import torch
    out = {}
    for name in names:
        x_np, q_np, spec = wl.make(name, seed=1)
        n = len(q_np)
        plan = se.Plan(spec["D"], spec["L"], spec["xi"], spec["M"], spec["P"], spec["window"],
                       dtype=torch.float32, device=dev, lam=spec.get("lam"), fft_sizes=1)
        plan.reserve(n)
        x = torch.tensor(x_np, dtype=torch.float32, device=dev)
        q = torch.tensor(q_np, dtype=torch.float32, device=dev)
        res = (torch.empty((n, 3), device=dev), torch.empty(n, device=dev),
               torch.empty((), dtype=torch.float64, device=dev))
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            for _ in range(3):
                plan.force(x, q, energy=True, out=res)
        torch.cuda.current_stream(dev).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="thread_local"):
            plan.force(x, q, energy=True, out=res)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for e0, e1 in ev:
            flush.zero_()
            e0.record()
            g.replay()
            e1.record()
        torch.cuda.synchronize(dev)
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps
        plan.set_profiling(True)
        for _ in range(5):
            flush.zero_()
            plan.force(x, q, energy=True, out=res)
        torch.cuda.synchronize(dev)
        pr = plan.profile()
        plan.set_profiling(False)
        st = {k: v / pr["calls"] for k, v in pr["ms"].items()}
        cnt = algorithmic_counts(spec["P"], plan.info()["nu"], spec["window"])
        frac = {}
        for k in ("spread", "gather"):
            tf = 2.0 * cnt[k] * n / (st[k] * 1e-3) / 1e12
            frac[k] = {"tflops": tf, "frac_of_fp32_peak": tf / FP32_PEAK_TFLOPS}
        inf = plan.info()
        out[name] = {"particles": n, "ms_per_step": ms, "value": n / (ms * 1e-3), "unit": "particles/s",
                     "stage_ms": st, "alu": frac,
                     "transform_lengths": {"Mt": list(inf["Mt_v"]), "s0Mt": list(inf["s0_mt_v"]),
                                           "sMt": list(inf["s_mt_v"]),
                                           "rule": "free-direction lengths rounded up to 2-3-5-7-smooth sizes"}}
        plan.close()
    return out


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
    x_np, q_np, spec = wl.make(WORKLOAD, seed=rank + 1)
    N = spec["N"]
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    if a.only is not None:
        if a.only == "batch":
            res = {"batch_form": run_batch(se, wl, dev, flush, a.steps)}
        else:
            res = {"other_workloads": run_other_workloads(se, wl, dev, flush, a.steps, names=(a.only,))}
        if rank == 0:
            print(json.dumps(res), flush=True)
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    def make_form(dtype, force_method=1):
        plan = se.Plan(spec["D"], spec["L"], spec["xi"], spec["M"], spec["P"], spec["window"], dtype=dtype, device=dev,
                       lam=spec.get("lam"), force_method=force_method)
        plan.reserve(N)
        x = torch.tensor(x_np, dtype=dtype, device=dev)
        q = torch.tensor(q_np, dtype=dtype, device=dev)
        out = (torch.empty((N, 3), dtype=dtype, device=dev), torch.empty(N, dtype=dtype, device=dev),
               torch.empty((), dtype=torch.float64, device=dev))
        return plan, x, q, out

    def capture(plan, x, q, out):
        s = torch.cuda.Stream(device=dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            for _ in range(3):
                plan.force(x, q, energy=True, out=out)
        torch.cuda.current_stream(dev).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        try:
            with torch.cuda.graph(g, capture_error_mode="thread_local"):
                plan.force(x, q, energy=True, out=out)
            return g
        except Exception as exc:  # graph capture unavailable: time eager calls
            sys.stderr.write(f"graph capture failed ({exc}); timing eager calls\n")
            torch.cuda.synchronize(dev)
            return None

    def timed(plan, x, q, out, g, steps, warmup):
        step = (lambda: g.replay()) if g is not None else (lambda: plan.force(x, q, energy=True, out=out))
        for _ in range(warmup):
            flush.zero_()
            step()
        torch.cuda.synchronize(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for e0, e1 in ev:
            flush.zero_()
            e0.record()
            step()
            e1.record()
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        ms = max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps, dev)
        if world > 1:
            torch.distributed.barrier()
        return ms, wall

    # ---- FP32 form (the headline) -------------------------------------------------
    plan32, x32, q32, out32 = make_form(torch.float32)
    g32 = capture(plan32, x32, q32, out32)
    clocks = Clocks(local)
    ms32, wall32 = timed(plan32, x32, q32, out32, g32, a.steps, a.warmup)
    clk = clocks.stop()
    value = aggregate_throughput(N, world, ms32 * 1e-3)

    # ---- FP64 form ---------------------------------------------------------------
    plan64, x64, q64, out64 = make_form(torch.float64)
    g64 = capture(plan64, x64, q64, out64)
    k64 = max(3, min(a.steps, 200))
    ms64, _ = timed(plan64, x64, q64, out64, g64, k64, min(a.warmup, 10))

    # ---- FP32 form with forces by method 2 of Sec. 7.2 (i k in the scaling) --------
    planm2, xm2, qm2, outm2 = make_form(torch.float32, force_method=2)
    gm2 = capture(planm2, xm2, qm2, outm2)
    msm2, _ = timed(planm2, xm2, qm2, outm2, gm2, k64, min(a.warmup, 10))

    # ---- stage profile of the FP32 form (eager calls, events on the plan's stream) --
    plan32.set_profiling(True)
    l0 = plan32.profile()["launches"]
    kp = max(3, min(a.steps, 200))
    for _ in range(kp):
        flush.zero_()
        plan32.force(x32, q32, energy=True, out=out32)
    torch.cuda.synchronize(dev)
    prof = plan32.profile()
    plan32.set_profiling(False)
    launches_per_step = (prof["launches"] - l0) / kp
    stage_ms = {k: v / prof["calls"] for k, v in prof["ms"].items()}
    info = plan32.info()
    counts = algorithmic_counts(spec["P"], info["nu"], spec["window"])
    ours = {k: stage_ms[k] for k in ("bin", "spread", "merge", "scale", "gather")}
    dom = max(ours, key=ours.get)
    if dom in ("spread", "gather"):
        flop = 2.0 * counts[dom] * N
        ach = flop / (stage_ms[dom] * 1e-3) / 1e12
        roof = {"kernel": "k_gather_flat<float,8,6,true>" if dom == "gather" else "k_spread_cl<float,8,6>",
                "bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP32_PEAK_TFLOPS, "traffic": NCU_TRAFFIC.get(dom),
                "per_launch": f"{flop:.3e} flop ({counts[dom]} FMA/particle x {N})",
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
    else:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"hbm_gbs": 6800.0}
        roof = {"kernel": dom, "bound": "hbm", "achieved": None, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": None, "traffic": None}
    # spread/gather GB/s on algorithmic bytes (16 B in per particle, 16 B out, grid once),
    # and as a fraction of the measured copy bandwidth (these stages are compute kernels:
    # 58 and 120 flop per algorithmic byte, so the fraction is small by construction)
    grid_bytes = 4 * info["Mt"] ** 3
    sg_bytes = N * (16 + 16 + 8) + 2 * grid_bytes
    sg_gbs = sg_bytes / ((stage_ms["spread"] + stage_ms["merge"] + stage_ms["gather"]) * 1e-3) / 1e9
    hbm_gbs = 6800.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            hbm_gbs = float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        pass

    # ---- end to end through the C ABI with host buffers ---------------------------
    xh = torch.tensor(x_np, dtype=torch.float32).pin_memory()
    qh = torch.tensor(q_np, dtype=torch.float32).pin_memory()
    Fh = torch.empty((N, 3), dtype=torch.float32).pin_memory()
    ph = torch.empty(N, dtype=torch.float32).pin_memory()
    eh = torch.empty((), dtype=torch.float64).pin_memory()
    ke = max(3, min(a.steps, 200))
    for _ in range(min(a.warmup, 5)):
        plan32.force_host(xh, qh, Fh, ph, eh)
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(ke):
        plan32.force_host(xh, qh, Fh, ph, eh)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / ke, dev)

    line = {"metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": _config(spec),
            "fp64_form": {"value": aggregate_throughput(N, world, ms64 * 1e-3), "unit": "particles/s", "ms_per_step": ms64,
                          "steps": k64, "speedup_fp32_over_fp64": ms64 / ms32},
            "force_method_2": {"value": aggregate_throughput(N, world, msm2 * 1e-3), "unit": "particles/s",
                               "ms_per_step": msm2, "steps": k64, "dtype": "f32",
                               "what": "forces by i k in the scaling (Sec. 7.2 method 2): four inverse transforms"},
            "roofline": roof,
            "stage_ms": stage_ms,
            "spread_gather_gbs": sg_gbs,
            "spread_gather_hbm_frac": {"value": sg_gbs / hbm_gbs, "peak_gbs": hbm_gbs,
                                       "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy), else 6800 GB/s"},
            "e2e": {"value": aggregate_throughput(N, world, e2e_s), "unit": "particles/s", "h2d_bytes_per_step": N * 16,
                    "d2h_bytes_per_step": N * 16 + 8, "api": "se_force with SE_HOST_IO (pinned host buffers)"},
            "gpu_launches": int(round(launches_per_step * a.steps)),
            "gpu_launches_per_step": launches_per_step,
            "clocks": clk, "wall_s_timed_region": wall32}

    # ---- batched independent systems: one CUDA graph vs one se_force per system ---
    if not a.no_batch:
        line["batch_form"] = run_batch(se, wl, dev, flush, min(a.steps, 50))
        line["other_workloads"] = run_other_workloads(se, wl, dev, flush, min(a.steps, 20))

    # ---- CPU baseline and accuracy (rank 0, one GPU only) -------------------------
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        idx = np.arange(N)
        t0 = time.perf_counter()
        pa, ga = cpu_oracle_sample(x_np, q_np, idx, spec["L"], spec["xi"])
        tc = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(idx) / tc, "unit": "particles/s",
                                "cores": len(os.sched_getaffinity(0)), "kind": "oracle", "cpu": cpu_model(),
                                "sample": f"phi+F at all {N} targets, one pass of the direct FP64 sum (oracle A)"}
        acc = {}
        for name, out in (("fp32", out32), ("fp64", out64), ("fp32_method2", outm2)):
            F = out[0].double().cpu().numpy()
            phi = out[1].double().cpu().numpy()
            acc[name] = {"phi": float(np.linalg.norm(phi - pa) / np.linalg.norm(pa)),
                         "F": float(np.linalg.norm(F + q_np[:, None] * ga) / np.linalg.norm(q_np[:, None] * ga))}
        line["accuracy_vs_oracle"] = acc
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
