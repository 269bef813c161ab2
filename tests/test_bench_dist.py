"""The multi-rank logic of bench.py on CPU: two gloo ranks, each timing its own
replica, agree on the slowest rank's time and on the whole-job throughput."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(1.5 + rank, torch.device("cpu"))
    out[rank] = (ms, bench.aggregate_throughput(20000, world, ms * 1e-3))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_throughput_aggregates():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        ms, v = out[r]
        assert ms == pytest.approx(2.5)
        assert v == pytest.approx(2 * 20000 / 2.5e-3)


def test_single_process_is_its_own_maximum():
    import bench
    assert bench.max_over_ranks(3.25, torch.device("cpu")) == 3.25


def test_reference_arm_prints_the_contract_line():
    """``bench.py --impl reference`` runs the oracle on the host cores and prints
    one JSON line with the base contract's keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
