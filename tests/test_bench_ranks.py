"""The replica path of bench.py (one process per GPU, no collective on the data path):
the slowest replica's time, the sum of the applies every replica finished within the bar,
and the whole-job throughput, checked with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r: its timed region took 100 + 50 r ms and 12 - r of its 12 applies met the bar
        ms = bench.rank_max(dist, [100.0 + 50.0 * rank, 10.0 * (rank + 1)], "cpu")
        good = bench.rank_sum(dist, [12.0 - rank], "cpu")
        out.put((rank, ms, good, bench.whole_job(good[0], ms[0])))
    finally:
        dist.destroy_process_group()


def test_two_replicas_aggregate_max_time_and_summed_applies():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, ms, good, value in res:
        assert ms == [150.0, 20.0]  # the slowest replica decides the time
        assert good == [23.0]  # every replica's applies that met the bar
        assert value == pytest.approx(23.0 / 0.150)


def test_one_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.rank_max(None, [3.0, 1.0], "cpu") == [3.0, 1.0]
    assert bench.rank_sum(None, [5.0], "cpu") == [5.0]
    assert bench.whole_job(12.0, 300.0) == pytest.approx(40.0)


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    args = argparse.Namespace(steps=1, warmup=0, cpu_seconds=1.0)
    assert bench.run_reference(args, rank=1, world=2) is None


def test_profile_summaries_parse():
    """bench.py reads the DRAM traffic and instruction counts of the step kernels from the
    committed ncu summaries (and uses them only while the kernel source hash matches)."""
    sys.path.insert(0, ROOT)
    import re

    import bench

    for path in (bench.PROFILE, bench.PROFILE_RELAXED):
        txt = open(path).read()
        assert re.search(r"kernel_source_hash:\s*[0-9a-f]{16}", txt)
        assert re.search(r"dram_bytes_per_launch_full_size:\s*[0-9.eE+]+", txt)
        assert "smsp__inst_executed.sum" in txt
    assert len(bench.kernel_hash()) == 16
