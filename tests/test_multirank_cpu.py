"""The benchmark's multi-process (N > 1) host logic on CPU ranks (gloo, world size 2).

Each rank decomposes its own tensor (weak scaling, no data-path collective); the only cross-rank
steps are the barrier and the max-over-ranks step time.  Checked here without a GPU: every rank
gets the slowest rank's time and the value counts the work of all ranks, and the reference arm
runs on rank 0 only (the other ranks return at once).
"""

import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, flops, out):
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms, value = bench.job_time_and_value(torch, dist, times[rank], flops, world, torch.device("cpu"))
        out[rank] = (ms, value)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_value_counts_every_rank():
    mp = torch.multiprocessing.get_context("spawn")
    world, flops = 2, 2.0e9
    times = [3.0, 5.0]
    with mp.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [mp.Process(target=_rank_main, args=(r, world, port, times, flops, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == max(times)
        assert value == pytest.approx(world * flops / (max(times) * 1e-3) / 1e12)


def test_single_process_keeps_its_own_time():
    sys.path.insert(0, ROOT)
    import bench

    ms, value = bench.job_time_and_value(torch, None, 4.0, 1.0e9, 1, torch.device("cpu"))
    assert ms == 4.0 and value == pytest.approx(1.0e9 / 4e-3 / 1e12)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup, cpu_slab = 1, 0, 8

    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(Args()) is None
    assert buf.getvalue() == ""
