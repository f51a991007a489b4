"""The N > 1 path of the benchmark on CPU: two gloo ranks (replicas only, no
data exchange): the step time is the slowest rank's, the value counts every
replica's edges, and rank 1 of the reference arm exits without work."""
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


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, ws, "cpu")
    out[rank] = (ms, bench.job_gteps(1_000_000, ms, ws))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        got = dict(out)
    for r in range(ws):
        ms, value = got[r]
        assert ms == 15.0
        assert value == pytest.approx(2 * 1_000_000 / 0.015 / 1e9)


def test_one_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.job_gteps(64_000_000, 125.0, 1) == pytest.approx(0.512)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup = 1, 0

    assert bench.run_reference(Args(), dict(bench.WORKLOAD)) == 0
