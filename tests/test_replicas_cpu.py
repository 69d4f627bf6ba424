"""Several GPUs run independent replicas of the training step (the step does
not shard, so there is no collective on the data path): the reported time is
the slowest rank's and the throughput counts every rank's steps.  The
aggregation is checked here with two gloo ranks on the CPU, and the CPU-oracle
arm does its work on rank 0 only."""
import argparse
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], world, "cpu")
        out.put((rank, ms, bench.replica_throughput(10, ms, world)))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_all_steps_count():
    world, times = 2, [4.0, 5.0]                  # ms for 10 steps on each rank
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [5.0, 5.0]                    # every rank sees the max
    assert got[0][2] == pytest.approx(2 * 10 / 0.005)           # 20 steps in 5 ms


def test_single_process_is_unchanged():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.replica_throughput(20, 50.0, 1) == pytest.approx(400.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(steps=1, warmup=3, workload="skewed-3M-1600x1060")
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
