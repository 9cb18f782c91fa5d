"""The multi-rank path of the benchmark on CPU: two gloo ranks (127.0.0.1)
aggregate their times and fluid-node counts the way the GPU ranks do (the
slowest rank's time, all ranks' nodes), and the reference arm does its work
on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, fluid = bench.aggregate(10.0 + rank, 1000 * (rank + 1), world, "cpu")
    q.put((rank, ms, fluid))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, fluid in got:
        assert ms == 11.0 and fluid == 3000.0


def test_single_rank_aggregate_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(5.0, 7, 1, "cpu") == (5.0, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(steps=2, warmup=1, ref_seconds=1.0)
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
