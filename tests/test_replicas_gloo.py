"""Multi-process host logic of the benchmark's replica mode on CPU (gloo,
world size 2): the whole-job figures are the slowest rank's time and the sum
of all ranks' units, and the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1 + r seconds for 100 (r + 1) units
        t, u = bench.reduce_over_ranks(torch, 1.0 + rank, 100 * (rank + 1), "cpu")
        out.put((rank, t, u, bench.dist_env()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo():
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, t, u, env in res:
        assert t == 2.0 and u == 300.0
        assert env == (rank, world, rank)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        steps, warmup, gpus = 1, 0, 2
    bench.reference_arm(Args, "euler3d-n5-amr", bench.WORKLOADS["euler3d-n5-amr"])
    assert capsys.readouterr().out == ""
