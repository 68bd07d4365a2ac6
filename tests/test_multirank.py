"""Multi-GPU bench logic on CPU: the path does not shard, so N ranks run N
independent replicas; the job time is the slowest rank's and the work is the
sum over ranks.  Checked with two gloo ranks (no GPU)."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, it = bench.combine_ranks(10.0 + 5.0 * rank, 100 + rank, dist, torch.device("cpu"))
    out[rank] = (t, it)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_combine_max_time_sum_work():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r] == (15.0, 201.0)


def test_single_rank_is_identity():
    import bench
    assert bench.combine_ranks(12.5, 100, None, None) == (12.5, 100.0)


def test_dist_env_defaults(monkeypatch):
    import bench
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (0, 0, 1)
    monkeypatch.setenv("RANK", "3")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "4")
    assert bench.dist_env() == (3, 1, 4)
