"""Multi-rank host logic of the benchmark (replicas, max-over-ranks timing) on CPU with gloo."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 100.0 + 50.0 * rank  # the slower replica decides
    got = bench.max_over_ranks(ms, world, dist, "cpu")
    out[rank] = (got, bench.aggregate_rate(world, got))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        assert res[r][0] == 150.0
        assert abs(res[r][1] - 2 * 1000.0 / 150.0) < 1e-12


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.aggregate_rate(1, 250.0) == 4.0
