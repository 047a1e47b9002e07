"""The N > 1 benchmark path's host logic with two gloo ranks on the CPU:
shards cover the batch exactly once, every rank sees the slowest rank's
time, and throughput is whole-job."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2009_13349_gb300 import parallel as P


def test_shards_partition_the_batch():
    for n in (0, 1, 7, 1000, 1_000_001):
        for world in (1, 2, 3, 8):
            spans = [P.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = P.env()
    local_ms = 100.0 + 50.0 * r               # rank 1 is the slow one
    dist.barrier()
    step = P.max_over_ranks(local_ms)
    out[r] = (w, r, step, P.job_throughput(1_000_000, w, step), P.rank_seed(1, r))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = 29500 + (os.getpid() % 1000)
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][2] == res[1][2] == 150.0
    assert res[0][3] == pytest.approx(2_000_000 / 0.150)
    assert {res[0][4], res[1][4]} == {1, 2}
    assert P.max_over_ranks(3.5) == 3.5       # no group: identity
