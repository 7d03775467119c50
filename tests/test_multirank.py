"""Multi-rank host logic of the benchmark on CPU: world-size-2 gloo ranks (no GPU).

The path has no exchange step: each rank solves its own matrices (weak scaling). What crosses ranks
is the barrier and the max-reduce of the timings, checked here, and the sharding helper.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    r, w, local = bench.dist_setup()
    assert (r, w, local) == (rank, world, rank)
    bench.barrier(w)
    m = bench.max_over_ranks(float(10 + rank), w)
    lo, hi = bench.shard(1000, r, w)
    out[rank] = (m, lo, hi)
    import torch.distributed as dist

    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_max_and_shards():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 11.0  # max over ranks
    assert (res[0][1], res[0][2]) == (0, 500) and (res[1][1], res[1][2]) == (500, 1000)


@pytest.mark.parametrize("total,world", [(0, 2), (7, 3), (2048, 8), (5, 8)])
def test_shards_partition_the_units(total, world):
    import bench

    seen = []
    for r in range(world):
        lo, hi = bench.shard(total, r, world)
        assert 0 <= lo <= hi <= total
        seen.extend(range(lo, hi))
    assert seen == list(range(total))
