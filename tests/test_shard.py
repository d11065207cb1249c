"""Sharded counting across ranks (no GPU): chunked round-robin covers every
root task exactly once, and world_size-2 gloo ranks combine their partial
counts into the single-process count."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import graphgen as gg
import oracle as O
from paper_2112_09761_gb300 import shard


@pytest.mark.parametrize("n,world,chunk", [(0, 2, 5), (1, 2, 5), (97, 2, 5), (1000, 3, 64),
                                           (1000, 4, 1), (10, 8, 3)])
def test_chunked_round_robin_partitions(n, world, chunk):
    seen = []
    for r in range(world):
        rs = shard.chunk_ranges(n, r, world, chunk)
        for lo, hi in rs:
            assert 0 <= lo < hi <= n and hi - lo <= chunk
            assert (lo // chunk) % world == r
        seen += [t for lo, hi in rs for t in range(lo, hi)]
    assert sorted(seen) == list(range(n))


def test_default_chunk():
    assert shard.default_chunk(10, 2) == 5          # never more than an even split
    assert shard.default_chunk(10**9, 2) == 2 * 152 * 64


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, pattern, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = gg.rmat_graph(10, 8, 77)
        n_tasks = O.num_tasks(g, pattern)
        total = shard.sharded_count(lambda lo, hi: O.count(g, pattern, False, lo, hi), n_tasks,
                                    rank, world, chunk=37)
        out[rank] = total
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("pattern", ["4-clique", "diamond", "tailed-triangle"])
def test_two_ranks_sum_to_the_whole(pattern):
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), pattern, out), nprocs=world,
                       start_method="spawn")
    whole = O.count(gg.rmat_graph(10, 8, 77), pattern)
    assert out[0] == out[1] == whole
