"""Splitting one count over several processes (one GPU each).

Root tasks are independent (edge parallelism, Section 5.1), so a count
shards by task ranges with no exchange except the final sum.  The split is
the paper's chunked round-robin (Section 7.1, policy 3): Omega is cut into
chunks of c tasks and chunk j goes to rank j mod world.  Each rank counts its
ranges with gpm_count_range; the integer partial counts are summed with one
all-reduce (8 bytes per rank).
"""
from __future__ import annotations


def chunk_ranges(n_tasks: int, rank: int, world: int, chunk: int) -> list[tuple[int, int]]:
    """Task ranges [lo, hi) of `rank` under chunked round-robin with chunk c."""
    if world < 1 or not 0 <= rank < world or chunk < 1:
        raise ValueError("bad rank / world / chunk")
    return [(lo, min(n_tasks, lo + chunk)) for lo in range(rank * chunk, n_tasks, world * chunk)]


def default_chunk(n_tasks: int, world: int, warps: int = 152 * 64, alpha: int = 2) -> int:
    """c = alpha x y with y the warps of one GPU (the paper's alpha = 2), at
    most an even split."""
    return max(1, min(alpha * warps, -(-n_tasks // max(1, world))))


def sharded_count(count_range, n_tasks: int, rank: int, world: int, chunk: int | None = None,
                  group=None) -> int:
    """Sum over all ranks of count_range(lo, hi) for each rank's ranges.

    `count_range` is the per-rank counter (gpm_count_range of a plan on that
    rank's GPU).  With world > 1 the partial counts are combined by an
    all-reduce of one int64 on the current torch.distributed group."""
    c = chunk or default_chunk(n_tasks, world)
    part = sum(count_range(lo, hi) for lo, hi in chunk_ranges(n_tasks, rank, world, c))
    if world == 1:
        return part
    import torch
    import torch.distributed as dist
    if part >= 1 << 63:
        raise OverflowError("partial count exceeds int64")
    backend = dist.get_backend(group)
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.tensor([part], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return int(t.item())
