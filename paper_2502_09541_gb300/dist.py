"""Multi-GPU layout of the star-join path: one process per GPU.

Fact chunks are independent (filter, probes and group-by run per row), so a
query shards by fact row ranges with the dimension tables replicated on every
GPU; the one exchange a sharded query needs is the sum of the per-group
partials (count and wrapping int64 sum per group, at most a few thousand
groups).  The benchmark runs weak scaling: every rank processes its own shard
of equal size and no collective touches the data path; the step time is the
maximum over ranks.
"""
from __future__ import annotations


def shard_rows(rank: int, world: int, rows_per_rank: int):
    """(row0, rows) of rank's shard of a world * rows_per_rank-row table."""
    if not 0 <= rank < world:
        raise ValueError("rank outside [0, world)")
    return rank * rows_per_rank, rows_per_rank


def split_range(rank: int, world: int, begin: int, end: int):
    """Contiguous near-equal split of [begin, end) for strong scaling."""
    n = end - begin
    lo = begin + n * rank // world
    hi = begin + n * (rank + 1) // world
    return lo, hi


def max_over_ranks(value: float, device="cpu") -> float:
    """Maximum of a per-rank float over the default process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_group_partials(gid, sums, cnts, n_groups: int, device="cpu"):
    """Sums per-group partial results of all ranks (dense over n_groups);
    returns (gid, sum, cnt) of the non-empty groups in ascending id, the
    result a single GPU computes over the whole table (two's-complement
    wrapping sums are order-free)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    s = torch.zeros(n_groups, dtype=torch.int64, device=device)
    c = torch.zeros(n_groups, dtype=torch.int64, device=device)
    g = torch.as_tensor(np.asarray(gid, dtype=np.int64), device=device)
    if len(g):
        s[g] = torch.as_tensor(np.asarray(sums, dtype=np.int64), device=device)
        c[g] = torch.as_tensor(np.asarray(cnts, dtype=np.uint64).astype(np.int64), device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    s, c = s.cpu().numpy(), c.cpu().numpy()
    nz = np.nonzero(c)[0]
    return nz.astype(np.uint64), s[nz], c[nz].astype(np.uint64)
