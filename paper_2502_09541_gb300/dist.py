"""Multi-GPU layout of the star-join path: one process per GPU.

Fact chunks are independent (filter, probes and group-by run per row), so a
query shards by fact row ranges with the dimension tables replicated on every
GPU; the one exchange a sharded query needs is the sum of the per-group
partials (count and wrapping int64 sum per group, at most a few thousand
groups).  The benchmark runs weak scaling: every rank processes its own shard
of equal size and no collective touches the data path; the step time is the
maximum over ranks.

The out-of-core sort and the partitioned join shard by partition instead:
after the range partition (Sections 6.1, 6.2) the partitions are independent,
so once every rank holds the same splitters (broadcast from rank 0) each rank
takes a set of whole partitions.  A sorted partition lands at the output
offset of the partitions before it, so the ranks of a sort need no exchange
at all; the ranks of a join sum their (count, payload sum, fingerprint).
Sums are reduced as two 32-bit halves so that the result wraps modulo 2^64
exactly as one GPU's does.
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


def _allreduce_u64(values, device="cpu"):
    """Sum of uint64 values over the ranks, modulo 2^64: each value is split
    into its high and low 32-bit halves, which int64 sums hold without
    overflow for fewer than 2^31 ranks."""
    import numpy as np
    import torch
    import torch.distributed as dist
    v = np.asarray(values, dtype=np.uint64)
    hi = torch.as_tensor((v >> np.uint64(32)).astype(np.int64), device=device)
    lo = torch.as_tensor((v & np.uint64(0xFFFFFFFF)).astype(np.int64), device=device)
    dist.all_reduce(hi, op=dist.ReduceOp.SUM)
    dist.all_reduce(lo, op=dist.ReduceOp.SUM)
    hi = hi.cpu().numpy().astype(np.uint64)
    lo = lo.cpu().numpy().astype(np.uint64)
    with np.errstate(over="ignore"):
        return (hi << np.uint64(32)) + lo


def reduce_group_partials(gid, sums, cnts, n_groups: int, device="cpu"):
    """Sums per-group partial results of all ranks (dense over n_groups);
    returns (gid, sum, cnt) of the non-empty groups in ascending id, the
    result a single GPU computes over the whole table (two's-complement
    wrapping sums are order-free)."""
    import numpy as np
    s = np.zeros(n_groups, dtype=np.uint64)
    c = np.zeros(n_groups, dtype=np.uint64)
    g = np.asarray(gid, dtype=np.int64)
    if len(g):
        s[g] = np.asarray(sums, dtype=np.int64).view(np.uint64)
        c[g] = np.asarray(cnts, dtype=np.uint64)
    s = _allreduce_u64(s, device)
    c = _allreduce_u64(c, device)
    nz = np.nonzero(c)[0]
    return nz.astype(np.uint64), s[nz].view(np.int64), c[nz]


def broadcast_splitters(splitters, device="cpu"):
    """Rank 0's splitters on every rank (the one input the ranks of a
    partitioned sort or join share)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    n = torch.tensor([len(splitters) if dist.get_rank() == 0 else 0], dtype=torch.int64, device=device)
    dist.broadcast(n, 0)
    t = torch.zeros(int(n.item()), dtype=torch.int64, device=device)
    if dist.get_rank() == 0 and len(splitters):
        t[:] = torch.as_tensor(np.asarray(splitters, dtype=np.uint64).view(np.int64), device=device)
    dist.broadcast(t, 0)
    return t.cpu().numpy().view(np.uint64)


def assign_partitions(sizes, world: int):
    """Partitions per rank: largest first to the least-loaded rank (ties to
    the lower rank), each rank's list in ascending partition id.  The same
    sizes give every rank the same assignment."""
    load = [0] * world
    parts = [[] for _ in range(world)]
    for p in sorted(range(len(sizes)), key=lambda q: (-int(sizes[q]), q)):
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(p)
        load[r] += int(sizes[p])
    return [sorted(x) for x in parts]


def partition_offsets(sizes):
    """Output offset of every partition: the pairs of the partitions before it."""
    out, at = [], 0
    for n in sizes:
        out.append(at)
        at += int(n)
    return out


def reduce_join_partials(count: int, payload_sum: int, pair_fp: int, device="cpu"):
    """(count, payload sum, pair fingerprint) summed over the ranks modulo 2^64."""
    import numpy as np
    r = _allreduce_u64(np.array([count, payload_sum, pair_fp], dtype=np.uint64), device)
    return int(r[0]), int(r[1]), int(r[2])
