"""The multi-rank path on CPU: world_size-2 gloo process groups exercise the
row sharding, the max-over-ranks step time and the reduction of per-group
partials (the partial results come from the oracle on each rank's shard, and
their reduction must equal the oracle over the whole table), sums that wrap
past 2^63, and the partition sharding of the sort and the join: splitters
broadcast from rank 0, whole partitions per rank, sorted partitions written at
their offsets with no exchange, join partials summed."""
import os
import socket

import numpy as np
import pytest

import datagen as G
import oracle as O
from paper_2502_09541_gb300 import dist as D

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROWS_PER_RANK = 40_000
TEMPLATE = "T3_10"


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        row0, n = D.shard_rows(rank, world, ROWS_PER_RANK)
        fact = G.star_fact(n, seed=9, row0=row0)  # this rank's shard, generated in place
        dims = G.star_dims(0)
        T = G.star_templates()[TEMPLATE]
        sums, cnts = O.star(T, fact, dims)
        nz = np.nonzero(cnts)[0]
        gid, s, c = D.reduce_group_partials(nz, sums[nz], cnts[nz], len(sums))
        ms = D.max_over_ranks(10.0 * (rank + 1))
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), gid=gid, s=s, c=c, ms=ms)
    finally:
        dist.destroy_process_group()


def test_sharded_star_reduces_to_single_table(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    fact = G.star_fact(world * ROWS_PER_RANK, seed=9)
    sums, cnts = O.star(G.star_templates()[TEMPLATE], fact, G.star_dims(0))
    nz = np.nonzero(cnts)[0]
    for r in range(world):
        z = np.load(tmp_path / f"r{r}.npz")
        assert np.array_equal(z["gid"], nz) and np.array_equal(z["s"], sums[nz]) and np.array_equal(z["c"], cnts[nz])
        assert float(z["ms"]) == 20.0  # step time = slowest rank


def test_shard_and_split_cover_without_overlap():
    world, per = 3, 1000
    spans = [D.shard_rows(r, world, per) for r in range(world)]
    assert spans == [(0, 1000), (1000, 1000), (2000, 1000)]
    parts = [D.split_range(r, 4, 10, 1013) for r in range(4)]
    assert parts[0][0] == 10 and parts[-1][1] == 1013
    assert all(parts[i][1] == parts[i + 1][0] for i in range(3))
    with pytest.raises(ValueError):
        D.shard_rows(3, 3, 10)


def _wrap_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        big = 2**63 - 1 if rank == 0 else 5
        gid, s, c = D.reduce_group_partials(np.array([3]), np.array([big], np.int64), np.array([1], np.uint64), 8)
        jc, js, jf = D.reduce_join_partials(2**64 - 3 if rank == 0 else 7, 2**63, 2**63 + rank)
        np.savez(os.path.join(out_dir, f"w{rank}.npz"), gid=gid, s=s, c=c, j=np.array([jc, js, jf], np.uint64))
    finally:
        dist.destroy_process_group()


def test_partial_sums_wrap_modulo_2_64(tmp_path):
    mp.spawn(_wrap_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        z = np.load(tmp_path / f"w{r}.npz")
        assert z["gid"].tolist() == [3] and z["c"].tolist() == [2]
        assert int(z["s"][0]) == -2**63 + 4  # (2^63 - 1) + 5 wraps
        assert z["j"].tolist() == [4, 0, 1]


N_SORT, P_SORT = 60_000, 7


def _sort_join_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # sort: the same input on every rank; rank 0 draws the splitters
        k, r = G.sort_input(N_SORT, "zipf", seed=4)
        spl = O.sample_splitters(O.sorted_u64(k[::50].copy()), P_SORT) if rank == 0 else np.zeros(0, np.uint64)
        spl = D.broadcast_splitters(spl)
        pk_, pr_, b = O.range_partition(k, r, spl)
        sizes = np.diff(b).tolist()
        mine = D.assign_partitions(sizes, world)[rank]
        offs = D.partition_offsets(sizes)
        out = {}
        for p in mine:  # this rank's partitions, sorted, at their output offsets
            sk, sr = O.sort_pairs(pk_[b[p]:b[p + 1]], pr_[b[p]:b[p + 1]])
            out[f"k{offs[p]}"], out[f"r{offs[p]}"] = sk, sr
        np.savez(os.path.join(out_dir, f"s{rank}.npz"), **out)
        # join: build key ranges by splitters over the build keys, full probe side per rank
        bk, bp = G.build_side(20_000)
        pk = G.probe_side(80_000, 20_000, 0.5, 1.0)
        jspl = O.sample_splitters(O.sorted_u64(bk.view(np.uint64)[::10].copy()), 5) if rank == 0 else \
            np.zeros(0, np.uint64)
        jspl = D.broadcast_splitters(jspl)
        pid = np.searchsorted(jspl, bk.view(np.uint64), side="right")
        jsizes = np.bincount(pid, minlength=len(jspl) + 1).tolist()
        keep = np.isin(pid, D.assign_partitions(jsizes, world)[rank])
        c, s, f = O.join(bk[keep], bp[keep], pk)
        np.save(os.path.join(out_dir, f"j{rank}.npy"), np.array(D.reduce_join_partials(c, s, f), np.uint64))
    finally:
        dist.destroy_process_group()


def test_partition_sharded_sort_and_join(tmp_path):
    world = 2
    mp.spawn(_sort_join_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    k, r = G.sort_input(N_SORT, "zipf", seed=4)
    ek, er = O.sort_pairs(k, r)
    gk = np.empty_like(ek)
    gr = np.empty_like(er)
    filled = np.zeros(N_SORT, bool)
    for rank in range(world):
        z = np.load(tmp_path / f"s{rank}.npz")
        for name in z.files:
            if name.startswith("k"):
                off = int(name[1:])
                n = len(z[name])
                gk[off:off + n], gr[off:off + n] = z[name], z["r" + name[1:]]
                assert not filled[off:off + n].any()
                filled[off:off + n] = True
    assert filled.all() and np.array_equal(gk, ek) and np.array_equal(gr, er)
    bk, bp = G.build_side(20_000)
    pk = G.probe_side(80_000, 20_000, 0.5, 1.0)
    exp = O.join(bk, bp, pk)
    for rank in range(world):
        assert tuple(np.load(tmp_path / f"j{rank}.npy").tolist()) == exp


def test_partition_assignment_is_balanced_and_deterministic():
    sizes = [50, 10, 40, 40, 5, 30, 25]
    a = D.assign_partitions(sizes, 3)
    assert sorted(p for x in a for p in x) == list(range(len(sizes)))
    loads = [sum(sizes[p] for p in x) for x in a]
    assert max(loads) - min(loads) <= max(sizes)
    assert a == D.assign_partitions(sizes, 3)
    assert D.partition_offsets([3, 0, 4]) == [0, 3, 3]
