"""The multi-rank path on CPU: world_size-2 gloo process groups exercise the
row sharding, the max-over-ranks step time and the reduction of per-group
partials; the partial results come from the oracle on each rank's shard, and
their reduction must equal the oracle over the whole table."""
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
