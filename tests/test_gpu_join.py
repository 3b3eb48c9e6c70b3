"""GPU parity of the partitioned hash join (count, wrapping payload sum, pair
fingerprint) against the oracle and the generator's own ground truth."""
import numpy as np
import pytest

import datagen as G
import oracle as O

pytestmark = pytest.mark.gpu

vx = pytest.importorskip("paper_2502_09541_gb300")


def _run(bk, bp, pk, budget=256 << 20, chunk=8 << 20, **kw):
    c = vx.vx_open(budget)
    try:
        cfg = vx.vx_get_config(c)
        cfg.chunk_bytes = chunk
        vx.vx_set_config(c, cfg)
        a = vx.vx_register_host_column(c, "bk", bk)
        b = vx.vx_register_host_column(c, "bp", bp)
        p = vx.vx_register_host_column(c, "pk", pk)
        o = vx.vx_join_opts()
        for k, v in kw.items():
            setattr(o, k, v)
        return vx.vx_join(c, a, b, p, o)
    finally:
        vx.vx_close(c)


@pytest.mark.parametrize("match,z", [(1.0, 0.0), (0.5, 0.0), (1.0, 1.0), (0.5, 1.0), (0.0, 0.0)])
@pytest.mark.parametrize("P,count_pass,part", [(1, 0, vx.VX_PART_SAMPLE), (3, 1, vx.VX_PART_SAMPLE),
                                               (4, 0, vx.VX_PART_LEARNED_PL), (5, 0, vx.VX_PART_LEARNED_MLP)])
def test_join_bit_exact(match, z, P, count_pass, part):
    nb, npr = 1_000_003, 4_000_037
    bk, bp = G.build_side(nb)
    pk = G.probe_side(npr, nb, match, z)
    r = _run(bk, bp, pk, n_partitions=P, count_pass=count_pass, partitioner=part, sample_size=100_000)
    exp = O.join(bk, bp, pk, nthreads=8)
    assert (r["count"], r["payload_sum"], r["pair_fp"]) == exp
    assert (r["count"], r["payload_sum"]) == G.probe_truth(npr, nb, match, z)
    assert r["n_partitions"] == P


def test_join_auto_partitions_under_small_budget():
    # 2M build rows need ~40 MB of table at load 0.8; a 24 MiB budget forces P > 1
    nb, npr = 2_000_000, 3_000_000
    bk, bp = G.build_side(nb)
    pk = G.probe_side(npr, nb, 1.0, 1.0)
    r = _run(bk, bp, pk, budget=24 << 20, chunk=1 << 20)
    assert r["n_partitions"] > 1
    assert (r["count"], r["payload_sum"], r["pair_fp"]) == O.join(bk, bp, pk, nthreads=8)


def test_join_skewed_build_keys_learned_sizing():
    # forcing a tiny load factor estimate is not possible; instead a heavily
    # skewed build key distribution makes the learned per-range size estimate
    # (nb / P) wrong for some ranges, which must be rebuilt and stay exact
    nb = 600_000
    bk = np.concatenate([np.arange(500_000, dtype=np.int64) * 7 + 1,
                         G.build_side(100_000)[0]]).astype(np.int64)
    bk = np.unique(bk)
    bp = (bk * 3 + 11).astype(np.int64)
    pk = np.concatenate([bk[::3], np.arange(10_000, dtype=np.int64) * 7 + 2])
    r = _run(bk, bp, pk, n_partitions=4, count_pass=0, partitioner=vx.VX_PART_SAMPLE, sample_size=1000)
    assert (r["count"], r["payload_sum"], r["pair_fp"]) == O.join(bk, bp, pk, nthreads=8)


def test_join_edge_cases():
    bk, bp = G.build_side(1000)
    empty = np.zeros(0, np.int64)
    r = _run(bk, bp, empty)
    assert (r["count"], r["payload_sum"], r["pair_fp"]) == (0, 0, 0)
    # build key equal to the all-ones sentinel is still joined
    bk2 = bk.copy()
    bk2[0] = -1
    pk = np.array([-1, bk2[1], 12345, -1], np.int64)
    r = _run(bk2, bp, pk)
    assert (r["count"], r["payload_sum"], r["pair_fp"]) == O.join(bk2, bp, pk)
    # duplicate build key
    bk3 = bk.copy()
    bk3[5] = bk3[6]
    with pytest.raises(vx.VxError) as e:
        _run(bk3, bp, pk)
    assert e.value.status == vx.VX_E_DUPKEY
