"""GPU parity of the paper's radix-partitioned join (Section 6.2:
RadixPartitionExKer, then HashJoinExKer): the clustering step and its
boundary array against a stable sort and the oracle's find_boundary (pinned
to the paper's worked example), and the whole join (count, wrapping payload
sum, pair fingerprint) against the oracle and the direct join, over several
chunks and group ranges, skewed probes, a build group too large for the
shared-memory table, the all-ones key and a duplicate build key."""
import numpy as np
import pytest

import datagen as G
import oracle as O

pytestmark = pytest.mark.gpu

vx = pytest.importorskip("paper_2502_09541_gb300")


@pytest.fixture(scope="module")
def ctx():
    c = vx.vx_open(512 << 20)
    yield c
    vx.vx_close(c)


@pytest.mark.parametrize("bits", [8, 16, 24])
@pytest.mark.parametrize("kind,n", [("build", 100_003), ("zipf", 250_001), ("narrow", 70_000), ("build", 1),
                                    ("build", 0)])
def test_radix_cluster_and_find_boundary(ctx, bits, kind, n):
    if kind == "build":
        k = G.build_side(n)[0].view(np.uint64)
    elif kind == "zipf":
        k = G.probe_side(n, 1_000_000, 1.0, 1.0).view(np.uint64)
    else:  # few distinct groups: long runs of empty groups between them
        k = (G.i32_uniform(n, 0, 40, 3, 9).astype(np.uint64) * np.uint64(997)) << np.uint64(3)
    ok, rows, bnd = vx.vx_radix_cluster(ctx, k, bits)
    mask = np.uint64((1 << bits) - 1)
    perm = np.argsort(k & mask, kind="stable")
    assert np.array_equal(ok, k[perm]) and np.array_equal(rows, perm.astype(np.uint32))
    assert np.array_equal(bnd.astype(np.uint64), O.find_boundary((ok & mask).astype(np.uint32), 1 << bits))


def _run(bk, bp, pk, budget=256 << 20, **kw):
    c = vx.vx_open(budget)
    try:
        a = vx.vx_register_host_column(c, "bk", bk)
        b = vx.vx_register_host_column(c, "bp", bp)
        p = vx.vx_register_host_column(c, "pk", pk)
        o = vx.vx_join_opts()
        o.algorithm = vx.VX_JOIN_RADIX
        for k, v in kw.items():
            setattr(o, k, v)
        return vx.vx_join(c, a, b, p, o)
    finally:
        vx.vx_close(c)


@pytest.mark.parametrize("match,z", [(1.0, 0.0), (0.5, 0.0), (1.0, 1.0), (0.5, 1.0), (0.0, 0.0)])
@pytest.mark.parametrize("bits", [16, 24])
def test_radix_join_bit_exact(match, z, bits):
    """A 256 MiB budget: several partition chunks per table and several group
    ranges in the join pass."""
    nb, npr = 2_000_003, 8_000_009
    bk, bp = G.build_side(nb)
    pk = G.probe_side(npr, nb, match, z)
    r = _run(bk, bp, pk, radix_bits=bits)
    exp = O.join(bk, bp, pk, nthreads=8)
    assert (r["count"], r["payload_sum"], r["pair_fp"]) == exp
    assert (r["count"], r["payload_sum"]) == G.probe_truth(npr, nb, match, z)
    assert r["algorithm"] == vx.VX_JOIN_RADIX and r["ranges"] > 1 and r["n_partitions"] == 1 << bits


def test_radix_join_large_group_and_sentinel():
    # 300 build keys share their low 24 bits (one group beyond the shared-memory
    # table); the all-ones key is a build key too
    bk, _ = G.build_side(200_000)
    heavy = ((np.arange(300, dtype=np.uint64) + np.uint64(1)) << np.uint64(24)) | np.uint64(5)
    bk = np.unique(np.concatenate([bk.view(np.uint64), heavy, np.array([2**64 - 1], np.uint64)])).view(np.int64)
    bp = (bk * 5 + 3).astype(np.int64)
    pk = np.concatenate([bk[::2], heavy.view(np.int64)[::3], np.array([-1, -1, 77], np.int64),
                         G.probe_side(50_000, 200_000, 0.5, 1.0)])
    r = _run(bk, bp, pk)
    assert (r["count"], r["payload_sum"], r["pair_fp"]) == O.join(bk, bp, pk, nthreads=8)


def test_radix_join_equals_direct_join_and_duplicate_key():
    bk, bp = G.build_side(500_000)
    pk = G.probe_side(3_000_000, 500_000, 0.5, 1.0, seed=3)
    r = _run(bk, bp, pk)
    c = vx.vx_open(256 << 20)
    try:
        d = vx.vx_join(c, vx.vx_register_host_column(c, "a", bk), vx.vx_register_host_column(c, "b", bp),
                       vx.vx_register_host_column(c, "p", pk), vx.vx_join_opts())
    finally:
        vx.vx_close(c)
    assert (r["count"], r["payload_sum"], r["pair_fp"]) == (d["count"], d["payload_sum"], d["pair_fp"])
    bk2 = bk.copy()
    bk2[7] = bk2[8]
    with pytest.raises(vx.VxError) as e:
        _run(bk2, bp, pk)
    assert e.value.status == vx.VX_E_DUPKEY
