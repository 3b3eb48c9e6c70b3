"""GPU results at the workloads' full sizes, in the launch configuration the
benchmark times (64 MiB chunks, three staging slots, the library's own
grids): the star join on the 600M-row fact table under a 4 GiB budget, the
partitioned join at 1e9 build / 8e9 probe rows under 24 GiB, and the
out-of-core sort at 2e9 pairs under 16 GiB (the largest sort whose input,
output and scratch fit the host's memory).

The star join is compared with the oracle over the whole 600M-row table
for two templates (the oracle's row-range threads use every host core), and
on a ragged 20M-row range under every materialization policy; per-group
additivity over disjoint row ranges covers three more, and every other kernel
shape must give the plain form's groups over the whole table.  The join and the sort
are too large for the oracle to rescan in a test, so they are checked by
properties that hold at any size: the join count and payload sum the
generator records while drawing the probe keys, and a sort output that is
ordered, stable and a permutation of its input."""
import os

import numpy as np
import pytest

import datagen as G
import oracle as O

pytestmark = pytest.mark.gpu

vx = pytest.importorskip("paper_2502_09541_gb300")

STAR_ROWS = 600_000_000
GROUP_CAP = 1 << 16


@pytest.fixture(scope="module")
def star_full():
    fact = G.star_fact(STAR_ROWS)
    dims = G.star_dims(0)
    c = vx.vx_open(4 << 30)
    try:
        fid = {k: vx.vx_register_host_column(c, k, fact[k]) for k in fact}
        did = {d: {a: vx.vx_register_host_column(c, f"{d}.{a}", arr) for a, arr in dims[d].items()}
               for d in dims}
        yield c, fact, dims, fid, did
    finally:
        vx.vx_close(c)


def _dense(gid, s, cnt):
    """Dense wrapping (sum, count) arrays indexed by group id."""
    ds = np.zeros(GROUP_CAP, np.uint64)
    dc = np.zeros(GROUP_CAP, np.uint64)
    ds[gid.astype(np.int64)] = s.view(np.uint64)
    dc[gid.astype(np.int64)] = cnt
    return ds, dc


def _run(c, T, fid, did, late=vx.VX_LATE_AUTO, rb=0, re=0):
    st, gid, s, cnt, stats = vx.vx_run_plan(c, vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, late, rb, re),
                                             GROUP_CAP)
    assert st == vx.VX_OK
    return gid, s, cnt, stats


@pytest.mark.parametrize("name", ["T2_0.1", "T2_10", "T3_1"])
def test_star_full_table_ranges_add_up(star_full, name):
    c, fact, dims, fid, did = star_full
    T = G.star_templates()[name]
    gid, s, cnt, stats = _run(c, T, fid, did)
    assert stats["rows"] == STAR_ROWS and stats["chunks"] > 1
    full_s, full_c = _dense(gid, s, cnt)
    # disjoint ragged ranges covering the table: per-group sums (wrapping) and
    # counts must add up to the full-table result exactly
    cuts = [0, 123_456_789, 400_000_001, 599_999_999, STAR_ROWS]
    acc_s = np.zeros(GROUP_CAP, np.uint64)
    acc_c = np.zeros(GROUP_CAP, np.uint64)
    for rb, re in zip(cuts[:-1], cuts[1:]):
        ps, pc = _dense(*_run(c, T, fid, did, rb=rb, re=re)[:3])
        acc_s += ps
        acc_c += pc
    assert np.array_equal(acc_s, full_s) and np.array_equal(acc_c, full_c)
    assert int(full_c.sum()) == stats["survivors"]


@pytest.mark.parametrize("name", ["T2_10", "T3_1"])
def test_star_full_table_matches_oracle(star_full, name):
    """Every group of the whole 600M-row table equals the oracle's (O2 of the
    star definition, Section 7.1 query shape), in the benchmark's plain form."""
    c, fact, dims, fid, did = star_full
    T = G.star_templates()[name]
    es, ec = O.star(T, fact, dims, nthreads=os.cpu_count() or 1)
    nz = np.nonzero(ec)[0]
    gid, s, cnt, stats = _run(c, T, fid, did)
    assert stats["rows"] == STAR_ROWS and stats["chunks"] > 1
    assert np.array_equal(gid, nz) and np.array_equal(s, es[nz]) and np.array_equal(cnt, ec[nz])


@pytest.mark.parametrize("name", ["T2_1", "T3_10"])
def test_star_full_table_sample_matches_oracle(star_full, name):
    c, fact, dims, fid, did = star_full
    T = G.star_templates()[name]
    rb, re = 317_777_773, 337_777_779  # 20M rows, neither end on a chunk or tile boundary
    es, ec = O.star(T, fact, dims, rb, re, nthreads=16)
    nz = np.nonzero(ec)[0]
    for late in (vx.VX_LATE_AUTO, vx.VX_LATE_FORCE_LATE, vx.VX_LATE_FORCE_EARLY):
        gid, s, cnt, _ = _run(c, T, fid, did, late, rb, re)
        assert np.array_equal(gid, nz) and np.array_equal(s, es[nz]) and np.array_equal(cnt, ec[nz])


def test_star_full_table_batched_form_equals_plain(star_full):
    c, fact, dims, fid, did = star_full
    T = G.star_templates()["T3_1"]
    plain = _dense(*_run(c, T, fid, did)[:3])
    cfg = vx.vx_get_config(c)
    cfg.use_graphs = 1
    cfg.chunk_bytes = 256 << 20
    cfg.n_slots = 2
    vx.vx_set_config(c, cfg)
    try:
        for _ in range(2):  # capture, then replay
            got = _dense(*_run(c, T, fid, did, vx.VX_LATE_PER_CHUNK)[:3])
            assert np.array_equal(got[0], plain[0]) and np.array_equal(got[1], plain[1])
    finally:
        cfg.use_graphs = 0
        cfg.chunk_bytes = 64 << 20
        cfg.n_slots = 3
        vx.vx_set_config(c, cfg)


@pytest.mark.parametrize("rows,bps", [(2, 4), (2, 6), (8, 4), (16, 8)])
def test_star_full_table_kernel_shapes_equal_plain(star_full, rows, bps):
    """The other launch shapes the autotuner may pick (the bulk-copy pipeline,
    the scalar kernel) over the whole table give the plain form's groups, which
    the test above compares with the oracle."""
    c, fact, dims, fid, did = star_full
    for name in ("T2_1", "T3_1"):
        T = G.star_templates()[name]
        plain = _dense(*_run(c, T, fid, did)[:3])
        cfg = vx.vx_get_config(c)
        saved = (cfg.kernel_rows, cfg.blocks_per_sm)
        cfg.kernel_rows, cfg.blocks_per_sm = rows, bps
        vx.vx_set_config(c, cfg)
        try:
            got = _dense(*_run(c, T, fid, did)[:3])
        finally:
            cfg.kernel_rows, cfg.blocks_per_sm = saved
            vx.vx_set_config(c, cfg)
        assert np.array_equal(got[0], plain[0]) and np.array_equal(got[1], plain[1]), name


def test_join_full_size_matches_generator_truth():
    nb, npr = 1_000_000_000, 8_000_000_000
    bk, bp = G.build_side(nb)
    pk = G.probe_side(npr, nb, 1.0, 0.0)
    truth = G.probe_truth(npr, nb, 1.0, 0.0)
    c = vx.vx_open(24 << 30)
    try:
        a = vx.vx_register_host_column(c, "bk", bk)
        b = vx.vx_register_host_column(c, "bp", bp)
        p = vx.vx_register_host_column(c, "pk", pk)
        r = vx.vx_join(c, a, b, p, vx.vx_join_opts())
        assert (r["count"], r["payload_sum"]) == truth
        assert r["n_partitions"] == 1 and r["overflow_retries"] == 0
    finally:
        vx.vx_close(c)


def _fmix(z):
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def _multiset_fingerprint(k, r, step=100_000_000):
    """Order-free fingerprint of the (key, row id) pairs: a wrapping sum of a
    mixing function of each pair."""
    total = np.uint64(0)
    with np.errstate(over="ignore"):
        for i in range(0, len(k), step):
            z = k[i:i + step] ^ (r[i:i + step].astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15))
            total += _fmix(z).sum(dtype=np.uint64)
    return int(total)


def test_sort_2e9_pairs_ordered_stable_permutation():
    n = 2_000_000_000
    k, r = G.sort_input(n, "zipf")
    fp_in = _multiset_fingerprint(k, r)
    ok = np.empty(n, np.uint64)
    orr = np.empty(n, np.uint32)
    scratch = np.empty(12 * (n + n // 16), np.uint8)  # a region per partition, as the benchmark runs it
    c = vx.vx_open(16 << 30)
    try:
        kc = vx.vx_register_host_column(c, "k", k)
        rc = vx.vx_register_host_column(c, "r", r)
        o = vx.vx_sort_opts()
        o.partitioner = vx.VX_PART_LEARNED_PL
        o.sample_size = 1 << 20
        o.host_scratch = scratch.ctypes.data
        o.host_scratch_bytes = scratch.nbytes
        st = vx.vx_sort(c, kc, rc, ok, orr, o)
        assert st["n_partitions"] > 1 and st["contiguous_layout"] == 1
    finally:
        vx.vx_close(c)
    del scratch, k, r
    step = 100_000_000
    for i in range(0, n, step):  # ordered by key, equal keys in input order (row id = input index)
        j = min(n, i + step + 1)
        kk, rr = ok[i:j], orr[i:j]
        assert np.all(kk[1:] >= kk[:-1])
        eq = kk[1:] == kk[:-1]
        assert np.all(rr[1:][eq] > rr[:-1][eq])
    assert _multiset_fingerprint(ok, orr) == fp_in
