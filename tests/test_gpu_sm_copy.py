"""Host-to-device staging by a copy kernel (vx_config.h2d_copy_blocks > 0)
instead of the copy engine: every executor's results stay bit-identical to
the copy engine's and to the oracle, including row ranges whose host
addresses are not 16-byte aligned relative to the staging slots."""
import numpy as np
import pytest

import datagen as G
import oracle as O

pytestmark = pytest.mark.gpu

vx = pytest.importorskip("paper_2502_09541_gb300")

N = 4_000_000


@pytest.fixture(scope="module")
def star():
    fact, dims = G.star_fact(N, seed=21), G.star_dims(0)
    c = vx.vx_open(512 << 20)
    fid = {k: vx.vx_register_host_column(c, k, fact[k]) for k in fact}
    did = {d: {a: vx.vx_register_host_column(c, f"{d}.{a}", arr) for a, arr in dims[d].items()} for d in dims}
    yield c, fact, dims, fid, did
    vx.vx_close(c)


def _set(c, blocks, chunk=8 << 20):
    cfg = vx.vx_get_config(c)
    cfg.h2d_copy_blocks = blocks
    cfg.chunk_bytes = chunk
    vx.vx_set_config(c, cfg)


@pytest.mark.parametrize("blocks", [32, 152])
@pytest.mark.parametrize("name", ["T2_1", "T3_10", "T1"])
def test_star_sm_copy_equals_copy_engine_and_oracle(star, blocks, name):
    c, fact, dims, fid, did = star
    T = G.star_templates()[name]
    rb, re = 1_001, 3_999_999  # ragged ends; sources 4-byte but not 16-byte aligned to their slots
    try:
        _set(c, 0)
        ref = vx.vx_run_plan(c, vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO, rb, re))
        _set(c, blocks)
        got = vx.vx_run_plan(c, vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO, rb, re))
    finally:
        _set(c, 0, 64 << 20)
    for x, y in zip(ref[1:4], got[1:4]):
        assert np.array_equal(x, y)
    es, ec = O.star(T, fact, dims, rb, re, nthreads=8)
    nz = np.nonzero(ec)[0]
    assert np.array_equal(got[1], nz) and np.array_equal(got[2], es[nz]) and np.array_equal(got[3], ec[nz])


@pytest.mark.parametrize("late", [vx.VX_LATE_AUTO, vx.VX_LATE_PER_CHUNK])
@pytest.mark.parametrize("name", ["T2_10", "T3_1"])
def test_star_graphs_sm_copy_equal_oracle(star, name, late):
    """The batched form as the benchmark times it: the pipeline captured in a
    graph (copy kernels at the highest priority, per-node priorities kept),
    two staging slots, per-chunk late decisions; the capture and its replay
    both equal the oracle on a ragged range."""
    c, fact, dims, fid, did = star
    T = G.star_templates()[name]
    rb, re = 1_001, 3_999_999
    cfg = vx.vx_get_config(c)
    saved = (cfg.use_graphs, cfg.chunk_bytes, cfg.n_slots, cfg.h2d_copy_blocks)
    cfg.use_graphs, cfg.chunk_bytes, cfg.n_slots, cfg.h2d_copy_blocks = 1, 8 << 20, 2, 32
    vx.vx_set_config(c, cfg)
    try:
        runs = [vx.vx_run_plan(c, vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, late, rb, re)) for _ in range(2)]
    finally:
        cfg.use_graphs, cfg.chunk_bytes, cfg.n_slots, cfg.h2d_copy_blocks = saved
        vx.vx_set_config(c, cfg)
    es, ec = O.star(T, fact, dims, rb, re, nthreads=8)
    nz = np.nonzero(ec)[0]
    for r in runs:
        assert r[0] == vx.VX_OK
        assert np.array_equal(r[1], nz) and np.array_equal(r[2], es[nz]) and np.array_equal(r[3], ec[nz])
    assert runs[0][4]["chunks"] > 2  # several chunks, so the copies overlap kernels


@pytest.mark.parametrize("plan", [0, 1])
def test_sort_sm_copy(plan):
    n = 2_000_003
    k, r = G.sort_input(n, "zipf", seed=2)
    c = vx.vx_open(256 << 20)
    try:
        _set(c, 64, 64 << 20)
        kc = vx.vx_register_host_column(c, "k", k)
        rc = vx.vx_register_host_column(c, "r", r)
        ok, orr = np.empty(n, np.uint64), np.empty(n, np.uint32)
        o = vx.vx_sort_opts()
        o.plan = plan
        o.max_slot_pairs = 300_000  # several partitions or runs
        vx.vx_sort(c, kc, rc, ok, orr, o)
    finally:
        vx.vx_close(c)
    ek, er = O.sort_pairs(k, r)
    assert np.array_equal(ok, ek) and np.array_equal(orr, er)


def test_join_sm_copy():
    nb, npr = 300_000, 3_000_000
    bk, bp = G.build_side(nb)
    pk = G.probe_side(npr, nb, 0.5, 1.0, seed=3)
    c = vx.vx_open(256 << 20)
    try:
        _set(c, 32, 4 << 20)
        a = vx.vx_register_host_column(c, "a", bk)
        b = vx.vx_register_host_column(c, "b", bp)
        p = vx.vx_register_host_column(c, "p", pk)
        r = vx.vx_join(c, a, b, p, vx.vx_join_opts())
    finally:
        vx.vx_close(c)
    assert (r["count"], r["payload_sum"], r["pair_fp"]) == O.join(bk, bp, pk, nthreads=8)


def test_config_rejects_bad_block_counts(star):
    c = star[0]
    cfg = vx.vx_get_config(c)
    for bad in (-1, 1025):
        cfg.h2d_copy_blocks = bad
        with pytest.raises(vx.VxError):
            vx.vx_set_config(c, cfg)


def test_serving_scan_sm_copy(star):
    """The serving engine's shared scan staged by the copy kernel: every query
    as alone and as the oracle."""
    c, fact, dims, fid, did = star
    names = ["T2_1", "T3_1", "T2_10", "T3_0.1"]
    ranges = [(0, N), (123_457, 2_500_001), (7, 3_999_999), (1_000_000, 1_000_000 + 777_777)]
    try:
        _set(c, 0)
        alone = [vx.vx_run_plan(c, vx.make_plan(G.star_templates()[n], fid, did, G.STAR_ATTR_CARD,
                                                vx.VX_LATE_AUTO, rb, re)) for n, (rb, re) in zip(names, ranges)]
        _set(c, 32)
        vx.vx_serve_start(c, chunk_rows=1 << 19, max_active=8)
        tickets = [vx.vx_submit(c, vx.make_plan(G.star_templates()[n], fid, did, G.STAR_ATTR_CARD,
                                                 vx.VX_LATE_AUTO, rb, re)) for n, (rb, re) in zip(names, ranges)]
        results = [vx.vx_wait(c, t) for t in tickets]
        vx.vx_serve_stop(c)
    finally:
        _set(c, 0, 64 << 20)
    for (n, (rb, re)), a, r in zip(zip(names, ranges), alone, results):
        assert r[0] == vx.VX_OK
        for x, y in zip(a[1:4], r[1:4]):
            assert np.array_equal(x, y), (n, rb, re)
    es, ec = O.star(G.star_templates()[names[1]], fact, dims, *ranges[1], nthreads=8)
    nz = np.nonzero(ec)[0]
    assert np.array_equal(results[1][1], nz) and np.array_equal(results[1][2], es[nz])
