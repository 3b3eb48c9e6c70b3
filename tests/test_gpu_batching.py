"""Batching: the star pipeline captured as one CUDA graph and replayed, the
autotuner of chunk size, ring depth and kernel launch shape, and every launch
shape it may pick.  Results must be identical to the oracle
(and to the executor's) on every replay."""
import numpy as np
import pytest

import datagen as G
import oracle as O

pytestmark = pytest.mark.gpu

vx = pytest.importorskip("paper_2502_09541_gb300")


@pytest.fixture(scope="module")
def star():
    n = 4_000_003
    fact = G.star_fact(n, seed=13)
    dims = G.star_dims(0)
    ctx = vx.vx_open(512 << 20)
    fid = {c: vx.vx_register_host_column(ctx, c, fact[c]) for c in fact}
    did = {d: {a: vx.vx_register_host_column(ctx, f"{d}.{a}", arr) for a, arr in dims[d].items()} for d in dims}
    yield ctx, fact, dims, fid, did
    vx.vx_close(ctx)


def _expect(T, fact, dims, rb=0, re=None):
    es, ec = O.star(T, fact, dims, rb, re, nthreads=8)
    nz = np.nonzero(ec)[0]
    return nz.astype(np.uint64), es[nz], ec[nz]


@pytest.mark.parametrize("name", ["T1", "T2_1", "T3_10", "T3_0.1"])
def test_graph_replay_bit_exact(star, name):
    ctx, fact, dims, fid, did = star
    cfg = vx.vx_get_config(ctx)
    cfg.use_graphs = 1
    cfg.chunk_bytes = 8 << 20
    vx.vx_set_config(ctx, cfg)
    T = G.star_templates()[name]
    if name == "T1":
        T = dict(T, dims=[{"dim": "date", "fk": "date_fk", "preds": [("year", 1, 1)]}])
    plan = vx.make_plan(T, fid, did, G.STAR_ATTR_CARD)
    gid_e, s_e, c_e = _expect(T, fact, dims)
    first = None
    for rep in range(3):  # capture, then two replays
        st, gid, s, c, stats = vx.vx_run_plan(ctx, plan)
        assert st == vx.VX_OK
        assert np.array_equal(gid, gid_e) and np.array_equal(s, s_e) and np.array_equal(c, c_e)
        if first is None:
            first = stats
        assert stats["chunks"] == first["chunks"] > 1
    cfg.use_graphs = 0
    vx.vx_set_config(ctx, cfg)


def test_graph_survives_table_rebuild_and_ranges(star):
    ctx, fact, dims, fid, did = star
    cfg = vx.vx_get_config(ctx)
    cfg.use_graphs = 1
    vx.vx_set_config(ctx, cfg)
    T = G.star_templates()["T2_10"]
    for rb, re in [(0, 0), (12_345, 3_000_001), (0, 0)]:
        vx.vx_drop_resident(ctx)
        plan = vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO, rb, re)
        st, gid, s, c, _ = vx.vx_run_plan(ctx, plan)
        gid_e, s_e, c_e = _expect(T, fact, dims, rb, None if re == 0 else re)
        assert np.array_equal(gid, gid_e) and np.array_equal(s, s_e) and np.array_equal(c, c_e)
    cfg.use_graphs = 0
    vx.vx_set_config(ctx, cfg)


def test_autotuner_picks_a_candidate_and_keeps_results(star):
    ctx, fact, dims, fid, did = star
    T = G.star_templates()["T3_1"]
    plan = vx.make_plan(T, fid, did, G.STAR_ATTR_CARD)
    best = vx.vx_autotune(ctx, plan, 2_000_000)
    assert best.chunk_bytes in [m << 20 for m in (8, 16, 32, 64, 128, 256)]
    assert best.n_slots in (2, 3, 4)
    assert best.kernel_rows in (0, 2, 8, 16) and best.blocks_per_sm in (4, 6, 8)
    assert best.h2d_copy_blocks in (0, 32)
    cur = vx.vx_get_config(ctx)
    assert cur.chunk_bytes == best.chunk_bytes and cur.n_slots == best.n_slots
    assert cur.kernel_rows == best.kernel_rows and cur.blocks_per_sm == best.blocks_per_sm
    st, gid, s, c, _ = vx.vx_run_plan(ctx, plan)
    gid_e, s_e, c_e = _expect(T, fact, dims)
    assert np.array_equal(gid, gid_e) and np.array_equal(s, s_e) and np.array_equal(c, c_e)


@pytest.mark.parametrize("rows,bps", [(0, 4), (2, 1), (2, 2), (2, 4), (2, 6), (2, 8), (8, 4), (8, 8), (16, 4), (16, 8)])
@pytest.mark.parametrize("late", [vx.VX_LATE_FORCE_EARLY, vx.VX_LATE_FORCE_LATE])
def test_kernel_shapes_bit_exact(star, rows, bps, late):
    """Every launch shape the autotuner may pick (one tile per block, the
    bulk-copy pipeline at 1 to 8 blocks per SM, i.e. 8 down to 2
    shared-memory stages, the scalar kernel at 8 or 16 rows per thread and 4
    or 8 blocks per SM), in both the fused and the split (late-column gather)
    forms, over a row range whose chunks end in partial groups of rows."""
    ctx, fact, dims, fid, did = star
    cfg = vx.vx_get_config(ctx)
    saved = (cfg.kernel_rows, cfg.blocks_per_sm, cfg.chunk_bytes)
    cfg.kernel_rows, cfg.blocks_per_sm, cfg.chunk_bytes = rows, bps, 8 << 20
    vx.vx_set_config(ctx, cfg)
    try:
        for name in ("T2_1", "T3_10"):
            T = G.star_templates()[name]
            st, gid, s, c, _ = vx.vx_run_plan(ctx, vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, late, 1_001, 3_999_999))
            gid_e, s_e, c_e = _expect(T, fact, dims, 1_001, 3_999_999)
            assert st == vx.VX_OK
            assert np.array_equal(gid, gid_e) and np.array_equal(s, s_e) and np.array_equal(c, c_e)
    finally:
        cfg.kernel_rows, cfg.blocks_per_sm, cfg.chunk_bytes = saved
        vx.vx_set_config(ctx, cfg)
