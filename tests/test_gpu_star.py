"""GPU parity of the streaming star-join path (chunked executor, dimension hash
tables, fused filter/probe/aggregate kernel, zero-copy late materialization),
of vx_filter's ordered compaction and of vx_groupby, against the oracle.
Integer results: the bar is bit-exact."""
import numpy as np
import pytest

import datagen as G
import oracle as O

pytestmark = pytest.mark.gpu

vx = pytest.importorskip("paper_2502_09541_gb300")


def _open(budget, chunk_bytes=None, **cfg_over):
    ctx = vx.vx_open(budget)
    cfg = vx.vx_get_config(ctx)
    if chunk_bytes:
        cfg.chunk_bytes = chunk_bytes
    for k, v in cfg_over.items():
        setattr(cfg, k, v)
    vx.vx_set_config(ctx, cfg)
    return ctx


DATE_CARDS = {"date": {"year": 7, "month": 12}}


@pytest.fixture(scope="module")
def q1_full():
    """The 6,000,000-row single-dimension query, 64 MiB budget, 8 MiB chunks."""
    fact, dim = G.q1_tables(6_000_000)
    ctx = _open(64 << 20, 8 << 20)
    fid = {c: vx.vx_register_host_column(ctx, c, fact[c]) for c in fact}
    did = {c: vx.vx_register_host_column(ctx, "date." + c, dim[c]) for c in ("key", "year", "month")}
    yield ctx, fact, dim, fid, did
    vx.vx_close(ctx)


def _q1_plan(fid, did, late=vx.VX_LATE_AUTO, row_begin=0, row_end=0):
    tmpl = {"dims": [{"dim": "date", "fk": "date_fk", "preds": [("year", 1993, 1993)]}],
            "fact_preds": [("discount", 1, 3), ("quantity", vx.I32MIN, 24)],
            "group": [], "agg": ("mul", "price", "discount")}
    return vx.make_plan(tmpl, fid, {"date": did}, {"date": {"year": 1, "month": 1}}, late, row_begin, row_end)


@pytest.mark.parametrize("late", [vx.VX_LATE_AUTO, vx.VX_LATE_FORCE_EARLY, vx.VX_LATE_FORCE_LATE])
@pytest.mark.parametrize("sched", [vx.VX_SCHED_IMMEDIATE, vx.VX_SCHED_DAG])
def test_q1_full_size_bit_exact(q1_full, late, sched):
    ctx, fact, dim, fid, did = q1_full
    cfg = vx.vx_get_config(ctx)
    cfg.sched = sched
    vx.vx_set_config(ctx, cfg)
    st, gid, s, c, stats = vx.vx_run_plan(ctx, _q1_plan(fid, did, late))
    exp = O.q1(fact, dim)
    assert st == vx.VX_OK
    assert (int(s[0]), int(c[0])) == exp
    assert stats["chunks"] == 12  # 8 MiB of 4 staged int32 columns per chunk
    if late == vx.VX_LATE_FORCE_LATE:
        assert stats["late_mask"] == 1  # price read by zero-copy
    if late == vx.VX_LATE_FORCE_EARLY:
        assert stats["late_mask"] == 0
    if late == vx.VX_LATE_AUTO:
        # estimated selectivity ~1.9% < TH = 1/16: price is late-materialized
        assert 0.01 < stats["est_selectivity"] < 0.03 and stats["late_mask"] == 1


@pytest.mark.parametrize("rb,re", [(0, 1), (5, 6), (0, 524_288), (1, 524_289), (123_457, 4_000_001),
                                   (5_999_999, 6_000_000), (100, 100)])
def test_q1_row_ranges_ragged(q1_full, rb, re):
    ctx, fact, dim, fid, did = q1_full
    st, gid, s, c, _ = vx.vx_run_plan(ctx, _q1_plan(fid, did, row_begin=rb, row_end=re))
    sub = {k: np.ascontiguousarray(v[rb:re]) for k, v in fact.items()}
    es, ec = O.q1(sub, dim)
    got = (int(s[0]), int(c[0])) if len(s) else (0, 0)
    assert got == (es, ec)


@pytest.fixture(scope="module")
def star_small():
    n = 3_000_000
    fact = G.star_fact(n, seed=7)
    dims = G.star_dims(0)
    ctx = _open(256 << 20, 16 << 20)
    fid = {c: vx.vx_register_host_column(ctx, c, fact[c]) for c in fact}
    did = {d: {a: vx.vx_register_host_column(ctx, f"{d}.{a}", arr) for a, arr in dims[d].items()} for d in dims}
    yield ctx, fact, dims, fid, did
    vx.vx_close(ctx)


@pytest.mark.parametrize("name", list(G.star_templates().keys()))
@pytest.mark.parametrize("late", [vx.VX_LATE_AUTO, vx.VX_LATE_FORCE_LATE, vx.VX_LATE_FORCE_EARLY])
def test_star_templates_bit_exact(star_small, name, late):
    ctx, fact, dims, fid, did = star_small
    T = G.star_templates()[name]
    plan = vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, late)
    st, gid, s, c, stats = vx.vx_run_plan(ctx, plan)
    es, ec = O.star(T, fact, dims, nthreads=8)
    nz = np.nonzero(ec)[0]
    assert st == vx.VX_OK
    assert np.array_equal(gid, nz.astype(np.uint64))
    assert np.array_equal(s, es[nz]) and np.array_equal(c, ec[nz])


@pytest.mark.parametrize("name", ["T2_10", "T3_1", "T1"])
def test_star_sparse_dimension_keys_use_hash_tables(name):
    """Dimension keys spread over a wide range (span > 2x rows) are stored in
    open-addressing tables instead of direct maps; results are unchanged."""
    n = 1_500_000
    fact = G.star_fact(n, seed=23)
    dims = G.star_dims(0)
    remap = lambda k: (k.astype(np.int64) * 7919 + 13).astype(np.int32)
    sdims = {d: dict(v, key=remap(v["key"])) for d, v in dims.items()}
    sfact = dict(fact)
    for _, _, fk in G.STAR_DIMS:
        sfact[fk] = remap(fact[fk])
    T = G.star_templates()[name]
    ctx = _open(256 << 20, 16 << 20)
    try:
        fid = {c: vx.vx_register_host_column(ctx, c, sfact[c]) for c in sfact}
        did = {d: {a: vx.vx_register_host_column(ctx, f"{d}.{a}", arr) for a, arr in sdims[d].items()}
               for d in sdims}
        for late in (vx.VX_LATE_FORCE_EARLY, vx.VX_LATE_FORCE_LATE):
            st, gid, s, c, _ = vx.vx_run_plan(ctx, vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, late))
            es, ec = O.star(T, sfact, sdims, nthreads=8)
            nz = np.nonzero(ec)[0]
            assert np.array_equal(gid, nz) and np.array_equal(s, es[nz]) and np.array_equal(c, ec[nz])
    finally:
        vx.vx_close(ctx)


def test_star_range_and_capacity(star_small):
    ctx, fact, dims, fid, did = star_small
    T = G.star_templates()["T3_10"]
    plan = vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO, 777, 2_345_679)
    st, gid, s, c, _ = vx.vx_run_plan(ctx, plan)
    es, ec = O.star(T, fact, dims, 777, 2_345_679, nthreads=8)
    nz = np.nonzero(ec)[0]
    assert np.array_equal(gid, nz) and np.array_equal(s, es[nz]) and np.array_equal(c, ec[nz])
    st, gid, s, c, _ = vx.vx_run_plan(ctx, plan, cap=3)
    assert st == vx.VX_E_CAPACITY and len(gid) == 3 and np.array_equal(gid, nz[:3])


def test_duplicate_dimension_key_reports_error():
    fact, dim = G.q1_tables(10_000)
    key = dim["key"].copy()
    key[5] = key[6]
    ctx = _open(32 << 20)
    try:
        fid = {c: vx.vx_register_host_column(ctx, c, fact[c]) for c in fact}
        did = {"key": vx.vx_register_host_column(ctx, "k", key),
               "year": vx.vx_register_host_column(ctx, "y", dim["year"]),
               "month": vx.vx_register_host_column(ctx, "m", dim["month"])}
        with pytest.raises(vx.VxError) as e:
            vx.vx_run_plan(ctx, _q1_plan(fid, did))
        assert e.value.status == vx.VX_E_DUPKEY
    finally:
        vx.vx_close(ctx)


def test_budget_too_small_is_nomem():
    fact, dim = G.q1_tables(100_000)
    ctx = _open(1 << 20, 8 << 20)
    try:
        fid = {c: vx.vx_register_host_column(ctx, c, fact[c]) for c in fact}
        did = {c: vx.vx_register_host_column(ctx, c, dim[c]) for c in ("key", "year", "month")}
        with pytest.raises(vx.VxError) as e:
            vx.vx_run_plan(ctx, _q1_plan(fid, did))
        assert e.value.status == vx.VX_E_NOMEM
    finally:
        vx.vx_close(ctx)


# ------------------------------------------------------------------ filter
@pytest.fixture(scope="module")
def filt():
    n = 5_000_123
    f = G.star_fact(n, seed=11)
    ctx = _open(128 << 20, 8 << 20)
    fid = {c: vx.vx_register_host_column(ctx, c, f[c]) for c in ("quantity", "discount", "price")}
    yield ctx, f, fid, n
    vx.vx_close(ctx)


@pytest.mark.parametrize("preds", [
    [("quantity", vx.VX_LT, 10, 0), ("discount", vx.VX_BETWEEN, 2, 5)],
    [("quantity", vx.VX_EQ, 7, 0)],
    [("price", vx.VX_GE, 9_990_000, 0), ("quantity", vx.VX_NE, 3, 0)],
    [("quantity", vx.VX_GT, 100, 0)],   # none pass
    [("quantity", vx.VX_GE, 1, 0)],     # all pass
    [("quantity", vx.VX_LT, -2**31, 0)],          # empty: nothing is below INT_MIN
    [("quantity", vx.VX_GT, 2**31 - 1, 0)],       # empty: nothing is above INT_MAX
    [("quantity", vx.VX_LE, 2**31 - 1, 0), ("discount", vx.VX_GE, -2**31, 0)],  # full ranges
    [("quantity", vx.VX_BETWEEN, 30, 20)],        # lo > hi: empty
    [("discount", vx.VX_NE, -5, 0), ("quantity", vx.VX_BETWEEN, -2**31, 2**31 - 1)],
])
def test_filter_rows_bit_exact(filt, preds):
    ctx, f, fid, n = filt
    opmap = {vx.VX_BETWEEN: O.BETWEEN, vx.VX_EQ: O.EQ, vx.VX_NE: O.NE, vx.VX_LT: O.LT, vx.VX_LE: O.LE,
             vx.VX_GT: O.GT, vx.VX_GE: O.GE}
    exp = O.filter_rows([(f[c], opmap[op], lo, hi) for c, op, lo, hi in preds], n)
    out = np.zeros(max(len(exp), 1), np.uint64)
    st, cnt = vx.vx_filter(ctx, [(fid[c], op, lo, hi) for c, op, lo, hi in preds], 0, 0, out)
    assert st == vx.VX_OK and cnt == len(exp)
    assert np.array_equal(out[:cnt], exp)


def test_filter_ranges_and_capacity(filt):
    ctx, f, fid, n = filt
    preds = [(fid["quantity"], vx.VX_LT, 25, 0)]
    for rb, re in [(1, 2049), (2047, 1_048_577), (4_999_000, 0), (17, 17)]:
        re_eff = n if re == 0 else re
        exp = O.filter_rows([(f["quantity"][rb:re_eff], O.LT, 25, 0)], re_eff - rb, row0=rb)
        out = np.zeros(max(len(exp), 1), np.uint64)
        st, cnt = vx.vx_filter(ctx, preds, rb, re, out)
        assert cnt == len(exp) and np.array_equal(out[:cnt], exp)
    exp = O.filter_rows([(f["quantity"], O.LT, 25, 0)], n)
    small = np.zeros(1000, np.uint64)
    st, cnt = vx.vx_filter(ctx, preds, 0, 0, small)
    assert st == vx.VX_E_CAPACITY and cnt == len(exp) and np.array_equal(small, exp[:1000])
    st, cnt = vx.vx_filter(ctx, preds, 0, 0, None)
    assert st == vx.VX_OK and cnt == len(exp)


# ------------------------------------------------------------------ group-by
def test_groupby_fact_columns_bit_exact(filt):
    ctx, f, fid, n = filt
    st, gid, s, c, _ = vx.vx_groupby(ctx, [(fid["discount"], 11), (fid["quantity"], 51)], vx.VX_AGG_MUL,
                                     fid["price"], fid["discount"], [(fid["quantity"], vx.VX_LE, 40, 0)])
    # oracle: a star query without dimensions whose group keys are fact columns
    q = O.OrStarQuery()
    q.n = n
    q.n_dims = 0
    q.n_fact_preds = 1
    q.fact_preds[0].col, q.fact_preds[0].op, q.fact_preds[0].lo, q.fact_preds[0].hi = \
        f["quantity"].ctypes.data, O.LE, 40, 0
    q.n_group_keys = 2
    q.group_keys[0].dim, q.group_keys[0].card, q.group_keys[0].fact_col = -1, 11, f["discount"].ctypes.data
    q.group_keys[1].dim, q.group_keys[1].card, q.group_keys[1].fact_col = -1, 51, f["quantity"].ctypes.data
    q.agg_op, q.agg_a, q.agg_b = O.AGG_MUL, f["price"].ctypes.data, f["discount"].ctypes.data
    es, ec = O.star_raw(q, nthreads=8)
    nz = np.nonzero(ec)[0]
    assert st == vx.VX_OK and np.array_equal(gid, nz) and np.array_equal(s, es[nz]) and np.array_equal(c, ec[nz])
    # invariant: group sums add up to the ungrouped total
    st, gid1, s1, c1, _ = vx.vx_groupby(ctx, [], vx.VX_AGG_MUL, fid["price"], fid["discount"],
                                        [(fid["quantity"], vx.VX_LE, 40, 0)])
    assert int(s1[0]) == int(s.astype(object).sum()) - (2**64 if int(s.astype(object).sum()) >= 2**63 else 0) or \
        (int(s1[0]) - int(s.astype(object).sum())) % 2**64 == 0
    assert int(c1[0]) == int(c.sum())


def test_groupby_code_out_of_range_is_error(filt):
    ctx, f, fid, n = filt
    with pytest.raises(vx.VxError) as e:
        vx.vx_groupby(ctx, [(fid["quantity"], 10)], vx.VX_AGG_COUNT, -1, -1, [])
    assert e.value.status == vx.VX_E_RANGE


@pytest.mark.parametrize("late", [vx.VX_LATE_FORCE_EARLY, vx.VX_LATE_FORCE_LATE])
def test_star_direct_maps_of_every_value_width(late):
    """Grouping by part brand (250) x supplier city (250) x year (7) gives the
    part map contributions up to 249 * 1750 (4-byte values), the supplier map up
    to 249 * 7 (2 bytes) and the date map up to 6 (1 byte); 437,500 groups
    accumulate in global memory.  Every group against the oracle."""
    n = 3_000_007
    fact, dims = G.star_fact(n, seed=23), G.star_dims(0)
    T = {"dims": [{"dim": "part", "fk": "fk_part", "preds": [("mfgr", 0, 3)]},
                  {"dim": "supp", "fk": "fk_supp", "preds": []},
                  {"dim": "date", "fk": "date_fk", "preds": [("year", 1, 6)]}],
         "fact_preds": [("discount", 1, 9)],
         "group": [("part", "brand"), ("supp", "city"), ("date", "year")],
         "agg": ("sub", "price", "cost")}
    ctx = _open(256 << 20, 8 << 20)
    try:
        fid = {c: vx.vx_register_host_column(ctx, c, fact[c]) for c in fact}
        did = {d: {a: vx.vx_register_host_column(ctx, f"{d}.{a}", arr) for a, arr in dims[d].items()} for d in dims}
        st, gid, s, c, stats = vx.vx_run_plan(ctx, vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, late), 1 << 19)
    finally:
        vx.vx_close(ctx)
    es, ec = O.star(T, fact, dims, nthreads=8)
    nz = np.nonzero(ec)[0]
    assert st == vx.VX_OK and len(nz) > 65536
    assert np.array_equal(gid, nz) and np.array_equal(s, es[nz]) and np.array_equal(c, ec[nz])
