"""Operator-at-a-time execution with host intermediates (Section 6.4's
chaining of IO-decoupled operators) against the oracle and the fused plan:
every star template, a ragged row range, fact group keys, and a budget far
smaller than the intermediates (32 MiB, of which the dimension tables take
about 10 MB, against 48 MB of entries per intermediate), so
both the staged and the zero-copy column reads of the operators run."""
import numpy as np
import pytest

import datagen as G
import oracle as O

pytestmark = pytest.mark.gpu

vx = pytest.importorskip("paper_2502_09541_gb300")

N = 3_000_017


@pytest.fixture(scope="module")
def star():
    fact = G.star_fact(N, seed=13)
    dims = G.star_dims(0)
    c = vx.vx_open(32 << 20)
    cfg = vx.vx_get_config(c)
    cfg.chunk_bytes = 4 << 20
    vx.vx_set_config(c, cfg)
    fid = {k: vx.vx_register_host_column(c, k, fact[k]) for k in fact}
    did = {d: {a: vx.vx_register_host_column(c, f"{d}.{a}", arr) for a, arr in dims[d].items()} for d in dims}
    yield c, fact, dims, fid, did
    vx.vx_close(c)


@pytest.mark.parametrize("name", ["T1", "T2_0.1", "T2_1", "T2_10", "T3_0.1", "T3_1", "T3_10"])
@pytest.mark.parametrize("rng", [(0, 0), (123_457, 2_871_113)])
def test_operators_match_oracle_and_fused(star, name, rng):
    c, fact, dims, fid, did = star
    T = G.star_templates()[name]
    rb, re = rng
    plan = vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO, rb, re)
    st, gid, s, cnt, stats = vx.vx_run_plan_operators(c, plan)
    es, ec = O.star(T, fact, dims, rb, re or None, nthreads=8)
    nz = np.nonzero(ec)[0]
    assert st == vx.VX_OK
    assert np.array_equal(gid, nz) and np.array_equal(s, es[nz]) and np.array_equal(cnt, ec[nz])
    fused = vx.vx_run_plan(c, plan)
    assert np.array_equal(fused[1], gid) and np.array_equal(fused[2], s) and np.array_equal(fused[3], cnt)
    # the intermediates went through host memory: more than the whole budget for the dense ones
    assert stats["bytes_d2h"] > 0 and stats["chunks"] > 1


def test_operators_with_fact_group_keys(star):
    c, fact, dims, fid, did = star
    T = {"dims": [{"dim": "date", "fk": "date_fk", "preds": [("year", 2, 5)]}],
         "fact_preds": [("quantity", 10, 30)], "group": [("date", "year")], "agg": ("sum", "price", None)}
    plan = vx.make_plan(T, fid, did, G.STAR_ATTR_CARD)
    # add discount (11 codes) as a fact group key after the dimension key
    plan.n_group_keys = 2
    plan.group_keys[1] = vx.vx_plan_gkey(-1, 0, 11, fid["discount"])
    st, gid, s, cnt, stats = vx.vx_run_plan_operators(c, plan)
    fused = vx.vx_run_plan(c, plan)
    assert st == vx.VX_OK
    assert np.array_equal(fused[1], gid) and np.array_equal(fused[2], s) and np.array_equal(fused[3], cnt)
    # brute force over numpy: year code * 11 + discount
    d = dims["date"]
    year_of = np.full(2556, -1, np.int64)
    year_of[d["key"]] = d["year"]
    y = year_of[fact["date_fk"]]
    keep = (y >= 2) & (y <= 5) & (fact["quantity"] >= 10) & (fact["quantity"] <= 30)
    g = y[keep] * 11 + fact["discount"][keep]
    want_cnt = np.bincount(g, minlength=77)
    want_sum = np.bincount(g, weights=fact["price"][keep].astype(np.float64), minlength=77)
    assert np.array_equal(cnt, want_cnt[gid.astype(np.int64)])
    assert np.array_equal(s.astype(np.float64), want_sum[gid.astype(np.int64)])


def test_operators_empty_range_and_no_survivors(star):
    c, fact, dims, fid, did = star
    T = dict(G.star_templates()["T2_1"])
    plan = vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO, 500, 500)
    st, gid, s, cnt, stats = vx.vx_run_plan_operators(c, plan)
    assert st == vx.VX_OK and len(gid) == 0 and stats["rows"] == 0
    T = {"dims": [{"dim": "date", "fk": "date_fk", "preds": [("year", 9, 9)]}], "fact_preds": [],
         "group": [], "agg": ("count", None, None)}
    st, gid, s, cnt, stats = vx.vx_run_plan_operators(c, vx.make_plan(T, fid, did, G.STAR_ATTR_CARD))
    assert st == vx.VX_OK and len(gid) == 0
