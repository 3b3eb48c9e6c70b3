"""Per-chunk cardinality regressor: the device ridge fit against the fp64
oracle, the statistics log against exact counts, and per-chunk late/early
materialization on a fact table whose selectivity is clustered by chunk."""
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


@pytest.mark.parametrize("n,d,lam", [(5000, 6, 0.0), (300, 4, 1e-3), (17, 8, 0.5)])
def test_ridge_fit_matches_oracle(ctx, n, d, lam):
    rng = np.random.default_rng(n)
    X = rng.normal(size=(n, d)).astype(np.float32)
    y = (X @ rng.normal(size=d) + 0.1 * rng.normal(size=n)).astype(np.float32)
    w = vx.vx_regressor_fit(ctx, X, y, lam)
    wo = O.lstsq_ridge(X.astype(np.float64), y.astype(np.float64), lam)
    assert np.allclose(w, wo, rtol=1e-4, atol=1e-5), (w, wo)


def test_singular_system_is_reported(ctx):
    X = np.ones((10, 2), np.float32)
    with pytest.raises(vx.VxError):
        vx.vx_regressor_fit(ctx, X, np.ones(10, np.float32), 0.0)


CLUSTER_T = {
    "dims": [{"dim": "cust", "fk": "fk_cust", "preds": [("nation", 0, 11)]},
             {"dim": "date", "fk": "date_fk", "preds": [("year", 5, 6)]}],
    "fact_preds": [("discount", 0, 2)],
    "group": [("date", "year"), ("cust", "nation")],
    "agg": ("sub", "price", "cost"),
}


def _open_with(fact, dims, budget=256 << 20, chunk=8 << 20):
    c = vx.vx_open(budget)
    cfg = vx.vx_get_config(c)
    cfg.chunk_bytes = chunk
    vx.vx_set_config(c, cfg)
    fid = {k: vx.vx_register_host_column(c, k, fact[k]) for k in fact}
    did = {d: {a: vx.vx_register_host_column(c, f"{d}.{a}", arr) for a, arr in dims[d].items()} for d in dims}
    return c, fid, did


def _check(res, T, fact, dims):
    st, gid, s, c, stats = res
    es, ec = O.star(T, fact, dims, nthreads=8)
    nz = np.nonzero(ec)[0]
    assert st == vx.VX_OK
    assert np.array_equal(gid, nz) and np.array_equal(s, es[nz]) and np.array_equal(c, ec[nz])
    return stats


def _chunk_rows(chunk_bytes, n_cols):
    """Rows per chunk: chunk bytes over all referenced int32 columns, rounded
    down to a multiple of 1024."""
    return max(chunk_bytes // (4 * n_cols) // 1024 * 1024, 1024)


def test_statistics_log_matches_exact_counts():
    n = 3_000_000
    fact = G.star_fact(n, seed=3)
    dims = G.star_dims(0)
    c, fid, did = _open_with(fact, dims)
    try:
        cfg = vx.vx_get_config(c)
        cfg.log_chunk_stats = 1
        vx.vx_set_config(c, cfg)
        T = G.star_templates()["T3_10"]  # 7 referenced fact columns
        stats = _check(vx.vx_run_plan(c, vx.make_plan(T, fid, did, G.STAR_ATTR_CARD)), T, fact, dims)
        X, y = vx.vx_chunk_log(c)
        cr = _chunk_rows(8 << 20, 7)
        assert stats["chunks"] == -(-n // cr) and X.shape == (stats["chunks"], 4)
        assert np.all(X[:, 0] == 1) and np.all((X[:, 1:3] >= 0) & (X[:, 1:3] <= 1))
        rows = np.array([min(cr, n - i * cr) for i in range(stats["chunks"])], np.float64)
        # the logged targets are exact survivor fractions per chunk
        surv = np.rint(y.astype(np.float64) * rows)
        assert int(surv.sum()) == stats["survivors"]
        vx.vx_chunk_log_clear(c)
        assert vx.vx_chunk_log(c)[1].size == 0
    finally:
        vx.vx_close(c)


def test_per_chunk_materialization_on_clustered_table():
    n = 6_000_000
    dims = G.star_dims(0)
    uni = G.star_fact(n // 2, seed=5)
    clu = G.star_fact(n, seed=6, clustered_date=True)
    c = vx.vx_open(256 << 20)
    try:
        cfg = vx.vx_get_config(c)
        cfg.chunk_bytes = 8 << 20
        vx.vx_set_config(c, cfg)
        did = {d: {a: vx.vx_register_host_column(c, f"{d}.{a}", arr) for a, arr in dims[d].items()} for d in dims}
        fu = {k: vx.vx_register_host_column(c, "u." + k, uni[k]) for k in uni}
        fc = {k: vx.vx_register_host_column(c, "c." + k, clu[k]) for k in clu}
        # plain runs over the uniform table log the regressor's training data
        cfg.log_chunk_stats = 1
        vx.vx_set_config(c, cfg)
        for name in ["T2_0.1", "T2_1", "T2_10", "T3_0.1", "T3_1", "T3_10"]:
            T = G.star_templates()[name]
            _check(vx.vx_run_plan(c, vx.make_plan(T, fu, did, G.STAR_ATTR_CARD)), T, uni, dims)
        cfg.log_chunk_stats = 0
        vx.vx_set_config(c, cfg)
        X, y = vx.vx_chunk_log(c)
        plan_auto = vx.make_plan(CLUSTER_T, fc, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO)
        plan_pc = vx.make_plan(CLUSTER_T, fc, did, G.STAR_ATTR_CARD, vx.VX_LATE_PER_CHUNK)
        a = _check(vx.vx_run_plan(c, plan_auto), CLUSTER_T, clu, dims)
        p0 = _check(vx.vx_run_plan(c, plan_pc), CLUSTER_T, clu, dims)  # sampled per-chunk estimate
        w, used = vx.vx_regressor_train(c, 1e-6)
        assert used == len(y) > 20 and np.all(np.isfinite(w))
        # least squares over a family that contains the raw sampled estimate
        # (w = e_2) fits the log at least as well as that estimate
        assert np.mean((X @ w - y) ** 2) <= np.mean((X[:, 2] - y) ** 2) + 1e-7
        p1 = _check(vx.vx_run_plan(c, plan_pc), CLUSTER_T, clu, dims)  # regressor's per-chunk estimate
        # the qualifying years sit in the last chunks: they stage price and
        # cost, the other chunks read nothing by zero-copy; one global
        # decision reads every survivor by zero-copy instead
        assert a["late_mask"] == 3 and a["late_chunks"] == 0
        for p in (p0, p1):
            assert 0 < p["late_chunks"] < p["chunks"]
            assert p["bytes_h2d"] + p["bytes_zero_copy"] < a["bytes_h2d"] + a["bytes_zero_copy"]
    finally:
        vx.vx_close(c)


@pytest.mark.parametrize("graphs", [0, 1])
def test_survivor_lists_sized_by_prediction_overflow_reruns_exactly(graphs):
    """The regressor sizes each slot's survivor list.  Zero weights predict
    no survivors, so every late chunk overflows its list: the chunks are
    flagged on the device, left out of the aggregate and rerun with a full
    list, and the result stays the oracle's.  A trained regressor gives lists
    far below the worst case of one entry per chunk row and no reruns."""
    n = 4_000_000
    fact = G.star_fact(n, seed=11)
    dims = G.star_dims(0)
    c, fid, did = _open_with(fact, dims)
    try:
        cfg = vx.vx_get_config(c)
        cfg.use_graphs = graphs
        vx.vx_set_config(c, cfg)
        worst = 8 * _chunk_rows(8 << 20, 6)  # T2: 4 row-logic columns + price, cost
        T = G.star_templates()["T2_10"]  # ~10 % of a chunk's rows survive
        plan = vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_PER_CHUNK)
        vx.vx_regressor_set(c, np.zeros(4, np.float32))
        for _ in range(2):  # with graphs: capture, then replay
            bad = _check(vx.vx_run_plan(c, plan), T, fact, dims)
            assert bad["late_chunks"] == bad["chunks"] and bad["overflow_retries"] == bad["chunks"]
            assert bad["surv_list_bytes"] < worst
        # the sampled selectivity itself (w = e_2) as the prediction, on a
        # template below TH (~1 %)
        T = G.star_templates()["T2_1"]
        plan = vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_PER_CHUNK)
        vx.vx_regressor_set(c, np.array([0, 0, 1, 0], np.float32))
        good = _check(vx.vx_run_plan(c, plan), T, fact, dims)
        assert good["late_chunks"] == good["chunks"] and good["overflow_retries"] == 0
        assert good["surv_list_bytes"] < worst / 20
    finally:
        vx.vx_close(c)
