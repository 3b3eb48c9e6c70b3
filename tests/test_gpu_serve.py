"""Serving: continuous batching over a shared circular scan.  Every query's
result in the mix must equal its result alone (vx_run_plan) and the oracle's,
bit-exactly; queries arriving while others run attach to the running scan."""
import threading
import time

import numpy as np
import pytest

import datagen as G
import oracle as O

pytestmark = pytest.mark.gpu

vx = pytest.importorskip("paper_2502_09541_gb300")

N = 6_000_000


@pytest.fixture(scope="module")
def tables():
    return G.star_fact(N, seed=17), G.star_dims(0)


def _open(budget, fact, dims):
    c = vx.vx_open(budget)
    fid = {k: vx.vx_register_host_column(c, k, fact[k]) for k in fact}
    did = {d: {a: vx.vx_register_host_column(c, f"{d}.{a}", arr) for a, arr in dims[d].items()} for d in dims}
    return c, fid, did


def _mix(n_queries, seed):
    """(template, row_begin, row_end) with log-uniform sizes over the table."""
    rng = np.random.default_rng(seed)
    names = list(G.star_templates().keys())
    out = []
    for _ in range(n_queries):
        size = int(np.exp(rng.uniform(np.log(50_000), np.log(N))))
        rb = int(rng.integers(0, N - size + 1))
        out.append((names[int(rng.integers(0, len(names)))], rb, rb + size))
    return out


def test_mix_equals_alone_and_oracle(tables):
    fact, dims = tables
    mix = _mix(30, 1)
    c, fid, did = _open(1 << 30, fact, dims)
    try:
        alone = []
        for name, rb, re in mix:
            T = G.star_templates()[name]
            alone.append(vx.vx_run_plan(c, vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO, rb, re)))
        vx.vx_serve_start(c, chunk_rows=1 << 19, max_active=8)
        tickets = []

        def submitter():  # Poisson-like arrivals while earlier queries run
            rng = np.random.default_rng(2)
            for name, rb, re in mix:
                T = G.star_templates()[name]
                tickets.append(vx.vx_submit(c, vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO, rb, re)))
                time.sleep(float(rng.exponential(0.002)))

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        results = [vx.vx_wait(c, t) for t in tickets]
        stats = vx.vx_serve_stats_get(c)
        vx.vx_serve_stop(c)
        assert stats["completed"] == len(mix) and stats["failed"] == 0
        assert stats["active_peak"] > 1  # queries overlapped on the device
        assert 0 < stats["p50_ms"] <= stats["p99_ms"] <= stats["max_ms"]
        for (name, rb, re), a, r in zip(mix, alone, results):
            assert r[0] == vx.VX_OK
            for x, y in zip(a[1:4], r[1:4]):
                assert np.array_equal(x, y), (name, rb, re)
            assert r[4]["ms_total"] > 0
        # spot-check against the oracle
        for (name, rb, re), r in list(zip(mix, results))[:6]:
            T = G.star_templates()[name]
            es, ec = O.star(T, fact, dims, rb, re, nthreads=8)
            nz = np.nonzero(ec)[0]
            assert np.array_equal(r[1], nz) and np.array_equal(r[2], es[nz]) and np.array_equal(r[3], ec[nz])
    finally:
        vx.vx_close(c)


def test_admission_under_a_small_budget(tables):
    fact, dims = tables
    mix = _mix(10, 3)
    # the staging ring plus the dimension tables leave room for few queries
    c, fid, did = _open(160 << 20, fact, dims)
    try:
        vx.vx_serve_start(c, chunk_rows=1 << 18, max_active=4)
        tickets = [vx.vx_submit(c, vx.make_plan(G.star_templates()[n], fid, did, G.STAR_ATTR_CARD,
                                                vx.VX_LATE_AUTO, rb, re)) for n, rb, re in mix]
        results = [vx.vx_wait(c, t) for t in tickets]
        stats = vx.vx_serve_stats_get(c)
        assert stats["completed"] == len(mix) and stats["active_peak"] <= 4
        for (name, rb, re), r in zip(mix, results):
            T = G.star_templates()[name]
            es, ec = O.star(T, fact, dims, rb, re, nthreads=8)
            nz = np.nonzero(ec)[0]
            assert np.array_equal(r[1], nz) and np.array_equal(r[2], es[nz]) and np.array_equal(r[3], ec[nz])
    finally:
        vx.vx_close(c)  # also stops the engine


def test_poll_unknown_ticket_and_empty_range(tables):
    fact, dims = tables
    c, fid, did = _open(512 << 20, fact, dims)
    try:
        vx.vx_serve_start(c)
        with pytest.raises(vx.VxError):
            vx.vx_poll(c, 12345)
        T = G.star_templates()["T2_1"]
        t = vx.vx_submit(c, vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO, 100, 100))
        st, gid, s, cnt, stats = vx.vx_wait(c, t)
        assert st == vx.VX_OK and len(gid) == 0
    finally:
        vx.vx_close(c)


def test_sort_and_join_queries_in_the_mix(tables):
    """Sort- and join-shaped queries (log-uniform row ranges of shared sort
    and join tables) served beside star queries: each result equals the same
    operator run alone on the context and the oracle, and the operators'
    work overlapped the star scan (their latency counted per kind)."""
    fact, dims = tables
    ns, nb, npr = 3_000_000, 400_000, 5_000_000
    sk, sr = G.sort_input(ns, "zipf", seed=4)
    bk, bp = G.build_side(nb)
    pk = G.probe_side(npr, nb, 0.5, 1.0, seed=6)
    c, fid, did = _open(1 << 30, fact, dims)
    try:
        kc = vx.vx_register_host_column(c, "sk", sk)
        rc = vx.vx_register_host_column(c, "sr", sr)
        a = vx.vx_register_host_column(c, "bk", bk)
        b = vx.vx_register_host_column(c, "bp", bp)
        p = vx.vx_register_host_column(c, "pk", pk)
        rng = np.random.default_rng(9)
        ops = []
        for i in range(8):
            n = ns if i % 2 == 0 else npr
            size = int(np.exp(rng.uniform(np.log(100_000), np.log(n))))
            rb = int(rng.integers(0, n - size + 1))
            ops.append(("sort" if i % 2 == 0 else "join", rb, rb + size, i % 4 == 0))
        # alone: the same operators on the context itself (sort on a copy of the range)
        alone = []
        for kind, rb, re, merge in ops:
            if kind == "sort":
                c2 = vx.vx_open(256 << 20)
                kcopy, rcopy = sk[rb:re].copy(), sr[rb:re].copy()  # registered: kept alive until closed
                try:
                    k2 = vx.vx_register_host_column(c2, "k", kcopy)
                    r2 = vx.vx_register_host_column(c2, "r", rcopy)
                    ok, orr = np.empty(re - rb, np.uint64), np.empty(re - rb, np.uint32)
                    o = vx.vx_sort_opts()
                    o.plan = vx.VX_SORT_MERGE if merge else vx.VX_SORT_PARTITION
                    vx.vx_sort(c2, k2, r2, ok, orr, o)
                finally:
                    vx.vx_close(c2)
                alone.append((ok, orr))
            else:
                alone.append(None)
        vx.vx_serve_start(c, chunk_rows=1 << 19, max_active=8)
        star_mix = _mix(12, 5)
        outs, tickets, stars = [], [], []
        for i, (kind, rb, re, merge) in enumerate(ops):
            name, srb, sre = star_mix[i]
            stars.append((name, srb, sre, vx.vx_submit(c, vx.make_plan(G.star_templates()[name], fid, did,
                                                                       G.STAR_ATTR_CARD, vx.VX_LATE_AUTO, srb, sre))))
            req = vx.vx_op_request()
            req.row_begin, req.row_end = rb, re
            req.device_budget = 192 << 20
            if kind == "sort":
                req.kind, req.key_col, req.val_col = vx.VX_QUERY_SORT, kc, rc
                ok, orr = np.empty(re - rb, np.uint64), np.empty(re - rb, np.uint32)
                req.out_keys, req.out_rowids = ok.ctypes.data, orr.ctypes.data
                req.sort.plan = vx.VX_SORT_MERGE if merge else vx.VX_SORT_PARTITION
                outs.append((ok, orr))
            else:
                req.kind, req.key_col, req.val_col, req.probe_col = vx.VX_QUERY_JOIN, a, b, p
                outs.append(None)
            tickets.append(vx.vx_submit_op(c, req))
            time.sleep(0.002)
        res = [vx.vx_wait_op(c, t) for t in tickets]
        star_res = [vx.vx_wait(c, t) for *_, t in stars]
        stats = vx.vx_serve_stats_get(c)
        vx.vx_serve_stop(c)
        assert stats["failed"] == 0
        assert stats["completed_kind"] == [len(stars), 4, 4]
        for k in range(3):
            assert 0 < stats["p50_kind_ms"][k] <= stats["p99_kind_ms"][k]
        for (kind, rb, re, merge), o, al, r in zip(ops, outs, alone, res):
            if kind == "sort":
                ek, er = O.sort_pairs(sk[rb:re], sr[rb:re])
                assert np.array_equal(o[0], ek) and np.array_equal(o[1], er)
                assert np.array_equal(al[0], ek) and np.array_equal(al[1], er)
            else:
                j = r["join"]
                exp = O.join(bk, bp, pk[rb:re], probe_row0=rb, nthreads=8)
                assert (j["count"], j["payload_sum"], j["pair_fp"]) == exp
                cj = vx.vx_open(256 << 20)
                pcopy = pk[rb:re].copy()  # registered: kept alive until closed
                try:
                    d = vx.vx_join(cj, vx.vx_register_host_column(cj, "a", bk), vx.vx_register_host_column(cj, "b", bp),
                                   vx.vx_register_host_column(cj, "p", pcopy), vx.vx_join_opts())
                finally:
                    vx.vx_close(cj)
                assert (d["count"], d["payload_sum"]) == (j["count"], j["payload_sum"])
        for (name, srb, sre, _), r in zip(stars, star_res):
            es, ec = O.star(G.star_templates()[name], fact, dims, srb, sre, nthreads=8)
            nz = np.nonzero(ec)[0]
            assert r[0] == vx.VX_OK and np.array_equal(r[1], nz) and np.array_equal(r[2], es[nz])
    finally:
        vx.vx_close(c)
