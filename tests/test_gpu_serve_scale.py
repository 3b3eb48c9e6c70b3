"""Serving at the workload's scale: a 600M-row star table shared by 1,000 star
queries (log-uniform sizes from 1e6 rows to the whole table, Poisson
arrivals) and by sort- and join-shaped queries on shared sort and join
tables.  Every star query's result in the mix equals its result alone
(vx_run_plan) bit for bit; the oracle checks the smallest queries and one
whole-table query; every sort is checked by its order, its stability and its
multiset against numpy, every join against the oracle."""
import threading
import time

import numpy as np
import pytest

import datagen as G
import oracle as O

pytestmark = pytest.mark.gpu

vx = pytest.importorskip("paper_2502_09541_gb300")

N = 600_000_000
N_STAR = 1000
N_SORT, N_BUILD, N_PROBE = 20_000_000, 2_000_000, 50_000_000


def _star_mix(rng, n):
    names = list(G.star_templates().keys())
    out = []
    for _ in range(n):
        size = int(np.exp(rng.uniform(np.log(1_000_000), np.log(N))))
        rb = int(rng.integers(0, N - size + 1))
        out.append((names[int(rng.integers(0, len(names)))], rb, rb + size))
    return out


def test_serving_at_scale_mix_equals_alone():
    fact = G.star_fact(N, seed=23)
    dims = G.star_dims(0)
    sk, sr = G.sort_input(N_SORT, "zipf", seed=8)
    bk, bp = G.build_side(N_BUILD)
    pk = G.probe_side(N_PROBE, N_BUILD, 1.0, 1.0, seed=12)
    rng = np.random.default_rng(31)
    mix = _star_mix(rng, N_STAR)
    mix.append((list(G.star_templates().keys())[4], 0, N))  # one whole-table query
    ops = []
    for i in range(10):
        n = N_SORT if i % 2 == 0 else N_PROBE
        size = int(np.exp(rng.uniform(np.log(1_000_000), np.log(n))))
        rb = int(rng.integers(0, n - size + 1))
        ops.append(("sort" if i % 2 == 0 else "join", rb, rb + size))

    c = vx.vx_open(16 << 30)
    try:
        fid = {k: vx.vx_register_host_column(c, k, fact[k]) for k in fact}
        did = {d: {a: vx.vx_register_host_column(c, f"{d}.{a}", arr) for a, arr in dims[d].items()} for d in dims}
        kc = vx.vx_register_host_column(c, "sk", sk)
        rc = vx.vx_register_host_column(c, "sr", sr)
        bkc = vx.vx_register_host_column(c, "bk", bk)
        bpc = vx.vx_register_host_column(c, "bp", bp)
        pkc = vx.vx_register_host_column(c, "pk", pk)
        plans = [vx.make_plan(G.star_templates()[n], fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO, rb, re)
                 for n, rb, re in mix]
        alone = [vx.vx_run_plan(c, p) for p in plans]

        vx.vx_serve_start(c, chunk_rows=1 << 21, max_active=32)
        tickets, op_tickets, outs = [], [], []

        def submitter():  # Poisson arrivals, the operators spread through the star stream
            arr = np.random.default_rng(5)
            every = len(plans) // len(ops)
            for i, p in enumerate(plans):
                tickets.append(vx.vx_submit(c, p))
                if i % every == 0 and i // every < len(ops):
                    kind, rb, re = ops[i // every]
                    req = vx.vx_op_request()
                    req.row_begin, req.row_end = rb, re
                    req.device_budget = 2 << 30
                    if kind == "sort":
                        req.kind, req.key_col, req.val_col = vx.VX_QUERY_SORT, kc, rc
                        ok, orr = np.empty(re - rb, np.uint64), np.empty(re - rb, np.uint32)
                        req.out_keys, req.out_rowids = ok.ctypes.data, orr.ctypes.data
                        outs.append((ok, orr))
                    else:
                        req.kind, req.key_col, req.val_col, req.probe_col = vx.VX_QUERY_JOIN, bkc, bpc, pkc
                        outs.append(None)
                    op_tickets.append(vx.vx_submit_op(c, req))
                time.sleep(float(arr.exponential(0.004)))

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        results = [vx.vx_wait(c, t, 600_000) for t in tickets]
        op_res = [vx.vx_wait_op(c, t) for t in op_tickets]
        stats = vx.vx_serve_stats_get(c)
        vx.vx_serve_stop(c)
    finally:
        vx.vx_close(c)

    assert stats["failed"] == 0
    assert stats["completed_kind"] == [len(plans), 5, 5]
    assert stats["active_peak"] > 1 and 0 < stats["p50_ms"] <= stats["p99_ms"]
    for (name, rb, re), a, r in zip(mix, alone, results):
        assert r[0] == vx.VX_OK
        for x, y in zip(a[1:4], r[1:4]):
            assert np.array_equal(x, y), (name, rb, re)
    # the oracle: the five smallest queries and the whole-table query
    order = sorted(range(len(mix) - 1), key=lambda i: mix[i][2] - mix[i][1])[:5] + [len(mix) - 1]
    for i in order:
        name, rb, re = mix[i]
        es, ec = O.star(G.star_templates()[name], fact, dims, rb, re, nthreads=16)
        nz = np.nonzero(ec)[0]
        r = results[i]
        assert np.array_equal(r[1], nz) and np.array_equal(r[2], es[nz]) and np.array_equal(r[3], ec[nz]), mix[i]
    for (kind, rb, re), o, r in zip(ops, outs, op_res):
        if kind == "sort":
            k, v = o
            assert np.all(k[1:] >= k[:-1])  # ordered
            same = k[1:] == k[:-1]
            assert np.all(v[1:][same] > v[:-1][same])  # stable: row ids rise within equal keys
            assert np.array_equal(np.sort(v), sr[rb:re])  # a permutation of the range's row ids
            assert np.array_equal(k, np.sort(sk[rb:re]))
        else:
            j = r["join"]
            assert (j["count"], j["payload_sum"], j["pair_fp"]) == O.join(bk, bp, pk[rb:re], probe_row0=rb,
                                                                         nthreads=16)
