"""Failure detection without a GPU fault: the executor's host-side wait limit.

The immediate schedule gives up when no chunk has completed a step (load,
kernel or store) for wait_timeout_ms.  A 1 ms limit on a plan whose chunks
take about 5 ms each over the host link (1 GiB chunks) makes that wait run
out with nothing wrong on the device: the call returns VX_E_TIMEOUT after
draining the work it had issued, and the same context then runs the plan to
the oracle's result under the default limit.  A limit
that each step meets never expires, however long the whole call takes.
"""
import numpy as np
import pytest

import datagen as G
import oracle as O

pytestmark = pytest.mark.gpu

vx = pytest.importorskip("paper_2502_09541_gb300")

ROWS = 100_000_000


@pytest.fixture(scope="module")
def star_ctx():
    fact = G.star_fact(ROWS, seed=5)
    dims = G.star_dims(0)
    c = vx.vx_open(4 << 30)
    try:
        fid = {k: vx.vx_register_host_column(c, k, fact[k]) for k in fact}
        did = {d: {a: vx.vx_register_host_column(c, f"{d}.{a}", arr) for a, arr in dims[d].items()}
               for d in dims}
        yield c, fact, dims, fid, did
    finally:
        vx.vx_close(c)


def test_wait_limit_expires_and_context_stays_usable(star_ctx):
    c, fact, dims, fid, did = star_ctx
    T = G.star_templates()["T3_1"]
    plan = vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_FORCE_EARLY)
    cfg = vx.vx_get_config(c)
    default_limit = cfg.wait_timeout_ms
    cfg.chunk_bytes = 1 << 30
    cfg.n_slots = 3
    cfg.wait_timeout_ms = 1
    vx.vx_set_config(c, cfg)
    try:
        with pytest.raises(vx.VxError) as e:
            vx.vx_run_plan(c, plan)
        assert e.value.status == vx.VX_E_TIMEOUT
        assert "wait limit" in str(e.value)
    finally:
        cfg.wait_timeout_ms = default_limit
        vx.vx_set_config(c, cfg)
    st, gid, s, cnt, stats = vx.vx_run_plan(c, plan)
    assert st == vx.VX_OK and stats["chunks"] >= 3
    es, ec = O.star(T, fact, dims, nthreads=16)
    nz = np.nonzero(ec)[0]
    assert np.array_equal(gid, nz) and np.array_equal(s, es[nz]) and np.array_equal(cnt, ec[nz])


def test_progressing_pipeline_outlives_its_wait_limit(star_ctx):
    """The limit bounds each wait, not the call: 8 MiB chunks complete far
    faster than a 5 ms limit, while the whole plan (2.4 GB over the link)
    takes longer than it."""
    c, fact, dims, fid, did = star_ctx
    T = G.star_templates()["T2_1"]
    plan = vx.make_plan(T, fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_FORCE_EARLY)
    cfg = vx.vx_get_config(c)
    default_limit, default_chunk = cfg.wait_timeout_ms, cfg.chunk_bytes
    cfg.chunk_bytes = 8 << 20
    cfg.wait_timeout_ms = 5
    vx.vx_set_config(c, cfg)
    try:
        st, gid, s, cnt, stats = vx.vx_run_plan(c, plan)
    finally:
        cfg.wait_timeout_ms = default_limit
        cfg.chunk_bytes = default_chunk
        vx.vx_set_config(c, cfg)
    assert st == vx.VX_OK and stats["ms_total"] > 5
    es, ec = O.star(T, fact, dims, nthreads=16)
    nz = np.nonzero(ec)[0]
    assert np.array_equal(gid, nz) and np.array_equal(s, es[nz]) and np.array_equal(cnt, ec[nz])


def test_radix_lookback_limit_gives_up_with_a_status():
    """The one-sweep radix passes wait for their predecessor tiles' published
    counts with a bounded poll.  A limit of one poll makes some waits run out
    (thousands of tiles race): the pass records it in its error word, keeps
    every write inside the buffers, and the call returns VX_E_TIMEOUT instead
    of hanging; the same context then sorts correctly at the default limit."""
    n = 20_000_000
    k, r = G.sort_input(n, "uniform", seed=2)
    c = vx.vx_open(1 << 30)
    try:
        cfg = vx.vx_get_config(c)
        cfg.lookback_spin_limit = 1
        vx.vx_set_config(c, cfg)
        with pytest.raises(vx.VxError) as e:
            vx.vx_radix_sort_pairs(c, k, r)
        assert e.value.status == vx.VX_E_TIMEOUT and "look-back" in str(e.value)
        cfg.lookback_spin_limit = 0
        vx.vx_set_config(c, cfg)
        ok, orr = vx.vx_radix_sort_pairs(c, k, r)
    finally:
        vx.vx_close(c)
    ek, er = O.sort_pairs(k, r)
    assert np.array_equal(ok, ek) and np.array_equal(orr, er)
