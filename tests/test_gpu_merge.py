"""GPU parity of the sort-by-merging plan (Section 6.1: SortExKernel, then
MergeExKernel) against the oracle: the exact cut of sorted runs, the in-HBM
merge of runs, and the whole out-of-core sort through the merge plan, on the
three key distributions and on heavy ties.  Integer work: bit-exact."""
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


def _runs(n, n_runs, dist, seed=0, ragged=True):
    """n (key, row id) pairs cut into n_runs runs (ragged lengths, empty runs
    allowed), each run sorted stably as the first pass leaves it."""
    if dist == "ties":
        k = G.i32_uniform(n, 0, 4, seed, 7).astype(np.uint64) * np.uint64(2**61)
    else:
        k, _ = G.sort_input(n, dist, seed=seed)
    r = np.arange(n, dtype=np.uint32)
    if ragged:
        cuts = np.sort(G.u64_uniform(n_runs - 1, seed + 1, 11) % np.uint64(n + 1))
        cuts = np.concatenate([[0], cuts, [n]]).astype(np.uint64)
    else:
        cuts = np.linspace(0, n, n_runs + 1).astype(np.uint64)
    for a, b in zip(cuts[:-1], cuts[1:]):
        perm = np.argsort(k[a:b], kind="stable")
        k[a:b], r[a:b] = k[a:b][perm], r[a:b][perm]
    return k, r, cuts


@pytest.mark.parametrize("dist", ["uniform", "zipf", "runs", "ties"])
@pytest.mark.parametrize("n_runs", [1, 2, 11, 64])
def test_exact_splits_match_oracle(ctx, dist, n_runs):
    n = 1_000_003
    k, _, cuts = _runs(n, n_runs, dist, seed=n_runs)
    ranks = np.array([0, 1, 4095, 4096, 250_000, 500_001, n - 1, n, n + 5], np.uint64)
    got = vx.vx_exact_splits(ctx, k, cuts, ranks)
    for q, kk in enumerate(ranks.tolist()):
        assert np.array_equal(got[q], O.exact_cut(k, cuts, kk)), (q, kk)


def test_exact_splits_equal_keys_take_runs_in_order(ctx):
    k = np.full(300_000, 5, np.uint64)
    cuts = np.array([0, 1, 100_000, 100_000, 299_999, 300_000], np.uint64)
    got = vx.vx_exact_splits(ctx, k, cuts, np.array([150_000], np.uint64))
    assert got[0].tolist() == [1, 99_999, 0, 50_000, 0]


@pytest.mark.parametrize("dist", ["uniform", "zipf", "runs", "ties"])
@pytest.mark.parametrize("n,n_runs", [(1, 1), (2047, 2), (2049, 3), (100_003, 17), (777_777, 64), (600_000, 256)])
def test_merge_runs_bit_exact(ctx, dist, n, n_runs):
    k, r, cuts = _runs(n, n_runs, dist, seed=n)
    ok, orr = vx.vx_merge_runs(ctx, k, r, cuts)
    ek, er = O.sort_pairs(k, r)  # merging stable runs = the stable sort of their concatenation
    assert np.array_equal(ok, ek) and np.array_equal(orr, er)


@pytest.mark.parametrize("dist", ["uniform", "zipf", "runs"])
def test_sort_merge_plan_bit_exact(dist):
    """A 40 MiB budget forces several runs and several merge partitions."""
    n = 3_000_017
    k, r = G.sort_input(n, dist, seed=3)
    c = vx.vx_open(40 << 20)
    try:
        kc = vx.vx_register_host_column(c, "k", k)
        rc = vx.vx_register_host_column(c, "r", r)
        ok = np.empty(n, np.uint64)
        orr = np.empty(n, np.uint32)
        o = vx.vx_sort_opts()
        o.plan = vx.VX_SORT_MERGE
        st = vx.vx_sort(c, kc, rc, ok, orr, o)
    finally:
        vx.vx_close(c)
    ek, er = O.sort_pairs(k, r)
    assert np.array_equal(ok, ek) and np.array_equal(orr, er)
    assert st["plan"] == vx.VX_SORT_MERGE and st["n_runs"] > 1 and st["n_partitions"] > 1
    # exact cuts: partition sizes differ by at most one pair
    assert st["max_partition"] - st["min_partition"] <= 1


def test_sort_merge_plan_forced_partitions_and_slot_cap():
    n = 1_500_000
    k, r = G.sort_input(n, "zipf", seed=9)
    c = vx.vx_open(256 << 20)
    try:
        kc = vx.vx_register_host_column(c, "k", k)
        rc = vx.vx_register_host_column(c, "r", r)
        ok = np.empty(n, np.uint64)
        orr = np.empty(n, np.uint32)
        o = vx.vx_sort_opts()
        o.plan = vx.VX_SORT_MERGE
        o.n_partitions = 37
        o.max_slot_pairs = 200_000
        scratch = np.empty(12 * n, np.uint8)
        o.host_scratch = scratch.ctypes.data
        o.host_scratch_bytes = scratch.nbytes
        st = vx.vx_sort(c, kc, rc, ok, orr, o)
    finally:
        vx.vx_close(c)
    ek, er = O.sort_pairs(k, r)
    assert np.array_equal(ok, ek) and np.array_equal(orr, er)
    assert st["n_partitions"] == 37 and st["n_runs"] == (n + 196_607) // 196_608


def test_sort_merge_plan_empty_and_tiny():
    for n in (0, 1, 5):
        k, r = G.sort_input(n, "uniform", seed=n) if n else (np.zeros(0, np.uint64), np.zeros(0, np.uint32))
        c = vx.vx_open(64 << 20)
        try:
            kc = vx.vx_register_host_column(c, "k", k)
            rc = vx.vx_register_host_column(c, "r", r)
            ok = np.empty(max(n, 1), np.uint64)[:n]
            orr = np.empty(max(n, 1), np.uint32)[:n]
            o = vx.vx_sort_opts()
            o.plan = vx.VX_SORT_MERGE
            vx.vx_sort(c, kc, rc, ok, orr, o)
        finally:
            vx.vx_close(c)
        ek, er = O.sort_pairs(k, r)
        assert np.array_equal(ok, ek) and np.array_equal(orr, er)


def _merge_sort(k, r, budget=40 << 20, **opts):
    c = vx.vx_open(budget)
    try:
        kc = vx.vx_register_host_column(c, "k", k)
        rc = vx.vx_register_host_column(c, "r", r)
        ok = np.empty(len(k), np.uint64)
        orr = np.empty(len(k), np.uint32)
        o = vx.vx_sort_opts()
        o.plan = vx.VX_SORT_MERGE
        for name, v in opts.items():
            setattr(o, name, v)
        st = vx.vx_sort(c, kc, rc, ok, orr, o)
    finally:
        vx.vx_close(c)
    return ok, orr, st


def test_sort_merge_plan_natural_runs():
    """An input of 64 presorted runs is merged as it is (pass 1 skipped): the
    same output as the oracle and as the plan that sorts its chunks first."""
    n = 3_000_017
    k, r = G.sort_input(n, "runs", seed=5)
    ek, er = O.sort_pairs(k, r)
    ok, orr, st = _merge_sort(k, r)
    assert np.array_equal(ok, ek) and np.array_equal(orr, er)
    assert st["natural_runs"] == 1 and 1 < st["n_runs"] <= 64 and st["radix_pass_pairs"] == 0
    assert st["max_partition"] - st["min_partition"] <= 1
    ok2, orr2, st2 = _merge_sort(k, r, runs_mode=1)
    assert np.array_equal(ok2, ek) and np.array_equal(orr2, er) and st2["natural_runs"] == 0
    # a shuffled input: the sample finds descents, the chunks are sorted
    ku, ru = G.sort_input(n, "uniform", seed=5)
    oku, oru, stu = _merge_sort(ku, ru)
    eku, eru = O.sort_pairs(ku, ru)
    assert np.array_equal(oku, eku) and np.array_equal(oru, eru) and stu["natural_runs"] == 0


def test_sort_merge_plan_natural_runs_ties_and_chunk_edges():
    """Ascending runs over four key values (equal keys in every run: the merge
    must keep input order), with run starts on the detection pass's chunk
    starts (chunks of max_slot_pairs rows) and between them."""
    n = 1_000_000
    v = G.i32_uniform(n, 0, 4, 3, 7).astype(np.uint64)
    starts = sorted({0, 100_000, 200_000, 250_001, 300_000, 777_777, 900_000, 999_999})
    k = np.empty(n, np.uint64)
    for a, b in zip(starts, starts[1:] + [n]):
        k[a:b] = np.sort(v[a:b])
    r = np.arange(n, dtype=np.uint32)
    ok, orr, st = _merge_sort(k, r, max_slot_pairs=100_000)
    ek, er = O.sort_pairs(k, r)
    assert np.array_equal(ok, ek) and np.array_equal(orr, er)
    # a run start is a descent unless the run's first key reaches the previous run's last
    assert st["natural_runs"] == 1 and st["n_runs"] == 1 + int(np.count_nonzero(k[1:] < k[:-1]))
    assert st["n_runs"] >= len(starts) - 1


def test_sort_merge_plan_too_many_runs_sorts_chunks():
    n = 1_200_000
    k = np.empty(n, np.uint64)
    bounds = np.linspace(0, n, 301).astype(np.int64)  # 300 runs: more than the merge takes
    src = G.u64_uniform(n, 2, 13)
    for a, b in zip(bounds[:-1], bounds[1:]):
        k[a:b] = np.sort(src[a:b])
    r = np.arange(n, dtype=np.uint32)
    ok, orr, st = _merge_sort(k, r)
    ek, er = O.sort_pairs(k, r)
    assert np.array_equal(ok, ek) and np.array_equal(orr, er) and st["natural_runs"] == 0
