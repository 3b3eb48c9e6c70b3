"""CPU tests of the shared input generators (no query arithmetic here)."""
import datetime
import math

import numpy as np

import datagen as G


def test_ranges_are_counter_based():
    a = G.i32_uniform(100_000, 1, 50, 0, G.SALT["quantity"])
    b = G.i32_uniform(40_000, 1, 50, 0, G.SALT["quantity"], row0=30_000)
    assert np.array_equal(a[30_000:70_000], b)
    assert a.min() == 1 and a.max() == 50
    # distinct salts and seeds give different streams
    c = G.i32_uniform(1000, 1, 50, 0, G.SALT["discount"])
    d = G.i32_uniform(1000, 1, 50, 1, G.SALT["quantity"])
    assert not np.array_equal(a[:1000], c) and not np.array_equal(a[:1000], d)


def test_uniform_inclusive_bounds_and_balance():
    a = G.i32_uniform(1_100_000, 0, 10, 0, G.SALT["discount"])
    counts = np.bincount(a, minlength=11)
    assert len(counts) == 11 and counts.min() > 0
    assert np.all(np.abs(counts / len(a) - 1 / 11) < 0.003)


def test_date_dimension_calendar():
    d = G.date_dim(0)
    assert sorted(d["key"].tolist()) == list(range(G.DATE_ROWS))
    assert not np.array_equal(d["key"], np.arange(G.DATE_ROWS))  # stored shuffled
    base = datetime.date(1992, 1, 1)
    for k, y, m in zip(d["key"].tolist(), d["year"].tolist(), d["month"].tolist()):
        day = base + datetime.timedelta(days=k)
        assert (day.year, day.month) == (y, m)
    assert (d["year"] == 1993).sum() == 365
    assert d["year"].max() == 1998


def test_star_dims_hierarchy():
    dims = G.star_dims(0)
    for name, rows, _ in G.STAR_DIMS:
        dd = dims[name]
        assert len(np.unique(dd["key"])) == rows
        for attr, card in G.STAR_ATTR_CARD[name].items():
            assert dd[attr].min() >= 0 and dd[attr].max() < card
    s = dims["supp"]
    assert np.array_equal(s["nation"] // 5, s["region"])
    assert np.array_equal(s["city"] // 10, s["nation"])


def test_zipf_frequencies_match_pmf():
    N, s, n = 1000, 1.1, 400_000
    k = G.u64_zipf(n, N, s, 0, 99, hashed=False)
    assert k.min() >= 1 and k.max() <= N
    H = sum(r ** -s for r in range(1, N + 1))
    counts = np.bincount(k.astype(np.int64), minlength=N + 1)
    for r in (1, 2, 3, 10, 100):
        p = r ** -s / H
        sd = math.sqrt(n * p * (1 - p))
        assert abs(counts[r] - n * p) < 5 * sd, (r, counts[r], n * p)


def test_zipf_heavy_hitter_share_at_2_pow_30():
    # top rank share of Zipf(1.1) over 2^30 ranks: 1 / H_{2^30,1.1}
    N, s = 1 << 30, 1.1
    from scipy.special import zeta  # Hurwitz zeta: H(N,s) = zeta(s,1) - zeta(s,N+1)
    H = float(zeta(s, 1) - zeta(s, N + 1))
    k = G.u64_zipf(200_000, N, s, 0, G.SALT["sort_key"], hashed=False)
    share = (k == 1).mean()
    assert abs(share - 1 / H) < 0.005, (share, 1 / H)


def test_presorted_runs_sorted_within_runs():
    total, runs = 64_000, 64
    k = G.u64_presorted_runs(total, total, runs, 0, 1)
    L = total // runs
    for r in range(runs):
        seg = k[r * L:(r + 1) * L]
        assert np.all(seg[1:] >= seg[:-1])
    # the start of a run is low again
    assert k[L] < k[L - 1]


def test_join_generator_truth_and_disjoint_misses():
    nb, npr = 5000, 20_000
    bk, bp = G.build_side(nb)
    assert len(np.unique(bk)) == nb
    for match, z in ((1.0, 0.0), (0.5, 0.0), (0.5, 1.0), (0.0, 0.0)):
        pk = G.probe_side(npr, nb, match, z)
        c, s = G.probe_truth(npr, nb, match, z)
        hit = np.isin(pk, bk)
        assert hit.sum() == c
        if match == 1.0:
            assert c == npr
        if match == 0.0:
            assert c == 0
        if match == 0.5:
            assert abs(c / npr - 0.5) < 0.02
        # payload sum of the referenced build rows, wrapping
        pos = {int(k): i for i, k in enumerate(bk.tolist())}
        tot = 0
        for k in pk[hit].tolist():
            tot = (tot + int(bp[pos[int(k)]])) & (2**64 - 1)
        assert tot == s
