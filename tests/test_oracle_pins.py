"""Pins of the oracle against things other than itself (CPU only).

Each oracle function is tied to brute force on tiny inputs, to the generator's
own ground truth, to closed forms, to invariants or to numbers the paper
prints, chosen so that a dropped term, a wrong sign or index, or a transposed
operand fails at least one test.
"""
import datetime
import os

import numpy as np
import pytest

import datagen as G
import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
M64 = 2**64 - 1


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split(":", 1)
        out[k.strip()] = v.strip()
    return out


def _wrap(x):
    x &= M64
    return x - 2**64 if x >= 2**63 else x


# ------------------------------------------------------------------ Q1
def test_q1_against_calendar_brute_force():
    """Brute force that never reads the dimension table: the year of a foreign
    key comes from Python's own calendar (day 1992-01-01 + fk)."""
    n = 4000
    fact, dim = G.q1_tables(n, seed=3)
    base = datetime.date(1992, 1, 1)
    s = c = 0
    for fk, q, d, p in zip(*(fact[k].tolist() for k in ("date_fk", "quantity", "discount", "price"))):
        if (base + datetime.timedelta(days=fk)).year == 1993 and 1 <= d <= 3 and q < 25:
            s += p * d
            c += 1
    assert O.q1(fact, dim) == (_wrap(s), c)


def test_q1_selectivity_matches_closed_form():
    g = _golden("q1_expected_selectivity.txt")
    num = eval(g["numerator"], {})
    den = eval(g["denominator"], {})
    n = 2_000_000
    fact, dim = G.q1_tables(n)
    _, c = O.q1(fact, dim)
    p = num / den
    sd = (n * p * (1 - p)) ** 0.5
    assert abs(c - n * p) < 5 * sd


def test_q1_missing_foreign_keys_drop_rows():
    fact, dim = G.q1_tables(3000, seed=1)
    full = O.q1(fact, dim)
    # remove the 1993 rows from the dimension: no fact row can qualify
    keep = dim["year"] != 1993
    dim2 = {k: np.ascontiguousarray(v[keep]) for k, v in dim.items()}
    assert O.q1(fact, dim2) == (0, 0)
    # dimension with all keys shifted out of range: empty join
    dim3 = dict(dim, key=np.ascontiguousarray(dim["key"] + 10_000))
    assert O.q1(fact, dim3) == (0, 0)
    assert full[1] > 0


def test_q1_duplicate_dimension_key_is_an_error():
    fact, dim = G.q1_tables(100)
    dim2 = dict(dim, key=dim["key"].copy())
    dim2["key"][1] = dim2["key"][0]
    with pytest.raises(RuntimeError):
        O.q1(fact, dim2)


def test_q1_wrapping_sum():
    # a single qualifying row whose product exceeds nothing, then many rows
    # whose total exceeds 2^63: the oracle sum is the two's-complement wrap
    n = 4
    dim = {"key": np.array([7], np.int32), "year": np.array([1993], np.int32)}
    fact = {"date_fk": np.full(n, 7, np.int32), "quantity": np.full(n, 1, np.int32),
            "discount": np.full(n, 3, np.int32), "price": np.full(n, 2**31 - 1, np.int32)}
    s, c = O.q1(fact, dim)
    assert c == n and s == _wrap(n * 3 * (2**31 - 1))


# ------------------------------------------------------------------ star
def _star_brute(T, fact, dims, n):
    """Dictionary-based nested evaluation of a star template."""
    look = {}
    for spec in T["dims"]:
        dd = dims[spec["dim"]]
        look[spec["dim"]] = {int(k): i for i, k in enumerate(dd["key"].tolist())}
    cards = [G.STAR_ATTR_CARD[d][a] for d, a in T["group"]]
    Gn = int(np.prod(cards)) if cards else 1
    sums = [0] * Gn
    cnts = [0] * Gn
    for i in range(n):
        ok = all(lo <= int(fact[c][i]) <= hi for c, lo, hi in T["fact_preds"])
        rows = {}
        for spec in T["dims"]:
            if not ok:
                break
            r = look[spec["dim"]].get(int(fact[spec["fk"]][i]))
            if r is None:
                ok = False
                break
            dd = dims[spec["dim"]]
            ok = all(lo <= int(dd[a][r]) <= hi for a, lo, hi in spec["preds"])
            rows[spec["dim"]] = r
        if not ok:
            continue
        g = 0
        for (d, a), card in zip(T["group"], cards):
            g = g * card + int(dims[d][a][rows[d]])
        op, a, b = T["agg"]
        va, vb = int(fact[a][i]), int(fact[b][i]) if b else 0
        v = {"sum": va, "mul": va * vb, "sub": va - vb}[op]
        sums[g] += v
        cnts[g] += 1
    return np.array([_wrap(s) for s in sums], np.int64), np.array(cnts, np.uint64)


@pytest.mark.parametrize("name", list(G.star_templates().keys()))
def test_star_against_brute_force(name):
    T = G.star_templates()[name]
    n = 3000
    fact = G.star_fact(n, seed=5)
    dims = G.star_dims(0)
    s, c = O.star(T, fact, dims)
    bs, bc = _star_brute(T, fact, dims, n)
    assert np.array_equal(s, bs) and np.array_equal(c, bc)


def test_star_thread_count_invariant_and_group_totals():
    T = G.star_templates()["T3_10"]
    fact = G.star_fact(200_000, seed=2)
    dims = G.star_dims(0)
    s1, c1 = O.star(T, fact, dims, nthreads=1)
    s8, c8 = O.star(T, fact, dims, nthreads=7)
    assert np.array_equal(s1, s8) and np.array_equal(c1, c8)
    # invariant: dropping the group keys gives one group holding the totals
    T1 = dict(T, group=[])
    st, ct = O.star(T1, fact, dims)
    assert st[0] == _wrap(int(s1.astype(object).sum())) and ct[0] == c1.sum()


def test_star_single_dim_equals_q1():
    T = G.star_templates()["T1"]
    n = 100_000
    fact = G.q1_fact(n)
    dims = {"date": {"key": G.date_dim()["key"], "year": G.date_dim()["year"] - 1992,
                     "month": G.date_dim()["month"] - 1}}
    s, c = O.star(T, fact, dims)
    assert (int(s[0]), int(c[0])) == O.q1(fact, G.date_dim())


# ------------------------------------------------------------------ filter
def test_filter_brute_force_and_order():
    n = 5000
    f = G.star_fact(n, seed=9)
    preds = [(f["quantity"], O.LT, 10, 0), (f["discount"], O.BETWEEN, 2, 5),
             (f["price"], O.NE, 0, 0)]
    rows = O.filter_rows(preds, n, row0=1000)
    exp = [1000 + i for i in range(n)
           if f["quantity"][i] < 10 and 2 <= f["discount"][i] <= 5]
    assert rows.tolist() == exp
    assert np.all(np.diff(rows.astype(np.int64)) > 0)


@pytest.mark.parametrize("op,lo,hi,fn", [
    (O.EQ, 7, 0, lambda v: v == 7), (O.NE, 7, 0, lambda v: v != 7), (O.LT, 7, 0, lambda v: v < 7),
    (O.LE, 7, 0, lambda v: v <= 7), (O.GT, 7, 0, lambda v: v > 7), (O.GE, 7, 0, lambda v: v >= 7),
    (O.BETWEEN, 3, 9, lambda v: 3 <= v <= 9)])
def test_filter_each_operator(op, lo, hi, fn):
    v = G.i32_uniform(2000, 0, 12, 4, 77)
    rows = O.filter_rows([(v, op, lo, hi)], len(v))
    assert rows.tolist() == [i for i, x in enumerate(v.tolist()) if fn(x)]


def test_filter_empty_and_all_pass():
    v = G.i32_uniform(1000, 0, 12, 4, 77)
    assert len(O.filter_rows([(v, O.GT, 100, 0)], 1000)) == 0
    assert O.filter_rows([(v, O.GE, 0, 0)], 1000).tolist() == list(range(1000))
    assert len(O.filter_rows([(v, O.GE, 0, 0)], 0)) == 0


# ------------------------------------------------------------------ sort
def _fingerprint(keys, rows):
    k = keys.astype(np.uint64)
    r = rows.astype(np.uint64)
    with np.errstate(over="ignore"):
        h = (k * np.uint64(0x9E3779B97F4A7C15)) ^ (r * np.uint64(0xC2B2AE3D27D4EB4F))
    return len(k), int(h.astype(object).sum() % 2**64), int(np.bitwise_xor.reduce(h))


@pytest.mark.parametrize("dist", ["uniform", "zipf", "runs"])
def test_sort_matches_numpy_stable_argsort(dist):
    n = 50_000
    k, r = G.sort_input(n, dist)
    ok, orr = O.sort_pairs(k, r)
    perm = np.argsort(k, kind="stable")  # independent library sort (radix/timsort)
    assert np.array_equal(ok, k[perm]) and np.array_equal(orr, r[perm])
    assert np.all(ok[1:] >= ok[:-1])
    assert _fingerprint(k, r) == _fingerprint(ok, orr)
    # stability: equal keys keep increasing row ids (row id = input index here)
    eq = ok[1:] == ok[:-1]
    assert np.all(orr[1:][eq] > orr[:-1][eq])
    if dist == "zipf":
        assert eq.sum() > 0


def test_sort_special_cases():
    k = np.full(1000, 42, np.uint64)
    r = np.arange(1000, dtype=np.uint32)[::-1].copy()
    ok, orr = O.sort_pairs(k, r)
    assert np.array_equal(orr, r)  # all keys equal -> input order
    ok, orr = O.sort_pairs(np.zeros(0, np.uint64), np.zeros(0, np.uint32))
    assert len(ok) == 0
    k = np.array([2**64 - 1, 0, 2**63, 1], np.uint64)
    ok, _ = O.sort_pairs(k, np.arange(4, dtype=np.uint32))
    assert ok.tolist() == [0, 1, 2**63, 2**64 - 1]  # unsigned order


# ------------------------------------------------------------------ exact cut of sorted runs
def _runs(dist, n, n_runs, seed=0):
    """n keys as n_runs consecutive runs, each sorted (stable, so equal keys
    keep their input order), as the sort-merge plan's first pass leaves them."""
    k, _ = G.sort_input(n, dist, seed=seed)
    cuts = np.linspace(0, n, n_runs + 1).astype(np.uint64)
    for a, b in zip(cuts[:-1], cuts[1:]):
        k[a:b] = np.sort(k[a:b], kind="stable")
    return k, cuts


@pytest.mark.parametrize("dist", ["uniform", "zipf", "runs"])
def test_exact_cut_brute_force(dist):
    """Pure-Python brute force: order the positions by (key, position), take
    the first k, count them per run."""
    n, n_runs = 600, 7
    k, cuts = _runs(dist, n, n_runs, seed=2)
    if dist == "zipf":  # heavy ties across runs
        k[:] = np.sort(k % np.uint64(5))
        for a, b in zip(cuts[:-1], cuts[1:]):
            k[a:b] = np.sort(k[a:b])
    order = sorted(range(n), key=lambda i: (int(k[i]), i))
    run_of = np.searchsorted(cuts, np.arange(n), side="right") - 1
    for kk in (0, 1, 99, 300, 599, 600, 900):
        want = np.zeros(n_runs, np.uint64)
        for i in order[:kk]:
            want[run_of[i]] += 1
        assert np.array_equal(O.exact_cut(k, cuts, kk), want), kk


def test_exact_cut_invariants():
    """Sums to k; everything left of the cut orders before everything right
    of it; grows with k; numpy's stable argsort gives the same counts."""
    n, n_runs = 40_000, 13
    k, cuts = _runs("zipf", n, n_runs, seed=3)
    perm = np.argsort(k, kind="stable")
    run_of = np.searchsorted(cuts, np.arange(n), side="right") - 1
    prev = np.zeros(n_runs, np.uint64)
    for kk in (0, 1, 4_999, 20_000, 33_333, n - 1, n):
        c = O.exact_cut(k, cuts, kk)
        assert int(c.sum()) == kk
        assert np.all(c >= prev)
        prev = c
        assert np.array_equal(c, np.bincount(run_of[perm[:kk]], minlength=n_runs).astype(np.uint64))
        left = [(int(k[cuts[r] + j]), int(cuts[r] + j)) for r in range(n_runs) for j in range(int(c[r]))]
        right = [(int(k[cuts[r] + j]), int(cuts[r] + j)) for r in range(n_runs)
                 for j in range(int(c[r]), int(cuts[r + 1] - cuts[r]))]
        if left and right:
            assert max(left) < min(right)


def test_exact_cut_special_cases():
    # one run: the cut is k itself; all keys equal: runs are taken whole, in order
    k = np.sort(G.u64_uniform(1000, 1, 9))
    assert O.exact_cut(k, np.array([0, 1000], np.uint64), 321).tolist() == [321]
    k = np.full(1000, 7, np.uint64)
    cuts = np.array([0, 100, 350, 350, 1000], np.uint64)
    assert O.exact_cut(k, cuts, 400).tolist() == [100, 250, 0, 50]
    assert O.exact_cut(k, cuts, 5000).tolist() == [100, 250, 0, 650]


# ------------------------------------------------------------------ join
@pytest.mark.parametrize("match,z", [(1.0, 0.0), (0.5, 0.0), (1.0, 1.0), (0.5, 1.0), (0.0, 0.0)])
def test_join_against_generator_truth(match, z):
    nb, npr = 20_000, 100_000
    bk, bp = G.build_side(nb)
    pk = G.probe_side(npr, nb, match, z)
    c, s, f = O.join(bk, bp, pk)
    tc, ts = G.probe_truth(npr, nb, match, z)
    assert (c, s) == (tc, ts)
    # cardinality = sum over keys of build count * probe count
    ub, cb = np.unique(bk, return_counts=True)
    up, cp = np.unique(pk, return_counts=True)
    common, ib, ip = np.intersect1d(ub, up, return_indices=True)
    assert c == int((cb[ib] * cp[ip]).sum())


def test_join_fingerprint_brute_force_and_threads():
    nb, npr = 300, 2000
    bk, bp = G.build_side(nb)
    pk = G.probe_side(npr, nb, 0.5, 0.0, seed=4)
    pos = {int(k): i for i, k in enumerate(bk.tolist())}
    fp = 0
    for j, k in enumerate(pk.tolist()):
        if int(k) in pos:
            pay = int(bp[pos[int(k)]]) & M64
            rot = ((pay << 17) | (pay >> 47)) & M64
            fp = (fp + O.pair_fp(1000 + j, pay)) & M64
            # the fingerprint is the SplitMix64 finalizer of row ^ rotl(payload,17)
            z = (1000 + j) ^ rot
            z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
            assert O.pair_fp(1000 + j, pay) == z ^ (z >> 31)
    assert O.join(bk, bp, pk, probe_row0=1000)[2] == fp
    assert O.join(bk, bp, pk, 1000, nthreads=1) == O.join(bk, bp, pk, 1000, nthreads=5)


def test_join_duplicate_build_key_is_an_error():
    bk, bp = G.build_side(10)
    bk[3] = bk[4]
    with pytest.raises(RuntimeError):
        O.join(bk, bp, bk)


# ------------------------------------------------------------------ find_boundary / partition
def test_find_boundary_worked_example():
    g = _golden("find_boundary_example.txt")
    keys = [int(x) for x in g["keys"].split()]
    hashes = [k & 0b11 for k in keys]
    assert hashes == [int(x) for x in g["hashes"].split()]
    b = O.find_boundary(np.array(hashes, np.uint32), 4)
    assert b.tolist() == [int(x) for x in g["boundary"].split()]


def test_find_boundary_equals_searchsorted():
    h = np.sort(G.i32_uniform(10_000, 0, 999, 2, 3)).astype(np.uint32)
    h = h[(h < 300) | (h > 310)]  # force a run of empty groups
    N = 1024
    b = O.find_boundary(h, N)
    assert np.array_equal(b, np.searchsorted(h, np.arange(N + 1), side="left"))
    assert O.find_boundary(np.zeros(0, np.uint32), 4).tolist() == [0, 0, 0, 0, 0]


def test_range_partition_stable_and_bounded():
    n, P = 30_000, 13
    k, r = G.sort_input(n, "zipf")
    spl = np.sort(G.u64_uniform(P - 1, 1, 5))
    ok, orr, b = O.range_partition(k, r, spl)
    pid = np.searchsorted(spl, k, side="right")  # number of splitters <= key
    perm = np.argsort(pid, kind="stable")
    assert np.array_equal(ok, k[perm]) and np.array_equal(orr, r[perm])
    assert np.array_equal(b, np.concatenate([[0], np.cumsum(np.bincount(pid, minlength=P))]))
    for p in range(P):
        seg = ok[b[p]:b[p + 1]]
        if len(seg):
            if p > 0:
                assert seg.min() >= spl[p - 1]
            if p < P - 1:
                assert seg.max() < spl[p]
    assert O.pid(int(spl[3]), spl) == 4 and O.pid(int(spl[3]) - 1, spl) == 3


# ------------------------------------------------------------------ splitters
def test_sample_and_pl_splitters_closed_forms():
    m = 100_001
    s = O.sorted_u64(G.u64_uniform(m, 0, 8))
    assert np.array_equal(s, np.sort(G.u64_uniform(m, 0, 8)))
    P = 32
    ss = O.sample_splitters(s, P)
    assert ss.tolist() == [int(s[p * m // P]) for p in range(1, P)]
    kn = O.pl_knots(s, 1024)
    assert kn[0] == s[0] and kn[-1] == s[-1]
    assert kn.tolist() == [int(s[j * (m - 1) // 1024]) for j in range(1025)]
    # P divides S: the inverse of the PL model lands exactly on knots
    pl = O.pl_splitters(kn, P)
    assert pl.tolist() == [int(kn[p * 1024 // P]) for p in range(1, P)]
    # P = 3 does not divide 1024: exact rational interpolation between knots
    pl3 = O.pl_splitters(kn, 3)
    for p, v in zip((1, 2), pl3.tolist()):
        j, rem = divmod(p * 1024, 3)
        assert v == int(kn[j]) + (int(kn[j + 1]) - int(kn[j])) * rem // 3
    # uniform keys: splitters near p/P of the key space
    for p, v in enumerate(pl.tolist(), start=1):
        assert abs(v / 2**64 - p / P) < 0.01


# ------------------------------------------------------------------ MLP
def _theta(H, seed=0):
    rng = np.random.default_rng(seed)
    return rng.normal(size=3 * H + 1)


def test_mlp_forward_closed_form_one_unit():
    # H = 1: y = gamma + softplus(alpha) * sigmoid(softplus(omega) * x + beta)
    om, be, al, ga = 0.3, -0.2, 1.1, 0.05
    x = 0.7
    sp = lambda v: np.log1p(np.exp(v))
    sg = lambda v: 1 / (1 + np.exp(-v))
    exp = ga + sp(al) * sg(sp(om) * x + be)
    assert abs(O.mlp_forward(np.array([om, be, al, ga]), 1, x) - exp) < 1e-14


def test_mlp_gradient_central_differences():
    H = 32
    th = _theta(H, 1)
    x = np.linspace(0, 1, 257)
    t = x ** 2
    L, g = O.mlp_loss_grad(th, H, x, t)
    eps = 1e-6
    for k in range(3 * H + 1):
        tp, tm = th.copy(), th.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (O.mlp_loss_grad(tp, H, x, t)[0] - O.mlp_loss_grad(tm, H, x, t)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 + 1e-4 * abs(fd), (k, fd, g[k])


def test_mlp_monotone_for_any_parameters():
    H = 32
    for seed in range(5):
        th = _theta(H, seed) * 3
        ys = [O.mlp_forward(th, H, x) for x in np.linspace(-0.5, 1.5, 401)]
        assert np.all(np.diff(ys) >= -1e-12)


def test_adam_first_step_closed_form():
    th = np.array([0.5, -1.0, 2.0])
    g = np.array([0.2, -3.0, 0.0])
    m1, m2 = np.zeros(3), np.zeros(3)
    O.adam_step(th, g, m1, m2, 1, lr=0.1, eps=1e-8)
    # bias-corrected first step moves each parameter by lr * g / (|g| + eps)
    exp = np.array([0.5, -1.0, 2.0]) - 0.1 * g / (np.abs(g) + 1e-8)
    assert np.allclose(th, exp, rtol=0, atol=1e-12)


# ------------------------------------------------------------------ regressor / TH
def test_regressor_exact_recovery_and_lstsq():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(500, 6))
    w = np.array([1.5, -2.0, 0.25, 0.0, 3.0, -0.5])
    assert np.allclose(O.lstsq_ridge(X, X @ w), w, atol=1e-10)
    y = X @ w + rng.normal(size=500)
    assert np.allclose(O.lstsq_ridge(X, y), np.linalg.lstsq(X, y, rcond=None)[0], atol=1e-10)


def test_threshold_reduces_to_paper_value():
    g = _golden("threshold_mi100.txt")
    E, C, N = float(g["elem_bytes"]), float(g["line_bytes"]), float(g["n_exchange"])
    # one link of zero-copy bandwidth B against copies spread over N equal links
    th = O.zero_copy_threshold(E, C, 1.0, N)
    assert th == float(g["threshold"]) == 1 / 64


def test_isolate_splitters_separates_heavy_keys():
    smp = np.array([1, 2, 9, 9, 9, 9, 11, 12, 12, 20], np.uint64)  # m = 10
    # P = 4: a value is heavy if it occurs >= 10 / 8 times -> 9 (4x) and 12 (2x)
    s = O.isolate_splitters(np.array([9, 9, 12], np.uint64), smp, 4)
    assert s.tolist() == [9, 10, 11, 12, 13]
    s = O.isolate_splitters(np.array([5, 5, 2**64 - 1, 2**64 - 1], np.uint64), smp, 5)
    assert s.tolist() == [5, 6, 2**64 - 1]
    # a key holding >= 1/P of the sample covers a quantile, so it is a
    # splitter and ends in a partition of its own, also when it is the
    # smallest key or sits on a single quantile
    for k in (np.array([3] * 60 + list(range(100, 140)), np.uint64),
              np.array(list(range(0, 33)) + [50] * 35 + list(range(60, 92)), np.uint64),
              np.array(list(range(0, 20)) + [50] * 36 + list(range(60, 104)), np.uint64)):
        sk = O.sorted_u64(k)
        spl = O.isolate_splitters(O.sample_splitters(sk, 3), sk, 3)
        pid = np.searchsorted(spl, k, side="right")
        heavy = int(np.bincount(k.astype(np.int64)).argmax())
        parts = set(pid[k == heavy].tolist())
        assert len(parts) == 1 and set(k[pid == parts.pop()].tolist()) == {heavy}
