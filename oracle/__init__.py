"""Oracle — TEST INFRASTRUCTURE ONLY.

Plain CPU definitions of every result of the out-of-core query hot path
(Vortex, arXiv 2502.09541): the single-dimension and star join queries
(Section 7.1), filter with stream compaction (Section 6.3), the stable sort of
(key, row id) pairs (Section 6.1) and the exact cut of sorted runs that its
merge plan partitions by, the equi-join with count / payload checksum
/ pair fingerprint (Section 6.2), find_boundary (Section 6.2.1, Fig. 9), range
partitioning, sample and piecewise-linear CDF splitters, the monotone CDF MLP
(fp64 forward/backward and Adam), the per-chunk cardinality regressor (fp64
least squares) and the zero-copy threshold (Section 6.3, TH equation).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package.  It shares no code with paper_2502_09541_gb300/ and never
imports it; both read the host buffers written by datagen/.

Parity pins (tests/test_oracle_pins.py) tie each function to something other
than itself: brute force on tiny inputs, generator-side ground truth, closed
forms, invariants, the worked find_boundary example and finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

BETWEEN, EQ, NE, LT, LE, GT, GE = range(7)
AGG_COUNT, AGG_SUM, AGG_MUL, AGG_SUB = range(4)
MAX_DIMS, MAX_PREDS = 8, 8
I32MIN, I32MAX = -2**31, 2**31 - 1


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-fvisibility=hidden", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


# ---------------------------------------------------------------- C structs
P32 = ctypes.POINTER(ctypes.c_int32)


class OrPred(ctypes.Structure):
    _fields_ = [("col", ctypes.c_void_p), ("op", ctypes.c_int32), ("lo", ctypes.c_int32),
                ("hi", ctypes.c_int32)]


class OrDim(ctypes.Structure):
    _fields_ = [("key", ctypes.c_void_p), ("rows", ctypes.c_uint64), ("n_attr", ctypes.c_int32),
                ("attr", ctypes.c_void_p * 4), ("n_preds", ctypes.c_int32),
                ("pred_attr", ctypes.c_int32 * 4), ("pred_op", ctypes.c_int32 * 4),
                ("pred_lo", ctypes.c_int32 * 4), ("pred_hi", ctypes.c_int32 * 4),
                ("fact_fk", ctypes.c_void_p)]


class OrGkey(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("attr", ctypes.c_int32), ("card", ctypes.c_int32),
                ("fact_col", ctypes.c_void_p)]


class OrStarQuery(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("n_dims", ctypes.c_int32), ("dims", OrDim * MAX_DIMS),
                ("n_fact_preds", ctypes.c_int32), ("fact_preds", OrPred * MAX_PREDS),
                ("n_group_keys", ctypes.c_int32), ("group_keys", OrGkey * 4),
                ("agg_op", ctypes.c_int32), ("agg_a", ctypes.c_void_p), ("agg_b", ctypes.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            u64, i64, i32, u32, dbl, vp, ci = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_uint32, ctypes.c_double, ctypes.c_void_p,
                                              ctypes.c_int)
            sig = {
                "or_q1": ([vp, vp, vp, vp, u64, vp, vp, u64, i32, i32, i32, i32, vp, vp], ci),
                "or_star": ([ctypes.POINTER(OrStarQuery), vp, vp, ci], ci),
                "or_star_groups": ([ctypes.POINTER(OrStarQuery)], u64),
                "or_filter": ([u64, u64, ci, vp, vp, u64, vp], ci),
                "or_sort_pairs": ([vp, vp, u64, vp, vp], ci),
                "or_pair_fp": ([u64, u64], u64),
                "or_join": ([vp, vp, u64, vp, u64, u64, vp, vp, vp, ci], ci),
                "or_find_boundary": ([vp, u64, u32, vp], None),
                "or_pid": ([u64, vp, u32], u32),
                "or_range_partition": ([vp, vp, u64, vp, u32, vp, vp, vp], None),
                "or_sort_u64": ([vp, u64], None),
                "or_sample_splitters": ([vp, u64, u32, vp], None),
                "or_pl_knots": ([vp, u64, u32, vp], None),
                "or_pl_splitters": ([vp, u32, u32, vp], None),
                "or_mlp_forward": ([vp, ci, dbl], dbl),
                "or_mlp_loss_grad": ([vp, ci, vp, vp, u64, vp], dbl),
                "or_adam_step": ([vp, vp, vp, vp, ci, ci, dbl, dbl, dbl, dbl], None),
                "or_zero_copy_threshold": ([dbl, dbl, dbl, dbl], dbl),
                "or_isolate_splitters": ([vp, u32, vp, u64, u32, vp], u32),
                "or_exact_cut": ([vp, vp, u32, u64, vp], ci),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _c(a, dt):
    a = np.ascontiguousarray(a, dtype=dt)
    return a


# ---------------------------------------------------------------- queries
def q1(fact, dim, year=1993, disc_lo=1, disc_hi=3, qty_lt=25, rows=None):
    """O1: SUM(price*discount) over fact rows joined to the date dimension with
    year == year, disc_lo <= discount <= disc_hi, quantity < qty_lt.
    Returns (wrapping int64 sum, qualifying row count)."""
    n = len(fact["date_fk"]) if rows is None else rows
    s, c = ctypes.c_int64(), ctypes.c_uint64()
    st = lib().or_q1(_p(fact["date_fk"]), _p(fact["quantity"]), _p(fact["discount"]), _p(fact["price"]),
                     n, _p(dim["key"]), _p(dim["year"]), len(dim["key"]), year, disc_lo, disc_hi, qty_lt,
                     ctypes.byref(s), ctypes.byref(c))
    if st:
        raise RuntimeError(f"or_q1 status {st}")
    return s.value, c.value


def _pred_triplet(op, lo, hi):
    return op, lo, hi


def star_query_struct(tmpl, fact, dims, row_begin=0, row_end=None, keep=None):
    """Build the oracle's query struct from a datagen star template.
    `keep` collects the numpy objects that must outlive the struct."""
    from datagen import STAR_ATTR_CARD  # template vocabulary only
    keep = [] if keep is None else keep
    row_end = len(next(iter(fact.values()))) if row_end is None else row_end
    n = row_end - row_begin

    def fcol(name):
        a = fact[name][row_begin:row_end]
        keep.append(a)
        return a.ctypes.data

    q = OrStarQuery()
    q.n = n
    q.n_dims = len(tmpl["dims"])
    dim_index = {}
    for d, spec in enumerate(tmpl["dims"]):
        dd = dims[spec["dim"]]
        attrs = list(STAR_ATTR_CARD[spec["dim"]].keys())
        od = q.dims[d]
        od.key = dd["key"].ctypes.data
        od.rows = len(dd["key"])
        od.n_attr = len(attrs)
        for k, a in enumerate(attrs):
            od.attr[k] = dd[a].ctypes.data
        od.n_preds = len(spec["preds"])
        for k, (a, lo, hi) in enumerate(spec["preds"]):
            od.pred_attr[k] = attrs.index(a)
            od.pred_op[k] = BETWEEN
            od.pred_lo[k] = lo
            od.pred_hi[k] = hi
        od.fact_fk = fcol(spec["fk"])
        dim_index[spec["dim"]] = d
    q.n_fact_preds = len(tmpl["fact_preds"])
    for k, (c, lo, hi) in enumerate(tmpl["fact_preds"]):
        q.fact_preds[k].col = fcol(c)
        q.fact_preds[k].op = BETWEEN
        q.fact_preds[k].lo = lo
        q.fact_preds[k].hi = hi
    q.n_group_keys = len(tmpl["group"])
    for k, (dname, a) in enumerate(tmpl["group"]):
        attrs = list(STAR_ATTR_CARD[dname].keys())
        g = q.group_keys[k]
        g.dim = dim_index[dname]
        g.attr = attrs.index(a)
        g.card = STAR_ATTR_CARD[dname][a]
    op, a, b = tmpl["agg"]
    q.agg_op = {"sum": AGG_SUM, "mul": AGG_MUL, "sub": AGG_SUB, "count": AGG_COUNT}[op]
    q.agg_a = fcol(a) if a else None
    q.agg_b = fcol(b) if b else None
    return q, keep


def star(tmpl, fact, dims, row_begin=0, row_end=None, nthreads=1):
    """O2: dense (sums[G], counts[G]) of a star template over fact rows
    [row_begin, row_end)."""
    q, keep = star_query_struct(tmpl, fact, dims, row_begin, row_end)
    G = lib().or_star_groups(ctypes.byref(q))
    sums = np.zeros(G, np.int64)
    cnts = np.zeros(G, np.uint64)
    st = lib().or_star(ctypes.byref(q), _p(sums), _p(cnts), nthreads)
    if st:
        raise RuntimeError(f"or_star status {st}")
    del keep
    return sums, cnts


def star_raw(q, nthreads=1):
    G = lib().or_star_groups(ctypes.byref(q))
    sums = np.zeros(G, np.int64)
    cnts = np.zeros(G, np.uint64)
    st = lib().or_star(ctypes.byref(q), _p(sums), _p(cnts), nthreads)
    if st:
        raise RuntimeError(f"or_star status {st}")
    return sums, cnts


def filter_rows(preds, n, row0=0):
    """Ascending row ids (row0 + i) of rows satisfying every (col, op, lo, hi)."""
    arr = (OrPred * max(1, len(preds)))()
    keep = []
    for k, (col, op, lo, hi) in enumerate(preds):
        col = _c(col, np.int32)
        keep.append(col)
        arr[k].col, arr[k].op, arr[k].lo, arr[k].hi = col.ctypes.data, op, lo, hi
    cnt = ctypes.c_uint64()
    lib().or_filter(n, row0, len(preds), arr, None, 0, ctypes.byref(cnt))
    out = np.empty(cnt.value, np.uint64)
    lib().or_filter(n, row0, len(preds), arr, _p(out), cnt.value, ctypes.byref(cnt))
    return out


# ---------------------------------------------------------------- sort / join
def sort_pairs(keys, rowids):
    keys = _c(keys, np.uint64)
    rowids = _c(rowids, np.uint32)
    ok = np.empty_like(keys)
    orr = np.empty_like(rowids)
    st = lib().or_sort_pairs(_p(keys), _p(rowids), len(keys), _p(ok), _p(orr))
    if st:
        raise RuntimeError(f"or_sort_pairs status {st}")
    return ok, orr


def exact_cut(keys, run_off, k):
    """Per run, how many of the first k elements of the stable order (by key,
    then position) lie in it (Section 6.1 merge data mapping)."""
    keys = _c(keys, np.uint64)
    ro = _c(run_off, np.uint64)
    out = np.zeros(len(ro) - 1, np.uint64)
    st = lib().or_exact_cut(_p(keys), _p(ro), len(ro) - 1, int(k), _p(out))
    if st:
        raise RuntimeError(f"or_exact_cut status {st}")
    return out


def pair_fp(probe_row, payload):
    return int(lib().or_pair_fp(probe_row & (2**64 - 1), payload & (2**64 - 1)))


def join(bkeys, bpay, pkeys, probe_row0=0, nthreads=1):
    """O4: (count, wrapping payload sum, pair fingerprint) of the equi-join."""
    bkeys = _c(bkeys, np.int64)
    bpay = _c(bpay, np.int64)
    pkeys = _c(pkeys, np.int64)
    c, s, f = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    st = lib().or_join(_p(bkeys), _p(bpay), len(bkeys), _p(pkeys), len(pkeys), probe_row0,
                       ctypes.byref(c), ctypes.byref(s), ctypes.byref(f), nthreads)
    if st:
        raise RuntimeError(f"or_join status {st}")
    return c.value, s.value, f.value


def find_boundary(hashes, N):
    h = _c(hashes, np.uint32)
    b = np.empty(N + 1, np.uint64)
    lib().or_find_boundary(_p(h), len(h), N, _p(b))
    return b


def pid(key, splitters):
    s = _c(splitters, np.uint64)
    return int(lib().or_pid(key, _p(s), len(s) + 1))


def range_partition(keys, rowids, splitters):
    keys = _c(keys, np.uint64)
    rowids = _c(rowids, np.uint32)
    s = _c(splitters, np.uint64)
    P = len(s) + 1
    ok, orr = np.empty_like(keys), np.empty_like(rowids)
    b = np.empty(P + 1, np.uint64)
    lib().or_range_partition(_p(keys), _p(rowids), len(keys), _p(s), P, _p(ok), _p(orr), _p(b))
    return ok, orr, b


def sorted_u64(a):
    a = np.array(a, dtype=np.uint64, copy=True)
    lib().or_sort_u64(_p(a), len(a))
    return a


def sample_splitters(sorted_sample, P):
    s = _c(sorted_sample, np.uint64)
    out = np.empty(max(P - 1, 0), np.uint64)
    lib().or_sample_splitters(_p(s), len(s), P, _p(out))
    return out


def pl_knots(sorted_sample, S=1024):
    s = _c(sorted_sample, np.uint64)
    out = np.empty(S + 1, np.uint64)
    lib().or_pl_knots(_p(s), len(s), S, _p(out))
    return out


def pl_splitters(knots, P):
    k = _c(knots, np.uint64)
    out = np.empty(max(P - 1, 0), np.uint64)
    lib().or_pl_splitters(_p(k), len(k) - 1, P, _p(out))
    return out


def isolate_splitters(splitters, sorted_sample, P):
    """Heavy-key isolation: de-duplicate, then give every splitter value that
    holds at least half a partition's share of the sample its own [v, v+1)."""
    s = _c(splitters, np.uint64)
    smp = _c(sorted_sample, np.uint64)
    out = np.zeros(max(2 * len(s), 1), np.uint64)
    k = lib().or_isolate_splitters(_p(s), len(s), _p(smp), len(smp), P, _p(out))
    return out[:k].copy()


# ---------------------------------------------------------------- MLP CDF model
def mlp_forward(theta, H, x):
    th = _c(theta, np.float64)
    return float(lib().or_mlp_forward(_p(th), H, float(x)))


def mlp_loss_grad(theta, H, x, t):
    th = _c(theta, np.float64)
    x = _c(x, np.float64)
    t = _c(t, np.float64)
    g = np.empty(3 * H + 1, np.float64)
    L = lib().or_mlp_loss_grad(_p(th), H, _p(x), _p(t), len(x), _p(g))
    return L, g


def adam_step(theta, grad, m1, m2, t, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
    """In place on float64 arrays theta, m1, m2."""
    lib().or_adam_step(_p(theta), _p(_c(grad, np.float64)), _p(m1), _p(m2), len(theta), t, lr, b1, b2, eps)


# ---------------------------------------------------------------- regressor / TH
def lstsq_ridge(X, y, lam=0.0):
    """Per-chunk cardinality regressor fit: w = argmin |X w - y|^2 + lam |w|^2,
    solved in fp64 from the normal equations (X^T X + lam I) w = X^T y."""
    X = np.asarray(X, np.float64)
    y = np.asarray(y, np.float64)
    A = X.T @ X + lam * np.eye(X.shape[1])
    return np.linalg.solve(A, X.T @ y)


def zero_copy_threshold(elem_bytes, gather_bytes, bw_zero_copy, bw_copy):
    return float(lib().or_zero_copy_threshold(elem_bytes, gather_bytes, bw_zero_copy, bw_copy))
