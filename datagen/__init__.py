"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

Holds only data generation (no query arithmetic).  The C core (``vxgen.c``) is
compiled on first use into ``datagen/libvxgen.so`` with gcc; every value is a
pure function of (seed, column salt, row index), so any row range can be
generated independently and the oracle and the GPU library read identical
bytes.

Workload recipes (all integer):
  * ``q1_tables``   — star-schema fact rows joined to a date dimension
                      (fact: date_fk U[0,2556), quantity U[1,50], discount U[0,10],
                      price U[90000,10000000]; dimension: 2,556 days from
                      1992-01-01 stored in shuffled order with their calendar year).
  * ``star_tables`` — 8-column fact table with four dimensions of 2,556 /
                      200,000 / 2,000,000 / 30,000 rows and 2-3 hierarchical
                      attribute codes (5-250 distinct values) each.
  * ``sort_input``  — (uint64 key, uint32 row id) pairs: uniform, Zipf(1.1)
                      over 2^30 ranks hashed by mix64, or presorted runs.
  * ``join_inputs`` — unique build keys mix64(i) with payload, probe foreign keys
                      uniform or Zipf(1.0) at a match rate.
These stand in for the Star Schema Benchmark and the radix-join setup the paper
evaluates on (Section 7); no item of those benchmarks is reproduced.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libvxgen.so")
_lock = threading.Lock()
_lib = None

NTHREADS = max(1, os.cpu_count() or 1)

# column salts (one independent counter stream per column)
SALT = {
    "date_fk": 11, "quantity": 12, "discount": 13, "price": 14, "cost": 15,
    "fk_supp": 16, "fk_part": 17, "fk_cust": 18,
    "dim_perm": 21, "supp_region": 22, "supp_nation": 23, "supp_city": 24,
    "part_mfgr": 25, "part_cat": 26, "part_brand": 27,
    "cust_region": 28, "cust_nation": 29, "cust_city": 30,
    "sort_key": 41, "sample_pos": 42, "probe": 51,
}


def build(force: bool = False) -> str:
    """Compile vxgen.c into libvxgen.so (portable C11, no arch flags)."""
    src = os.path.join(_HERE, "vxgen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-fvisibility=hidden", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


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
                "vxg_mix64": ([u64], u64),
                "vxg_base": ([u64, u64], u64),
                "vxg_u64": ([u64, u64], u64),
                "vxg_fill_i32_uniform": ([vp, u64, u64, u64, u64, i32, i32, ci], None),
                "vxg_fill_u64_uniform": ([vp, u64, u64, u64, u64, ci], None),
                "vxg_fill_rowid_u32": ([vp, u64, u64, ci], None),
                "vxg_fill_u64_zipf": ([vp, u64, u64, u64, u64, u64, dbl, ci, ci], None),
                "vxg_zipf_rank": ([u64, u64, u64, u64, dbl], u64),
                "vxg_fill_u64_presorted_runs": ([vp, u64, u64, u64, u64, u64, u64, ci], None),
                "vxg_fill_build_keys": ([vp, u64, u64, ci], None),
                "vxg_fill_build_payload": ([vp, u64, u64, ci], None),
                "vxg_fill_probe_keys": ([vp, u64, u64, u64, i64, dbl, u64, u64, ci], None),
                "vxg_probe_truth": ([u64, u64, u64, i64, dbl, u64, u64, vp, vp], None),
                "vxg_permutation_i32": ([vp, u64, u64, u64], None),
                "vxg_date_of_key": ([i32, vp, vp], None),
                "vxg_fill_child_code": ([vp, vp, u64, i32, i32, u64, u64], None),
                "vxg_sample_positions": ([vp, u64, u64, u64, u64], None),
                "vxg_fill_i32_ramp": ([vp, u64, u64, u64, i32, ci], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def mix64(x: int) -> int:
    return int(lib().vxg_mix64(x & 0xFFFFFFFFFFFFFFFF))


# ---------------------------------------------------------------- columns
def i32_uniform(n, lo, hi, seed, salt, row0=0, out=None):
    out = np.empty(n, np.int32) if out is None else out
    lib().vxg_fill_i32_uniform(_ptr(out), n, row0, seed, salt, lo, hi, NTHREADS)
    return out


def u64_uniform(n, seed, salt, row0=0, out=None):
    out = np.empty(n, np.uint64) if out is None else out
    lib().vxg_fill_u64_uniform(_ptr(out), n, row0, seed, salt, NTHREADS)
    return out


def rowid_u32(n, row0=0, out=None):
    out = np.empty(n, np.uint32) if out is None else out
    lib().vxg_fill_rowid_u32(_ptr(out), n, row0, NTHREADS)
    return out


def u64_zipf(n, N, s, seed, salt, row0=0, hashed=True, out=None):
    out = np.empty(n, np.uint64) if out is None else out
    lib().vxg_fill_u64_zipf(_ptr(out), n, row0, seed, salt, N, s, 0 if hashed else 1, NTHREADS)
    return out


def zipf_rank(seed, salt, row, N, s):
    return int(lib().vxg_zipf_rank(seed, salt, row, N, s))


def u64_presorted_runs(n, total, n_runs, seed, salt, row0=0, out=None):
    out = np.empty(n, np.uint64) if out is None else out
    lib().vxg_fill_u64_presorted_runs(_ptr(out), n, row0, total, n_runs, seed, salt, NTHREADS)
    return out


def permutation_i32(n, seed, salt):
    out = np.empty(n, np.int32)
    lib().vxg_permutation_i32(_ptr(out), n, seed, salt)
    return out


def date_of_key(key: int):
    y, m = ctypes.c_int32(), ctypes.c_int32()
    lib().vxg_date_of_key(key, ctypes.byref(y), ctypes.byref(m))
    return y.value, m.value


def child_code(n, parent, fanout, card, seed, salt):
    out = np.empty(n, np.int32)
    lib().vxg_fill_child_code(_ptr(out), None if parent is None else _ptr(parent), n, fanout, card,
                              seed, salt)
    return out


def sample_positions(m, n, seed, salt=SALT["sample_pos"]):
    out = np.empty(m, np.uint64)
    lib().vxg_sample_positions(_ptr(out), m, n, seed, salt)
    return out


# ---------------------------------------------------------------- workloads
DATE_ROWS = 2556
Q1_YEAR, Q1_DISC_LO, Q1_DISC_HI, Q1_QTY_LT = 1993, 1, 3, 25


def date_dim(seed=0):
    """Date dimension: key = shuffled 0..2555, year/month of day 1992-01-01 + key."""
    key = permutation_i32(DATE_ROWS, seed, SALT["dim_perm"])
    year = np.empty(DATE_ROWS, np.int32)
    month = np.empty(DATE_ROWS, np.int32)
    for i, k in enumerate(key.tolist()):
        year[i], month[i] = date_of_key(k)
    return {"key": key, "year": year, "month": month}


def q1_fact(n, seed=0, row0=0, out=None):
    """The four fact columns of the single-dimension query."""
    out = out or {}
    cols = {}
    cols["date_fk"] = i32_uniform(n, 0, DATE_ROWS - 1, seed, SALT["date_fk"], row0, out.get("date_fk"))
    cols["quantity"] = i32_uniform(n, 1, 50, seed, SALT["quantity"], row0, out.get("quantity"))
    cols["discount"] = i32_uniform(n, 0, 10, seed, SALT["discount"], row0, out.get("discount"))
    cols["price"] = i32_uniform(n, 90_000, 10_000_000, seed, SALT["price"], row0, out.get("price"))
    return cols


def q1_tables(n, seed=0):
    return q1_fact(n, seed), date_dim(seed)


# Star schema dimensions: (name, rows, fact fk column)
STAR_DIMS = [("date", 2556, "date_fk"), ("supp", 200_000, "fk_supp"),
             ("part", 2_000_000, "fk_part"), ("cust", 30_000, "fk_cust")]
STAR_FACT_COLS = ["date_fk", "fk_supp", "fk_part", "fk_cust", "quantity", "discount", "price", "cost"]
# attribute cardinalities per dimension (codes are in [0, card))
STAR_ATTR_CARD = {
    "date": {"year": 7, "month": 12},
    "supp": {"region": 5, "nation": 25, "city": 250},
    "part": {"mfgr": 5, "category": 25, "brand": 250},
    "cust": {"region": 5, "nation": 25, "city": 250},
}


def star_dims(seed=0):
    """Four dimensions; every dimension has an int32 key (shuffled 0..rows-1)
    and hierarchical int32 attribute codes (region->nation->city style)."""
    dims = {}
    d = date_dim(seed)
    dims["date"] = {"key": d["key"], "year": d["year"] - 1992, "month": d["month"] - 1}
    for name, rows, _ in STAR_DIMS[1:]:
        key = permutation_i32(rows, seed, SALT["dim_perm"] + rows)
        a0n, a1n, a2n = list(STAR_ATTR_CARD[name].keys())
        p = {"supp": "supp", "part": "part", "cust": "cust"}[name]
        s0, s1, s2 = {"supp": ("supp_region", "supp_nation", "supp_city"),
                      "part": ("part_mfgr", "part_cat", "part_brand"),
                      "cust": ("cust_region", "cust_nation", "cust_city")}[p]
        c0 = child_code(rows, None, 0, 5, seed, SALT[s0])
        c1 = child_code(rows, c0, 5, 25, seed, SALT[s1])
        c2 = child_code(rows, c1, 10, 250, seed, SALT[s2])
        dims[name] = {"key": key, a0n: c0, a1n: c1, a2n: c2}
    return dims


def star_fact(n, seed=0, row0=0, out=None, clustered_date=False, total=None):
    """Eight fact columns (int32): four uniform foreign keys and four measures.
    clustered_date: date_fk ascends with the row (a table appended in date
    order) instead of being uniform; `total` is the table's full row count."""
    out = out or {}
    rng = {"date_fk": (0, 2555), "fk_supp": (0, 199_999), "fk_part": (0, 1_999_999),
           "fk_cust": (0, 29_999), "quantity": (1, 50), "discount": (0, 10),
           "price": (90_000, 10_000_000), "cost": (1_000, 100_000)}
    cols = {c: i32_uniform(n, lo, hi, seed, SALT[c], row0, out.get(c)) for c, (lo, hi) in rng.items()}
    if clustered_date:
        d = cols["date_fk"]
        lib().vxg_fill_i32_ramp(_ptr(d), n, row0, total or n, DATE_ROWS, NTHREADS)
    return cols


def star_templates():
    """Star-join query templates (plain dicts; the binding and the oracle wrapper
    each convert them).  Predicates are inclusive ranges [lo, hi] on int32.

    T1: one probe (date) + fact predicates, scalar SUM(price*discount).
    T2: three probes, group by (year, part category) = 175 groups, SUM(price-cost).
    T3: four probes, group by (year, cust nation, supp region) = 875 groups,
        SUM(price-cost).
    price and cost are payload columns (read only for qualifying rows).
    Selectivity variants sel in {'0.1', '1', '10'} percent (approximate).
    """
    I32MIN, I32MAX = -2**31, 2**31 - 1
    T = {}
    T["T1"] = {
        "dims": [{"dim": "date", "fk": "date_fk", "preds": [("year", 1, 1)]}],
        "fact_preds": [("discount", 1, 3), ("quantity", I32MIN, 24)],
        "group": [], "agg": ("mul", "price", "discount"),
    }
    # T2: part category <= cat_hi, supplier region <= reg_hi, quantity <= qty_hi
    for sel, (cat_hi, reg_hi, qty_hi) in {"10": (4, 2, 42), "1": (1, 1, 16), "0.1": (0, 0, 6)}.items():
        T[f"T2_{sel}"] = {
            "dims": [{"dim": "part", "fk": "fk_part", "preds": [("category", 0, cat_hi)]},
                     {"dim": "supp", "fk": "fk_supp", "preds": [("region", 0, reg_hi)]},
                     {"dim": "date", "fk": "date_fk", "preds": []}],
            "fact_preds": [("quantity", I32MIN, qty_hi)],
            "group": [("date", "year"), ("part", "category")],
            "agg": ("sub", "price", "cost"),
        }
    # T3: customer nation <= nat_hi, year code >= yr_lo, part mfgr <= 3, discount range
    for sel, (nat_hi, yr_lo, disc) in {"10": (11, 0, (0, 2)), "1": (3, 4, (2, 3)), "0.1": (0, 6, (2, 3))}.items():
        T[f"T3_{sel}"] = {
            "dims": [{"dim": "cust", "fk": "fk_cust", "preds": [("nation", 0, nat_hi)]},
                     {"dim": "supp", "fk": "fk_supp", "preds": []},
                     {"dim": "date", "fk": "date_fk", "preds": [("year", yr_lo, 6)]},
                     {"dim": "part", "fk": "fk_part", "preds": [("mfgr", 0, 3)]}],
            "fact_preds": [("discount", disc[0], disc[1])],
            "group": [("date", "year"), ("cust", "nation"), ("supp", "region")],
            "agg": ("sub", "price", "cost"),
        }
    return T


def sort_input(n, dist="uniform", seed=0, row0=0, total=None, keys=None, rowids=None):
    """(uint64 key, uint32 row id) pairs. dist: uniform | zipf | runs."""
    total = n if total is None else total
    if dist == "uniform":
        k = u64_uniform(n, seed, SALT["sort_key"], row0, keys)
    elif dist == "zipf":
        k = u64_zipf(n, 1 << 30, 1.1, seed, SALT["sort_key"], row0, True, keys)
    elif dist == "runs":
        k = u64_presorted_runs(n, total, 64, seed, SALT["sort_key"], row0, keys)
    else:
        raise ValueError(dist)
    r = rowid_u32(n, row0, rowids)
    return k, r


def build_side(n_build, row0=0, keys=None, payload=None):
    k = np.empty(n_build, np.int64) if keys is None else keys
    p = np.empty(n_build, np.int64) if payload is None else payload
    lib().vxg_fill_build_keys(_ptr(k), len(k), row0, NTHREADS)
    lib().vxg_fill_build_payload(_ptr(p), len(p), row0, NTHREADS)
    return k, p


def probe_side(n_probe, n_build, match=1.0, zipf_s=0.0, seed=0, row0=0, out=None):
    o = np.empty(n_probe, np.int64) if out is None else out
    lib().vxg_fill_probe_keys(_ptr(o), len(o), row0, n_build, int(round(match * 1e6)), zipf_s,
                              seed, SALT["probe"], NTHREADS)
    return o


def probe_truth(n_probe, n_build, match=1.0, zipf_s=0.0, seed=0, row0=0, nthreads=None):
    """(match count, wrapping payload sum) recorded while drawing the probes;
    row ranges are redrawn on nthreads threads (the C call releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    def part(lo, hi):
        c, s = ctypes.c_uint64(), ctypes.c_uint64()
        lib().vxg_probe_truth(hi - lo, row0 + lo, n_build, int(round(match * 1e6)), zipf_s, seed,
                              SALT["probe"], ctypes.byref(c), ctypes.byref(s))
        return c.value, s.value

    k = max(1, min(nthreads or NTHREADS, n_probe // (1 << 20) or 1))
    cuts = [n_probe * i // k for i in range(k + 1)]
    with ThreadPoolExecutor(k) as ex:
        parts = list(ex.map(part, cuts[:-1], cuts[1:]))
    return sum(c for c, _ in parts), sum(s for _, s in parts) % (1 << 64)


def join_inputs(n_build, n_probe, match=1.0, zipf_s=0.0, seed=0):
    bk, bp = build_side(n_build)
    pk = probe_side(n_probe, n_build, match, zipf_s, seed)
    return bk, bp, pk
