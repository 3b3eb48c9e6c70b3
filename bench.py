"""Benchmark of the out-of-core star-join path on one GB300.

Workload (default, "star"): 600,000,000-row fact table of 8 int32 columns
(19.2 GB) held in pinned host memory, four dimensions of 2,556 / 200,000 /
2,000,000 / 30,000 rows, device budget 4 GiB.  One step runs the six star
templates with 3-4 chained probes at ~0.1 / 1 / 10 % combined selectivity
(group-by over 175 or 875 groups, SUM(price - cost) with both payload columns
late-materialized when the estimate is below TH).

Reported (one JSON line): host GB/s consumed (referenced column bytes x rows /
step time) with dimension tables resident, against the pinned host->device
peak measured in the same run; the dominant kernel's HBM roofline; an
end-to-end figure through the public call with dimension tables rebuilt from
host memory every step; the oracle timed on the host cores on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--rows R] [--budget-gb G]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TEMPLATES = ["T2_0.1", "T2_1", "T2_10", "T3_0.1", "T3_1", "T3_10"]
METRIC = "Host-data GB/s vs measured H2D peak (learned vs plain); p50/p99 query latency"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rows", type=int, default=600_000_000)
    ap.add_argument("--budget-gb", type=float, default=4.0)
    ap.add_argument("--cpu-sample-rows", type=int, default=0, help="oracle sample rows (0 = auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip serving, sort and join measurements")
    ap.add_argument("--serve-queries", type=int, default=400)
    ap.add_argument("--sort-pairs", type=int, default=1_000_000_000)
    ap.add_argument("--join-build", type=int, default=250_000_000)
    ap.add_argument("--join-probe", type=int, default=2_000_000_000)
    ap.add_argument("--workload", default="star", choices=["star", "sort", "join", "serve", "ops"],
                    help="star: the full benchmark line; sort / join / serve: that part alone")
    ap.add_argument("--serve-plain-queries", type=int, default=100)
    ap.add_argument("--sweep-queries", type=int, default=60, help="mixed serving queries per arrival rate (0: no sweep)")
    ap.add_argument("--sweep-sort-pairs", type=int, default=100_000_000)
    ap.add_argument("--sweep-join-build", type=int, default=50_000_000)
    ap.add_argument("--sweep-join-probe", type=int, default=600_000_000)
    ap.add_argument("--serve-chunk-rows", type=int, default=1 << 21, help="rows per shared-scan chunk")
    ap.add_argument("--serve-max-active", type=int, default=32, help="queries attached to the scan at once")
    ap.add_argument("--serve-slots", type=int, default=0, help="staging slots of the shared scan (0: library default)")
    ap.add_argument("--kernel-rows", type=int, default=0, choices=[0, 2, 8, 16],
                    help="plain form's fused-kernel shape (vx_config.kernel_rows; 2 = bulk-copy pipeline)")
    ap.add_argument("--blocks-per-sm", type=int, default=4, help="plain form's vx_config.blocks_per_sm")
    ap.add_argument("--clustered-rows", type=int, default=300_000_000,
                    help="date-clustered fact table of the per-chunk materialization comparison (0: skip)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    return rank, world, local


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                mhz.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


# fused chunk kernel shapes by vx_config.kernel_rows
KERNEL_SHAPES = {0: "one tile per block (4 rows per thread)", 2: "bulk-copy pipeline (4 rows per thread)",
                 8: "scalar, 8 rows per thread", 16: "scalar, 16 rows per thread"}
STAR_KERNEL_END = {"vx_star.cu": b"// ---- end of the fused chunk kernel's device code",
                   "vx_star.cuh": b"// ---- end of what the fused chunk kernel's device code reads",
                   "vx_probe.cuh": None}  # the row-logic helpers: the whole file


def kernel_source_digest():
    """sha256 of the fused star kernel's device code: vx_star.cu and
    vx_star.cuh, each up to its end marker, and vx_probe.cuh (ties a stored
    ncu figure to that code)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2502_09541_gb300", "csrc")
    for f, end in STAR_KERNEL_END.items():
        with open(os.path.join(csrc, f), "rb") as fh:
            text = fh.read()
        cut = text.find(end) if end else -1
        h.update(text if cut < 0 else text[:cut])
    return h.hexdigest()


def traffic_ratio():
    """DRAM bytes per algorithmic byte of the fused chunk kernel, from the
    committed ncu summary; None if absent or taken on other kernel sources."""
    p = os.path.join(ROOT, "profiles", "star_chunk_kernel_traffic.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line and not line.startswith(("#", " ")):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_sources_sha256") != kernel_source_digest():
        return None
    try:
        return float(vals["dram_per_algorithmic_byte"])
    except (KeyError, ValueError):
        return None


def make_data(rows, pinned=False, row0=0):
    """Fact rows [row0, row0 + rows) (optionally in page-locked host memory
    allocated by PyTorch, the 'pinned host memory' the workload holds its
    table in) and the four dimensions."""
    import datagen as G
    out = None
    if pinned:
        import torch
        out = {c: torch.empty(rows, dtype=torch.int32, pin_memory=True).numpy() for c in G.STAR_FACT_COLS}
    fact = G.star_fact(rows, row0=row0, out=out)
    dims = G.star_dims(0)
    return fact, dims


def cpu_baseline(fact, dims, sample_rows, nthreads=None):
    """The oracle as it stands, on the host cores (nthreads, default all),
    over the first sample_rows fact rows of every template of one step."""
    import datagen as G
    import oracle as O
    nthreads = nthreads or os.cpu_count() or 1
    logical = 0
    t0 = time.perf_counter()
    for name in TEMPLATES:
        T = G.star_templates()[name]
        O.star(T, fact, dims, 0, sample_rows, nthreads=nthreads)
        cols = {c for c, _, _ in T["fact_preds"]} | {d["fk"] for d in T["dims"]} | \
            {c for c in T["agg"][1:] if c}
        logical += 4 * len(cols) * sample_rows
    dt = time.perf_counter() - t0
    return logical / dt / 1e9, nthreads, dt


def single_thread_baseline(fact, dims, sample_rows):
    """The same oracle on one host thread, over a tenth of the sample (at
    most 2M rows) so that it stays within a few seconds."""
    n1 = max(1, min(sample_rows // 10, 2_000_000))
    v1, _, dt1 = cpu_baseline(fact, dims, n1, nthreads=1)
    return {"value": round(v1, 3), "unit": "GB/s", "cores": 1,
            "sample": f"first {n1} fact rows x 6 templates ({dt1:.1f} s)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import datagen as G  # noqa: F401
    sample = args.cpu_sample_rows or 20_000_000
    fact, dims = make_data(sample)
    for _ in range(args.warmup):
        pass  # the oracle has no warm state
    vals, dts = [], []
    for _ in range(args.steps):
        v, cores, dt = cpu_baseline(fact, dims, sample)
        vals.append(v)
        dts.append(dt)
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * statistics.median(dts), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"star join, {TEMPLATES} over the first {sample} rows of the 600M-row fact table",
                   "rows": sample},
        "cpu_baseline": {"value": round(v, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {sample} fact rows, 6 templates",
                         "single_thread": single_thread_baseline(fact, dims, sample)},
        "e2e": {"value": round(v, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_serving(vx, G, ctx, fid, did, args):
    """Continuous batching: Poisson arrivals of star queries (templates mixed,
    sizes log-uniform over [1M rows, whole table], random offsets); mean
    inter-arrival = half the mean single-query link time at the measured peak.
    The plain form serves the first --serve-plain-queries of the same arrivals
    one at a time, first come first served, through vx_run_plan."""
    np_ = __import__("numpy")
    rng = np_.random.default_rng(1)
    names = TEMPLATES
    n = args.rows
    qs = []
    for _ in range(args.serve_queries):
        size = int(math.exp(rng.uniform(math.log(1_000_000), math.log(n))))
        rb = int(rng.integers(0, n - size + 1))
        qs.append((names[int(rng.integers(0, len(names)))], rb, rb + size))
    mean_rows = sum(q[2] - q[1] for q in qs) / len(qs)
    gap_s = 0.5 * mean_rows * 20 / 210e9
    arrivals = np_.cumsum(rng.exponential(gap_s, len(qs))) - gap_s
    tmpls = G.star_templates()
    plans = [vx.make_plan(tmpls[name], fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO, rb, re) for name, rb, re in qs]
    logical_of = [(q[2] - q[1]) * 4 * (len(tmpls[q[0]]["dims"]) + len(tmpls[q[0]]["fact_preds"]) + 2) for q in qs]

    vx.vx_serve_start(ctx, chunk_rows=args.serve_chunk_rows, max_active=args.serve_max_active,
                      n_slots=args.serve_slots)
    t0 = time.perf_counter()
    tickets = []
    for plan, ta in zip(plans, arrivals):
        now = time.perf_counter() - t0
        if ta > now:
            time.sleep(ta - now)
        tickets.append(vx.vx_submit(ctx, plan))
    for t in tickets:
        st = vx.vx_wait(ctx, t)[0]
        assert st == vx.VX_OK
    wall = time.perf_counter() - t0
    s = vx.vx_serve_stats_get(ctx)
    vx.vx_serve_stop(ctx)
    out = {"queries": len(qs), "p50_ms": round(s["p50_ms"], 3), "p99_ms": round(s["p99_ms"], 3),
           "mean_ms": round(s["mean_ms"], 3), "max_ms": round(s["max_ms"], 3),
           "qps": round(len(qs) / wall, 2), "host_gbs": round(sum(logical_of) / wall / 1e9, 3),
           "scan_h2d_gbs": round(s["bytes_h2d"] / wall / 1e9, 3), "active_peak": int(s["active_peak"]),
           "kernel_busy": round(s["ms_kernel"] / (wall * 1e3), 3), "admit_busy": round(s["ms_admit"] / (wall * 1e3), 3),
           "cycle_host_busy": round(s["ms_cycle"] / (wall * 1e3), 3), "slot_wait_busy": round(s["ms_wait"] / (wall * 1e3), 3),
           "cycles": int(s["cycles"]),
           "kernel_grows_s": round(s["work_rows"] / (s["ms_kernel"] * 1e6), 2) if s["ms_kernel"] else None,
           "mean_interarrival_ms": round(gap_s * 1e3, 3), "form": "shared circular scan"}

    k = min(args.serve_plain_queries, len(qs))
    if k:
        lat = []
        t0 = time.perf_counter()
        for plan, ta in zip(plans[:k], arrivals[:k]):
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            assert vx.vx_run_plan(ctx, plan)[0] == vx.VX_OK
            lat.append(1e3 * (time.perf_counter() - t0 - ta))
        wall = time.perf_counter() - t0
        out["plain"] = {"queries": k, "p50_ms": round(float(np_.percentile(lat, 50)), 3),
                        "p99_ms": round(float(np_.percentile(lat, 99)), 3), "mean_ms": round(float(np_.mean(lat)), 3),
                        "qps": round(k / wall, 2), "host_gbs": round(sum(logical_of[:k]) / wall / 1e9, 3),
                        "form": "one query at a time, first come first served (same arrivals)"}
    return out


def run_serving_sweep(vx, G, ctx, fid, did, args):
    """Mixed serving at a sweep of arrival rates: 70 % star queries, 15 %
    join-shaped (probe-row ranges of a shared join table) and 15 % sort-shaped
    (row ranges of a shared pair table), sizes log-uniform; the saturation
    rate is the throughput of a burst of all queries at once, then Poisson
    arrivals at fractions of it.  Sort queries run one at a time in the
    engine's operator thread, so they share one output and one intermediate
    buffer here (their results are checked in the tests, not here)."""
    import numpy as np
    n_star = args.rows
    ns, nb, npr = args.sweep_sort_pairs, args.sweep_join_build, args.sweep_join_probe
    t0 = time.perf_counter()
    sk, sr = G.sort_input(ns, "zipf", seed=8, keys=pinned_array(ns, np.uint64), rowids=pinned_array(ns, np.uint32))
    bk, bp = G.build_side(nb, keys=pinned_array(nb, np.int64), payload=pinned_array(nb, np.int64))
    pk = G.probe_side(npr, nb, 1.0, 1.0, out=pinned_array(npr, np.int64))
    ok, orr = pinned_array(ns, np.uint64), pinned_array(ns, np.uint32)
    scratch = pinned_array(12 * (ns + ns // 16) + (1 << 24), np.uint8)
    gen = time.perf_counter() - t0
    kc = vx.vx_register_host_column(ctx, "sweep.sk", sk)
    rc = vx.vx_register_host_column(ctx, "sweep.sr", sr)
    a = vx.vx_register_host_column(ctx, "sweep.bk", bk)
    b = vx.vx_register_host_column(ctx, "sweep.bp", bp)
    p = vx.vx_register_host_column(ctx, "sweep.pk", pk)
    tmpls = G.star_templates()
    rng = np.random.default_rng(11)

    def draw(k):
        qs = []
        for _ in range(k):
            u = rng.uniform()
            kind = "star" if u < 0.7 else "join" if u < 0.85 else "sort"
            n = {"star": n_star, "join": npr, "sort": ns}[kind]
            size = int(math.exp(rng.uniform(math.log(1_000_000), math.log(n))))
            rb = int(rng.integers(0, n - size + 1))
            qs.append((kind, TEMPLATES[int(rng.integers(0, len(TEMPLATES)))], rb, rb + size))
        return qs

    def submit(q):
        kind, name, rb, re = q
        if kind == "star":
            return ("star", vx.vx_submit(ctx, vx.make_plan(tmpls[name], fid, did, G.STAR_ATTR_CARD,
                                                          vx.VX_LATE_AUTO, rb, re)))
        req = vx.vx_op_request()
        req.row_begin, req.row_end = rb, re
        if kind == "sort":
            req.kind, req.key_col, req.val_col = vx.VX_QUERY_SORT, kc, rc
            req.out_keys, req.out_rowids = ok.ctypes.data, orr.ctypes.data
            req.sort.host_scratch = scratch.ctypes.data
            req.sort.host_scratch_bytes = scratch.nbytes
        else:
            req.kind, req.key_col, req.val_col, req.probe_col = vx.VX_QUERY_JOIN, a, b, p
        return ("op", vx.vx_submit_op(ctx, req))

    def run(qs, arrivals):
        vx.vx_serve_start(ctx, chunk_rows=args.serve_chunk_rows, max_active=args.serve_max_active,
                          n_slots=args.serve_slots)
        t_start = time.perf_counter()
        tickets = []
        for q, ta in zip(qs, arrivals):
            now = time.perf_counter() - t_start
            if ta > now:
                time.sleep(ta - now)
            tickets.append(submit(q))
        for kind, t in tickets:
            if kind == "star":
                assert vx.vx_wait(ctx, t)[0] == vx.VX_OK
            else:
                vx.vx_wait_op(ctx, t)
        wall = time.perf_counter() - t_start
        st = vx.vx_serve_stats_get(ctx)
        vx.vx_serve_stop(ctx)
        return wall, st

    k = args.sweep_queries
    wall, st = run(draw(k), [0.0] * k)  # burst: the saturation throughput
    sat = k / wall
    out = {"mix": "70% star, 15% join, 15% sort", "queries_per_point": k, "generate_s": round(gen, 1),
           "saturation_qps": round(sat, 2), "sort_pairs": ns, "join_build": nb, "join_probe": npr,
           "rate_sweep": []}
    for f in (0.25, 0.5, 0.75, 0.9, 1.0, 1.2):
        qs = draw(k)
        arrivals = np.cumsum(rng.exponential(1.0 / (f * sat), k)) - 1.0 / (f * sat)
        wall, st = run(qs, arrivals)
        out["rate_sweep"].append({
            "load": f, "rate_qps": round(f * sat, 2), "qps": round(k / wall, 2), "p50_ms": round(st["p50_ms"], 2),
            "p99_ms": round(st["p99_ms"], 2),
            "p50_ms_kind": {n: round(st["p50_kind_ms"][i], 2) for i, n in enumerate(("star", "sort", "join"))},
            "p99_ms_kind": {n: round(st["p99_kind_ms"][i], 2) for i, n in enumerate(("star", "sort", "join"))},
            "completed_kind": dict(zip(("star", "sort", "join"), st["completed_kind"])), "failed": st["failed"]})
    for col in (kc, rc, a, b, p):
        vx.vx_unregister_host_column(ctx, col)
    return out


# a star query whose qualifying years sit in the last chunks of a table
# appended in date order (fact rows' date_fk ascends with the row)
CLUSTER_T = {
    "dims": [{"dim": "cust", "fk": "fk_cust", "preds": [("nation", 0, 11)]},
             {"dim": "date", "fk": "date_fk", "preds": [("year", 5, 6)]}],
    "fact_preds": [("discount", 0, 2)],
    "group": [("date", "year"), ("cust", "nation")],
    "agg": ("sub", "price", "cost"),
}


def run_clustered(vx, G, ctx, did, args):
    """Late/early materialization decided per chunk by the regressor (learned)
    against one decision per plan (plain) on a date-clustered fact table: the
    survivors crowd into the last chunks, where staging the payload columns
    beats reading them by zero-copy.  Same executor configuration for both;
    results compared equal."""
    import numpy as np
    n = args.clustered_rows
    clu = G.star_fact(n, seed=6, clustered_date=True,
                      out={c: pinned_array(n, np.int32) for c in G.STAR_FACT_COLS})
    fc = {k: vx.vx_register_host_column(ctx, "clustered." + k, clu[k]) for k in clu}
    plans = {"plain": vx.make_plan(CLUSTER_T, fc, did, G.STAR_ATTR_CARD, vx.VX_LATE_AUTO),
             "learned": vx.make_plan(CLUSTER_T, fc, did, G.STAR_ATTR_CARD, vx.VX_LATE_PER_CHUNK)}
    res, out = {}, {"rows": n, "template": "cust.nation<=11, date.year in [5,6], discount in [0,2]"}
    for _ in range(2):  # warm-up: dimension tables resident, host pages touched
        for pl in plans.values():
            vx.vx_run_plan(ctx, pl)
    times = {k: [] for k in plans}
    for _ in range(3):
        for k, pl in plans.items():
            st, gid, sm, cnt, stats = vx.vx_run_plan(ctx, pl)
            assert st == vx.VX_OK
            times[k].append(stats)
            res[k] = (gid, sm, cnt)
    for k, ss in times.items():
        ms = statistics.median(x["ms_total"] for x in ss)
        x = ss[-1]
        out[k] = {"gbs": round(x["bytes_logical"] / (ms * 1e6), 1), "ms": round(ms, 2),
                  "link_bytes": int(x["bytes_h2d"] + x["bytes_zero_copy"]), "late_chunks": int(x["late_chunks"]),
                  "chunks": int(x["chunks"]), "late_mask": int(x["late_mask"])}
    out["equal"] = all(np.array_equal(a, b) for a, b in zip(res["plain"], res["learned"]))
    return out


def run_ops_extra(vx, G, args, ctx=None, fid=None, did=None):
    """Operator-at-a-time execution with host intermediates against the fused
    plan on the same context: a sparse template (T2_1, about 1 % of rows
    survive the filter and probes) and a dense one (T3_10); each timed as its
    second call, results compared equal."""
    own = ctx is None
    if own:
        fact, dims = make_data(args.rows, pinned=True)
        ctx = vx.vx_open(int(args.budget_gb * (1 << 30)))
        fid = {c: vx.vx_register_host_column(ctx, c, fact[c]) for c in fact}
        did = {d: {a: vx.vx_register_host_column(ctx, f"{d}.{a}", arr) for a, arr in dims[d].items()} for d in dims}
    import datagen as G_
    import numpy as np
    tmpls = G_.star_templates()
    out = {"rows": args.rows}
    try:
        for name in ("T2_1", "T3_10"):
            plan = vx.make_plan(tmpls[name], fid, did, G_.STAR_ATTR_CARD)
            res = {}
            for form, fn in (("fused", vx.vx_run_plan), ("operators", vx.vx_run_plan_operators)):
                fn(ctx, plan)
                st, gid, sm, cnt, stats = fn(ctx, plan)
                assert st == vx.VX_OK
                res[form] = (gid, sm, cnt, stats)
            f, o = res["fused"][3], res["operators"][3]
            out[name] = {"fused_ms": round(f["ms_total"], 2), "operators_ms": round(o["ms_total"], 2),
                         "operators_h2d_bytes": int(o["bytes_h2d"]), "operators_d2h_bytes": int(o["bytes_d2h"]),
                         "operators_zero_copy_bytes": int(o["bytes_zero_copy"]), "fused_h2d_bytes": int(f["bytes_h2d"]),
                         "equal": all(np.array_equal(a, b) for a, b in zip(res["fused"][:3], res["operators"][:3]))}
    finally:
        if own:
            vx.vx_close(ctx)
    return out


def pinned_array(n, dtype):
    """A numpy view of page-locked host memory allocated by PyTorch (the
    copy engines read it at full link rate; registered pageable memory is
    slower on this link)."""
    import numpy as np
    import torch
    dt = np.dtype(dtype)
    return torch.empty(n * dt.itemsize, dtype=torch.uint8, pin_memory=True).numpy().view(dt)


def run_sort_extra(vx, G, args):
    """Out-of-core sort of (uint64 key, uint32 row id) pairs, 16 GiB budget:
    partition-then-sort with sample splitters (plain) vs learned PL and MLP
    models, and the merge plan (sorted runs, exact cuts), on Zipf(1.1) keys
    and on 64 presorted runs."""
    import numpy as np
    n = args.sort_pairs
    t0 = time.perf_counter()
    k, r = G.sort_input(n, "zipf", keys=pinned_array(n, np.uint64), rowids=pinned_array(n, np.uint32))
    gen = time.perf_counter() - t0
    ok = pinned_array(n, np.uint64)
    orr = pinned_array(n, np.uint32)
    scratch = pinned_array(12 * (n + n // 16), np.uint8)  # room for a region per partition
    ctx = vx.vx_open(16 << 30)
    out = {"pairs": n, "dist": "zipf(1.1)", "budget_gib": 16, "generate_s": round(gen, 1)}
    try:
        kc = vx.vx_register_host_column(ctx, "k", k)
        rc = vx.vx_register_host_column(ctx, "r", r)
        # map the (already page-locked) output and scratch buffers once, outside the timed sorts
        for buf in (ok, orr, scratch):
            vx.vx_register_host_column(ctx, "pin", buf.view(np.uint32) if buf.dtype != np.uint32 else buf)
        o = vx.vx_sort_opts()
        o.host_scratch = scratch.ctypes.data
        o.host_scratch_bytes = scratch.nbytes
        vx.vx_sort(ctx, kc, rc, ok, orr, o)  # warm-up: first pass over freshly pinned host pages

        def form(part, plan, runs_mode=0):
            o = vx.vx_sort_opts()
            o.partitioner = part
            o.plan = plan
            o.runs_mode = runs_mode
            o.host_scratch = scratch.ctypes.data
            o.host_scratch_bytes = scratch.nbytes
            o.sample_size = 1 << 20
            # two runs per form, the faster reported (single runs of a form
            # have come out up to 35 % slow on some machines, whichever form ran)
            runs = [vx.vx_sort(ctx, kc, rc, ok, orr, o) for _ in range(2)]
            st = min(runs, key=lambda r: r["ms_total"])
            d = {"gpairs_s": round(n / st["ms_total"] / 1e6, 3), "ms": round(st["ms_total"], 1),
                 "ms_runs": [round(r["ms_total"], 1) for r in runs],
                 "partitions": st["n_partitions"], "imbalance": round(st["imbalance"], 3),
                 "passthrough": st["passthrough_partitions"], "overflow_retries": st["overflow_retries"],
                 "ms_partition": round(st["ms_partition"], 1), "ms_sort": round(st["ms_sort"], 1),
                 "ms_train": round(st["ms_train"], 1),
                 "partition_regions": bool(st["contiguous_layout"]),
                 "out_of_region_pairs": st["out_of_region_pairs"],
                 "link_gbs": round((st["bytes_h2d"] + st["bytes_d2h"]) / st["ms_total"] / 1e6, 1)}
            if plan == vx.VX_SORT_MERGE:  # pass 1 sorts runs, pass 2 merges: no sample, exact cuts
                d.update({"runs": st["n_runs"], "natural_runs": bool(st["natural_runs"]),
                          "ms_cut": round(st["ms_sample"], 2), "ms_merge_kernel": round(st["ms_merge_kernel"], 1)})
                if st["ms_merge_kernel"] > 0:
                    hbm_peak, _ = measured_peaks()
                    ach = 24 * st["merge_pass_pairs"] / (st["ms_merge_kernel"] * 1e6)
                    d["merge_roofline"] = {"kernel": "merge_round_kernel", "bound": "hbm", "unit": "GB/s",
                                           "achieved": round(ach, 1), "peak": hbm_peak,
                                           "frac": round(ach / hbm_peak, 4)}
            return d, st

        for name, part, plan in (("plain_sample", vx.VX_PART_SAMPLE, vx.VX_SORT_PARTITION),
                                 ("learned_pl", vx.VX_PART_LEARNED_PL, vx.VX_SORT_PARTITION),
                                 ("learned_mlp", vx.VX_PART_LEARNED_MLP, vx.VX_SORT_PARTITION),
                                 ("merge_exact", vx.VX_PART_SAMPLE, vx.VX_SORT_MERGE)):
            out[name], last = form(part, plan)
            if plan == vx.VX_SORT_PARTITION:
                st = last
        # the plain form again, staged by a 32-block copy kernel instead of
        # the copy engine (stores stay on the copy engine)
        cfg = vx.vx_get_config(ctx)
        cfg.h2d_copy_blocks = 32
        vx.vx_set_config(ctx, cfg)
        out["plain_sample_copy_kernel"] = form(vx.VX_PART_SAMPLE, vx.VX_SORT_PARTITION)[0]
        cfg.h2d_copy_blocks = 0
        vx.vx_set_config(ctx, cfg)
        out["sorted"] = bool(np.all(ok[1:] >= ok[:-1]))
        # per-partition radix sorts against HBM: 24 algorithmic bytes per pair
        # and executed pass (the one-sweep scatter reads and writes the 12-byte
        # pair; the single 8-byte key read of the digit histograms is left
        # out), from the last form's device time
        if st["ms_sort_kernel"] > 0:
            hbm_peak, peak_kind = measured_peaks()
            ach = 24 * st["radix_pass_pairs"] / (st["ms_sort_kernel"] * 1e6)
            out["radix_roofline"] = {"kernel": "rx_downsweep (one-sweep LSD pass)", "bound": "hbm", "unit": "GB/s",
                                     "achieved": round(ach, 1), "peak": hbm_peak, "frac": round(ach / hbm_peak, 4),
                                     "peak_kind": peak_kind, "pass_pairs": int(st["radix_pass_pairs"]),
                                     "ms_sort_kernel": round(st["ms_sort_kernel"], 1)}
        # uniform 64-bit keys (every digit pass runs): both plans
        G.sort_input(n, "uniform", keys=k, rowids=r)
        vx.vx_sort(ctx, kc, rc, ok, orr, vx.vx_sort_opts())  # first pass over the rewritten pages
        out["uniform"] = {"plain_sample": form(vx.VX_PART_SAMPLE, vx.VX_SORT_PARTITION)[0],
                          "merge_exact": form(vx.VX_PART_SAMPLE, vx.VX_SORT_MERGE)[0]}
        out["uniform"]["sorted"] = bool(np.all(ok[1:] >= ok[:-1]))
        # 64 presorted runs (the third key distribution): partition-then-sort
        # against the merge plan on the same input
        G.sort_input(n, "runs", keys=k, rowids=r)
        vx.vx_sort(ctx, kc, rc, ok, orr, vx.vx_sort_opts())  # first pass over the rewritten pages
        out["presorted_runs"] = {"plain_sample": form(vx.VX_PART_SAMPLE, vx.VX_SORT_PARTITION)[0],
                                 "learned_pl": form(vx.VX_PART_LEARNED_PL, vx.VX_SORT_PARTITION)[0],
                                 "merge_exact": form(vx.VX_PART_SAMPLE, vx.VX_SORT_MERGE)[0],
                                 # the same plan made to sort its chunks into runs first
                                 "merge_sorted_chunks": form(vx.VX_PART_SAMPLE, vx.VX_SORT_MERGE, 1)[0]}
        out["presorted_runs"]["sorted"] = bool(np.all(ok[1:] >= ok[:-1]))
    finally:
        vx.vx_close(ctx)
    return out


def run_join_extra(vx, G, args):
    """Partitioned hash join: unique build keys with payload, uniform probe
    keys at match rate 1.0, 24 GiB budget; plain (exact count pass) vs learned
    (model-implied table sizes) at P = 2, and the planner's own P."""
    nb, npr = args.join_build, args.join_probe
    t0 = time.perf_counter()
    import numpy as np
    bk, bp = G.build_side(nb, keys=pinned_array(nb, np.int64), payload=pinned_array(nb, np.int64))
    pk = G.probe_side(npr, nb, 1.0, 0.0, out=pinned_array(npr, np.int64))
    gen = time.perf_counter() - t0
    ctx = vx.vx_open(24 << 30)
    out = {"build_rows": nb, "probe_rows": npr, "budget_gib": 24, "generate_s": round(gen, 1)}
    try:
        a = vx.vx_register_host_column(ctx, "bk", bk)
        b = vx.vx_register_host_column(ctx, "bp", bp)
        p = vx.vx_register_host_column(ctx, "pk", pk)
        vx.vx_join(ctx, a, b, p, vx.vx_join_opts())  # warm-up: first pass over freshly pinned host pages
        for name, P, cp, part in (("planner", 0, 0, vx.VX_PART_LEARNED_PL), ("plain_p2", 2, 1, vx.VX_PART_SAMPLE),
                                  ("learned_p2", 2, 0, vx.VX_PART_LEARNED_PL)):
            o = vx.vx_join_opts()
            o.n_partitions = P
            o.count_pass = cp
            o.partitioner = part
            r = vx.vx_join(ctx, a, b, p, o)
            out[name] = {"gtuples_s": round((nb + npr) / r["ms_total"] / 1e6, 3), "ms": round(r["ms_total"], 1),
                         "partitions": r["n_partitions"], "count": r["count"],
                         "link_gbs": round(r["bytes_h2d"] / r["ms_total"] / 1e6, 1),
                         "overflow_retries": r["overflow_retries"], "ms_build": round(r["ms_build"], 1),
                         "ms_probe": round(r["ms_probe"], 1), "ms_kernel": round(r["ms_kernel"], 1)}
        out["count_ok"] = out["planner"]["count"] == npr
        # probe kernel against HBM's random-access ceiling, measured in this run
        # on a table of the planner's size (one random 32-byte bucket read per
        # probe is the algorithmic minimum; longer walks read more)
        budget_slots = int(0.98 * ((24 << 30) - (256 << 20)) / 16)
        table_bytes = 16 * min(budget_slots, 2 * nb)
        ceiling = vx.vx_probe_hbm_random(ctx, table_bytes, 64 << 20)
        pr = vx.vx_join(ctx, a, b, p, vx.vx_join_opts())
        ach = npr / (pr["ms_probe_kernel"] * 1e6)
        out["probe_roofline"] = {"kernel": "join_probe_kernel", "bound": "hbm_random", "unit": "G reads/s",
                                 "achieved": round(ach, 2), "peak": round(ceiling, 2), "frac": round(ach / ceiling, 4),
                                 "table_gb": round(table_bytes / 1e9, 2), "ms_probe_kernel": round(pr["ms_probe_kernel"], 1),
                                 "peak_kind": "vx_probe_hbm_random in this run"}
        # the other probe distributions of the workload (planner form): match
        # rate 50 % and Zipf(1.0) foreign keys, drawn into the same pinned buffer;
        # count and wrapping payload sum against the truth recorded while drawing
        for match, zs in ((0.5, 0.0), (1.0, 1.0), (0.5, 1.0)):
            G.probe_side(npr, nb, match, zs, out=pk)
            c_true, s_true = G.probe_truth(npr, nb, match, zs)
            # the first call after the host rewrote the probe column runs its
            # build-side copies slower (host-side effect; kernels unchanged), so
            # the figure is the second call and the first is kept beside it
            first = vx.vx_join(ctx, a, b, p, vx.vx_join_opts())
            t = time.perf_counter()
            r = vx.vx_join(ctx, a, b, p, vx.vx_join_opts())
            call_ms = 1e3 * (time.perf_counter() - t)
            out[f"match{match:g}_zipf{zs:g}"] = {
                "gtuples_s": round((nb + npr) / r["ms_total"] / 1e6, 3), "ms": round(r["ms_total"], 1),
                "first_call_ms": round(first["ms_total"], 1), "call_ms": round(call_ms, 1),
                "ms_build": round(r["ms_build"], 1), "ms_probe": round(r["ms_probe"], 1),
                "ms_kernel": round(r["ms_kernel"], 1),
                "ms_sample": round(r["ms_sample"], 1), "overflow_retries": r["overflow_retries"],
                "link_gbs": round(r["bytes_h2d"] / r["ms_total"] / 1e6, 1),
                "count": r["count"], "exact": r["count"] == c_true and r["payload_sum"] == s_true}
            if (match, zs) == (1.0, 1.0):
                # the paper's radix-partitioned join (2^24 groups joined in shared
                # memory) on the same skewed probes; its host intermediates are
                # allocated and page-locked inside the call (ms_total), the two
                # passes alone are ms
                o = vx.vx_join_opts()
                o.algorithm = vx.VX_JOIN_RADIX
                rr = vx.vx_join(ctx, a, b, p, o)
                ms = rr["ms_partition"] + rr["ms_probe"]
                out["radix_match1_zipf1"] = {
                    "gtuples_s": round((nb + npr) / ms / 1e6, 3), "ms": round(ms, 1), "ms_total": round(rr["ms_total"], 1),
                    "ms_partition": round(rr["ms_partition"], 1), "ms_join": round(rr["ms_probe"], 1),
                    "ms_join_kernel": round(rr["ms_probe_kernel"], 1), "ranges": rr["ranges"],
                    "link_gbs": round((rr["bytes_h2d"] + rr["bytes_d2h"]) / ms / 1e6, 1),
                    "exact": rr["count"] == c_true and rr["payload_sum"] == s_true}
    finally:
        vx.vx_close(ctx)
    return out


def run_ours(args):
    import torch

    import datagen as G
    import paper_2502_09541_gb300 as vx

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    vx.load()
    from paper_2502_09541_gb300.dist import shard_rows
    t_gen = time.perf_counter()
    row0, _ = shard_rows(rank, world, args.rows)  # weak scaling: a disjoint shard of equal size per rank
    fact, dims = make_data(args.rows, pinned=True, row0=row0)
    t_gen = time.perf_counter() - t_gen

    budget = int(args.budget_gb * (1 << 30))
    arena = torch.empty(budget, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    ctx = vx.vx_open_ex(arena.data_ptr(), budget, stream.cuda_stream)
    fid = {c: vx.vx_register_host_column(ctx, c, fact[c]) for c in fact}
    did = {d: {a: vx.vx_register_host_column(ctx, f"{d}.{a}", arr) for a, arr in dims[d].items()} for d in dims}
    tmpls = G.star_templates()
    plans = [vx.make_plan(tmpls[n], fid, did, G.STAR_ATTR_CARD) for n in TEMPLATES]

    # link peak measured in this run (pinned copies, 64 MiB chunks)
    h2d_peak, d2h_peak, bid_peak = vx.vx_probe_link(ctx, min(2 << 30, budget // 4), 64 << 20)

    def step(collect, plan_list=None):
        for p in plan_list or plans:
            t = time.perf_counter()
            st, gid, s, c, stats = vx.vx_run_plan(ctx, p)
            stats["host_ms"] = 1e3 * (time.perf_counter() - t)  # the call as the caller sees it
            assert st == vx.VX_OK
            collect.append(stats)

    def timed(n_steps, plan_list=None):
        """n_steps steps between CUDA events on the library's compute stream."""
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        out = []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n_steps):
            step(out, plan_list)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ms], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        return ms / n_steps, out

    # ---- plain form: executor with host-issued copies, 64 MiB chunks, one
    # late/early decision per plan; its warm-up steps log per-chunk statistics
    cfg = vx.vx_get_config(ctx)
    cfg.log_chunk_stats = 1
    cfg.kernel_rows = args.kernel_rows
    cfg.blocks_per_sm = args.blocks_per_sm
    vx.vx_set_config(ctx, cfg)
    for _ in range(max(args.warmup, 3)):
        step([])
    cfg.log_chunk_stats = 0
    vx.vx_set_config(ctx, cfg)
    with ClockSampler(local) as clk:
        ms_step, stats_all = timed(args.steps)
    clocks = clk.summary()
    logical = sum(s["bytes_logical"] for s in stats_all) / args.steps
    link = sum(s["bytes_h2d"] + s["bytes_zero_copy"] for s in stats_all) / args.steps
    plain_gbs = logical * world / (ms_step * 1e6)
    link_gbs = link / (ms_step * 1e6)
    launches = int(sum(s["kernel_launches"] for s in stats_all))
    rows_step = sum(s["rows"] for s in stats_all) / args.steps
    per_q_ms = {}
    for i, n in enumerate(TEMPLATES):
        per_q_ms[n] = round(statistics.median(s["ms_total"] for s in stats_all[i::len(TEMPLATES)]), 3)

    # copy / compute overlap of one run of every template (per-chunk CUDA
    # events on the copy and compute streams), outside the timed steps
    cfg.log_timeline = 1
    vx.vx_set_config(ctx, cfg)
    overlap = {}
    for i, n in enumerate(TEMPLATES):
        st_, _, _, _, qs = vx.vx_run_plan(ctx, plans[i])
        overlap[n] = timeline_summary(vx.vx_last_timeline(ctx), qs["bytes_h2d"])
    cfg.log_timeline = 0
    vx.vx_set_config(ctx, cfg)

    # dominant kernel: the fused chunk kernel; algorithmic HBM bytes = staged
    # column bytes it reads (rows x staged columns x 4), over its own CUDA-event
    # time (immediate schedule: events around each launch; captured graphs:
    # event nodes around each launch), one launch per chunk
    hbm_peak, peak_kind = measured_peaks()
    tr = traffic_ratio()

    def fused_roofline(stats_list):
        staged_bytes = sum(s["bytes_h2d"] for s in stats_list)
        k_ms = sum(s["ms_kernel"] for s in stats_list)
        nl = int(sum(s["chunks"] for s in stats_list))
        a = staged_bytes / (k_ms * 1e6) if k_ms > 0 else None
        return {"bound": "hbm", "kernel": "star_chunk_kernel", "achieved": round(a, 1) if a else None,
                "peak": hbm_peak, "unit": "GB/s", "frac": round(a / hbm_peak, 4) if a else None,
                "peak_kind": peak_kind,
                "traffic": round(tr * staged_bytes / max(1, nl)) if tr else None,
                "algorithmic_bytes_per_launch": round(staged_bytes / max(1, nl)),
                "avg_launch_us": round(1000 * k_ms / max(1, nl), 2), "launches": nl}

    roofline_plain = fused_roofline(stats_all)

    # the late-materialization gather: link-bound zero-copy reads of the
    # survivors' payload columns from mapped host memory (64-byte granules)
    g_ms = sum(s.get("ms_gather", 0.0) for s in stats_all)
    zc_bytes = sum(s["bytes_zero_copy"] for s in stats_all)
    zc_vals = sum(s["survivors"] * bin(s["late_mask"]).count("1") for s in stats_all)
    gather = None
    if g_ms > 0:
        gather = {"kernel": "star_gather_kernel", "bound": "link", "unit": "GB/s",
                  "achieved": round(zc_bytes / (g_ms * 1e6), 1), "peak": round(h2d_peak, 1),
                  "frac": round(zc_bytes / (g_ms * 1e6) / h2d_peak, 4), "peak_kind": "H2D copy, measured in this run",
                  "granule_bytes": 64, "values_read": int(zc_vals),
                  "algorithmic_gbs": round(4 * zc_vals / (g_ms * 1e6), 2),
                  "survivors_per_launch": round(sum(s["survivors"] for s in stats_all if s["late_mask"]) /
                                                max(1, sum(s["chunks"] for s in stats_all if s["late_mask"]))),
                  "avg_launch_us": round(1000 * g_ms / max(1, sum(s["chunks"] for s in stats_all if s["late_mask"])), 2)}
        # its ceiling: the same number of sparse reads per launch over a window
        # of one chunk's rows of one column, alone on an idle link
        late = [s for s in stats_all if s["late_mask"]]
        n_launch = max(1, sum(s["chunks"] for s in late))
        reads = max(1, round(zc_vals / n_launch))
        window = 4 * max(1, round(sum(s["rows"] for s in late) / n_launch))
        us_first, us_warm, _ = vx.vx_probe_zero_copy_gather(ctx, window, reads)
        gather["ceiling"] = {"probe": "vx_probe_zero_copy_gather", "reads_per_launch": reads, "window_bytes": window,
                             "us_first": round(us_first, 2), "us_warm": round(us_warm, 2),
                             "g_reads_per_s": round(reads / us_warm / 1e3, 3),
                             "granule_gbs": round(64 * reads / us_warm / 1e3, 1)}
        gather["of_ceiling"] = round(us_warm / gather["avg_launch_us"], 4) if gather["avg_launch_us"] else None

    # ---- learned / batched form: regressor trained on the plain form's log,
    # per-chunk late/early decisions, autotuned chunking, captured graphs
    w, n_log = vx.vx_regressor_train(ctx, 1e-6)
    tuned = vx.vx_autotune(ctx, plans[TEMPLATES.index("T3_1")], min(args.rows, 100_000_000))
    cfg = vx.vx_get_config(ctx)
    cfg.use_graphs = 1
    # the batched form stages with a 32-block copy kernel (launched at the
    # highest priority): on hosts where the copy engine's rate drops (it does
    # after a long run of other GPU work on the same machine) the copy kernel
    # holds the link's rate; the plain form stages by copy engine, and the
    # line reports the better form
    cfg.h2d_copy_blocks = 32
    tuned.h2d_copy_blocks = 32
    vx.vx_set_config(ctx, cfg)
    lplans = [vx.make_plan(tmpls[n], fid, did, G.STAR_ATTR_CARD, vx.VX_LATE_PER_CHUNK) for n in TEMPLATES]
    step([], lplans)  # captures the graphs
    with ClockSampler(local) as clk2:
        ms_learned, stats_l = timed(args.steps, lplans)
    learned_gbs = sum(s["bytes_logical"] for s in stats_l) / args.steps * world / (ms_learned * 1e6)
    roofline_learned = fused_roofline(stats_l)
    link_l = sum(s["bytes_h2d"] + s["bytes_zero_copy"] for s in stats_l) / args.steps / (ms_learned * 1e6)
    # the copy kernel that stages the batched form: by device time it is the
    # largest kernel of that form (it runs as long as the link is busy), bound
    # by the host link.  Its launches timed with CUDA events on the
    # host-to-device stream (the per-chunk timeline of one run of every
    # template, the same configuration without graph capture)
    copy_roofline = None
    if tuned.h2d_copy_blocks:
        cfg.use_graphs = 0
        cfg.log_timeline = 1
        vx.vx_set_config(ctx, cfg)
        cb, cms, cn = 0, 0.0, 0
        for p in lplans:
            _, _, _, _, qs = vx.vx_run_plan(ctx, p)
            tl = vx.vx_last_timeline(ctx)
            if len(tl):
                cb += qs["bytes_h2d"]
                cms += float((tl[:, 3] - tl[:, 2]).sum())
                cn += len(tl)
        cfg.log_timeline = 0
        cfg.use_graphs = 1
        vx.vx_set_config(ctx, cfg)
        if cms > 0:
            ach = cb / (cms * 1e6)
            copy_roofline = {"kernel": "host_copy_kernel (%d blocks)" % tuned.h2d_copy_blocks, "bound": "link",
                             "unit": "GB/s", "achieved": round(ach, 1), "peak": round(h2d_peak, 1),
                             "frac": round(ach / h2d_peak, 4), "peak_kind": "H2D copy, measured in this run",
                             "bytes_per_launch": round(cb / max(1, cn)),
                             "avg_launch_us": round(1000 * cms / max(1, cn), 1), "launches": cn}
    forms = {
        "plain": {"value": round(plain_gbs, 3), "ms_per_step": round(ms_step, 3), "link_gbs": round(link_gbs, 1),
                  "chunk_bytes": 64 << 20, "sched": "immediate", "late": "per plan",
                  "kernel_shape": {"kernel": KERNEL_SHAPES[args.kernel_rows], "blocks_per_sm": args.blocks_per_sm}},
        "learned": {"value": round(learned_gbs, 3), "ms_per_step": round(ms_learned, 3),
                    "link_gbs": round(link_l, 1), "chunk_bytes": int(tuned.chunk_bytes),
                    "n_slots": int(tuned.n_slots),
                    "kernel_shape": {"kernel": KERNEL_SHAPES.get(int(tuned.kernel_rows), "?"),
                                     "blocks_per_sm": int(tuned.blocks_per_sm)},
                    "h2d_staging": ("copy kernel, %d blocks" % tuned.h2d_copy_blocks) if tuned.h2d_copy_blocks
                    else "copy engine",
                    "graphs": True, "late": "per chunk (regressor)",
                    "regressor_chunks_logged": int(n_log), "clocks": clk2.summary()},
    }
    use_learned = learned_gbs >= plain_gbs
    host_gbs = learned_gbs if use_learned else plain_gbs

    def step_roofline(stats_list, ms):
        """Time the step's bytes need at the measured peaks (link: copy-engine
        bytes plus zero-copy granules against the pinned H2D peak of this run;
        HBM: each staged byte written by the copy engine and read by the fused
        kernel) over the measured step time."""
        link_b = sum(s["bytes_h2d"] + s["bytes_zero_copy"] for s in stats_list) / args.steps
        hbm_b = 2 * sum(s["bytes_h2d"] for s in stats_list) / args.steps
        t_link = link_b / (h2d_peak * 1e6)
        t_hbm = hbm_b / (hbm_peak * 1e6)
        return {"bound": "link" if t_link >= t_hbm else "hbm", "link_bytes": int(link_b), "hbm_bytes": int(hbm_b),
                "link_peak_gbs": round(h2d_peak, 1), "hbm_peak_gbs": hbm_peak,
                "roofline_ms": round(max(t_link, t_hbm), 3), "ms_per_step": round(ms, 3),
                "link_gbs": round(link_b / (ms * 1e6), 1), "link_frac": round(link_b / (ms * 1e6) / h2d_peak, 4),
                "frac": round(max(t_link, t_hbm) / ms, 4)}

    forms["plain"]["step_roofline"] = step_roofline(stats_all, ms_step)
    forms["learned"]["step_roofline"] = step_roofline(stats_l, ms_learned)
    for fname, sl in (("plain", stats_all), ("learned", stats_l)):
        forms[fname]["query_link_gbs"] = {
            n: round(statistics.median((s["bytes_h2d"] + s["bytes_zero_copy"]) / (s["ms_total"] * 1e6)
                                       for s in sl[i::len(TEMPLATES)]), 1) for i, n in enumerate(TEMPLATES)}
    cfg.use_graphs = 0
    cfg.chunk_bytes = 64 << 20
    cfg.n_slots = 3
    cfg.kernel_rows = args.kernel_rows
    cfg.blocks_per_sm = args.blocks_per_sm
    # the end-to-end run stages the way the better form did
    cfg.h2d_copy_blocks = int(tuned.h2d_copy_blocks) if use_learned else 0
    vx.vx_set_config(ctx, cfg)

    # end to end through the public call: dimension tables rebuilt from host
    # columns every step, fact chunks copied from pinned host memory, results
    # read back to host
    e2e_stats = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vx.vx_drop_resident(ctx)
        step(e2e_stats)
    e2e_s = (time.perf_counter() - t0) / args.steps
    dim_bytes = sum(4 * len(dims[d]) * len(dims[d]["key"]) for d in dims)
    e2e_h2d = sum(s["bytes_h2d"] + s["bytes_zero_copy"] for s in e2e_stats) / args.steps + dim_bytes
    e2e_d2h = sum(s["bytes_d2h"] for s in e2e_stats) / args.steps
    e2e_gbs = logical * world / (e2e_s * 1e9)
    e2e_staging = "copy kernel, %d blocks" % cfg.h2d_copy_blocks if cfg.h2d_copy_blocks else "copy engine"
    cfg.h2d_copy_blocks = 0
    vx.vx_set_config(ctx, cfg)

    # the fused kernel's roofline in the form the value comes from (the other
    # form's under forms); what any kernel reading each launch's bytes once
    # reaches at that launch size (a plain coalesced read of them right after
    # their copy-engine transfer, event-timed the same way) is its practical
    # ceiling.  Measured after the end-to-end steps have released the graphs.
    for rf in (roofline_plain, roofline_learned):
        if rf["achieved"]:
            try:
                ceil_gbs = vx.vx_probe_stream(ctx, rf["algorithmic_bytes_per_launch"], 15)
            except vx.VxError:
                continue
            rf["launch_ceiling"] = {"kernel": "stream_read_kernel (vx_probe_stream)", "achieved": round(ceil_gbs, 1),
                                    "frac": round(ceil_gbs / hbm_peak, 4),
                                    "fused_of_ceiling": round(rf["achieved"] / ceil_gbs, 4)}
            # the same read while a chunk-sized host-to-device copy streams in,
            # as the fused kernel runs inside the pipeline
            try:
                cc = vx.vx_probe_stream_copying(ctx, rf["algorithmic_bytes_per_launch"], 15, 256 << 20)
                rf["launch_ceiling"]["under_copy"] = {"kernel": "stream_read_kernel (vx_probe_stream_copying)",
                                                      "copy_bytes": 256 << 20, "achieved": round(cc, 1),
                                                      "frac": round(cc / hbm_peak, 4),
                                                      "fused_of_ceiling": round(rf["achieved"] / cc, 4)}
            except vx.VxError:
                pass
    roofline = roofline_learned if use_learned and roofline_learned["achieved"] else roofline_plain
    roofline["form"] = "learned" if roofline is roofline_learned else "plain"
    # the step as a whole is bound by the host link: its roofline rides along
    roofline["step"] = forms["learned" if use_learned else "plain"]["step_roofline"]
    forms["plain"]["roofline"] = {k: roofline_plain.get(k) for k in ("achieved", "frac", "avg_launch_us",
                                                                     "algorithmic_bytes_per_launch", "launch_ceiling")}
    forms["learned"]["roofline"] = {k: roofline_learned.get(k) for k in ("achieved", "frac", "avg_launch_us",
                                                                         "algorithmic_bytes_per_launch",
                                                                         "launch_ceiling")}

    operators = run_ops_extra(vx, G, args, ctx, fid, did) if not args.no_extras else None
    serving = run_serving(vx, G, ctx, fid, did, args) if not args.no_extras and args.serve_queries > 0 else None
    if serving is not None and args.sweep_queries > 0:
        serving["mixed"] = run_serving_sweep(vx, G, ctx, fid, did, args)
        serving["rate_sweep"] = serving["mixed"]["rate_sweep"]
    clustered = run_clustered(vx, G, ctx, did, args) if not args.no_extras and args.clustered_rows else None

    line = {
        "metric": METRIC, "value": round(host_gbs, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": round(ms_learned if use_learned else ms_step, 3),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"star join: {args.rows}-row fact (8 int32 cols, host-resident), dims 2556/200000/"
                               f"2000000/30000, templates {TEMPLATES}, budget {args.budget_gb} GiB",
                   "rows": args.rows, "l2": "inputs larger than L2 (fact columns stream from host)",
                   "form": "learned" if use_learned else "plain"},
        "forms": forms,
        # link use of the form the value comes from
        "link": {"h2d_peak_gbs": round(h2d_peak, 1), "d2h_peak_gbs": round(d2h_peak, 1),
                 "bidir_peak_gbs": round(bid_peak, 1), "link_gbs": round(link_l if use_learned else link_gbs, 1),
                 "link_frac": round((link_l if use_learned else link_gbs) / h2d_peak, 4),
                 "host_frac": round(host_gbs / world / h2d_peak, 4)},
        "rows_per_s": round(rows_step * world / (ms_step / 1000)),
        "query_ms": per_q_ms,
        "overlap": overlap,
        "call_overhead_ms": round(statistics.median(s["host_ms"] - s["ms_total"] for s in stats_all), 3),
        "roofline": roofline, "roofline_zero_copy_gather": gather, "roofline_h2d_copy": copy_roofline,
        "e2e": {"value": round(e2e_gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": int(e2e_h2d),
                "d2h_bytes_per_step": int(e2e_d2h), "h2d_staging": e2e_staging},
        "gpu_launches": (int(sum(s["kernel_launches"] for s in stats_l)) +
                         (int(sum(s["chunks"] for s in stats_l)) if tuned.h2d_copy_blocks else 0)) if use_learned
        else launches,  # the form the value comes from; a copy-kernel launch per chunk when it stages
        "clocks": clocks,
        "setup_s": {"generate": round(t_gen, 1)},
    }
    if operators:
        line["operators"] = operators
    if serving:
        line["serving"] = serving
    if clustered:
        line["clustered"] = clustered
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = args.cpu_sample_rows or min(args.rows, 20_000_000)
        v, cores, dt = cpu_baseline(fact, dims, sample)
        line["cpu_baseline"] = {"value": round(v, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                                "sample": f"first {sample} fact rows x 6 templates ({dt:.1f} s)",
                                "single_thread": single_thread_baseline(fact, dims, sample)}
    vx.vx_close(ctx)
    del arena
    if rank == 0 and world == 1 and not args.no_extras:
        del fact
        line["sort"] = run_sort_extra(vx, G, args)
        line["join"] = run_join_extra(vx, G, args)
    line["link_frac"] = line["link"]["link_frac"]
    busy = [v["link_busy"] for v in overlap.values() if v]
    # fraction of each query's pipeline time the host-to-device copy engine
    # was busy (per-chunk timeline): 1.0 = copies back to back, fully
    # overlapping the kernels, whatever rate the link gives at the time
    line["copy_engine_busy"] = round(min(busy), 4) if busy else None
    line["roofline"]["step"]["copy_engine_busy"] = line["copy_engine_busy"]
    line["summary"] = summarize(line)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def timeline_summary(tl, bytes_h2d):
    """Copy / compute overlap of one pipeline from its per-chunk timeline
    (columns: chunk, issue, h2d start/end, kernel start/end, d2h start/end;
    ms).  Copies of one stream run one after another, so their busy time is
    the sum of their durations; gaps are idle link time between them."""
    if len(tl) == 0:
        return None
    h0, h1, k0, k1 = tl[:, 2], tl[:, 3], tl[:, 4], tl[:, 5]
    wall = float(max(k1.max(), h1.max()) - h0.min())
    dur = h1 - h0
    per_chunk = bytes_h2d / len(tl)
    gbs = per_chunk / np.maximum(dur, 1e-6) / 1e6
    gaps = np.maximum(h0[1:] - h1[:-1], 0) if len(tl) > 1 else np.zeros(0)
    # kernel time hidden under copies: kernel c overlaps copy c+1
    hidden = float(sum(max(0.0, float(min(k1[c], h1[c + 1]) - max(k0[c], h0[c + 1]))) for c in range(len(tl) - 1)))
    return {"chunks": int(len(tl)), "wall_ms": round(wall, 3), "link_busy": round(float(dur.sum()) / wall, 4),
            "chunk_copy_gbs": {"min": round(float(gbs.min()), 1), "median": round(float(np.median(gbs)), 1),
                               "max": round(float(gbs.max()), 1)},
            "gap_ms": {"sum": round(float(gaps.sum()), 3), "max": round(float(gaps.max()) if len(gaps) else 0.0, 3)},
            "kernel_ms": round(float((k1 - k0).sum()), 3),
            "kernel_hidden_frac": round(hidden / max(float((k1 - k0)[:-1].sum()), 1e-9), 4),
            "tail_ms": round(float(k1[-1] - h1[-1]), 3)}


def summarize(line):
    """The figures a reader needs first, repeated compactly as the line's last
    key: both star forms with their link use, the out-of-core operators
    learned vs plain, serving latency."""
    f = line["forms"]
    out = {"value": line["value"], "form": line["config"]["form"],
           "star_gbs": {k: f[k]["value"] for k in ("plain", "learned")},
           "star_link_frac": {k: f[k]["step_roofline"]["link_frac"] for k in ("plain", "learned")},
           "star_step_roofline_frac": {k: f[k]["step_roofline"]["frac"] for k in ("plain", "learned")},
           "fused_kernel_hbm_frac": line["roofline"].get("frac"),
           "fused_kernel_of_launch_ceiling": (line["roofline"].get("launch_ceiling") or {}).get("fused_of_ceiling"),
           "fused_kernel_of_ceiling_under_copy": ((line["roofline"].get("launch_ceiling") or {}).get("under_copy")
                                                  or {}).get("fused_of_ceiling"),
           "copy_engine_busy": line.get("copy_engine_busy")}
    g = line.get("roofline_zero_copy_gather")
    if g:
        out["gather_link_frac"] = g.get("frac")
        out["gather_survivors_per_launch"] = g.get("survivors_per_launch")
        out["gather_of_sparse_read_ceiling"] = g.get("of_ceiling")
    cr = line.get("roofline_h2d_copy")
    if cr:
        out["h2d_copy_kernel_link_frac"] = cr.get("frac")
    sv = line.get("serving")
    if sv:
        out["serving_ms"] = {"p50": sv.get("p50_ms"), "p99": sv.get("p99_ms")}
        if sv.get("rate_sweep"):
            out["serving_sweep"] = [{"load": r["load"], "p50": r["p50_ms"], "p99": r["p99_ms"], "qps": r["qps"]}
                                    for r in sv["rate_sweep"]]
    so = line.get("sort")
    if so:
        out["sort_ms"] = {k: so[k]["ms"] for k in so if isinstance(so[k], dict) and "ms" in so[k]}
        pr = so.get("presorted_runs")
        if pr:
            out["sort_runs_ms"] = {k: v["ms"] for k, v in pr.items() if isinstance(v, dict)}
        un = line["sort"].get("uniform")
        if un:
            out["sort_uniform_ms"] = {k: v["ms"] for k, v in un.items() if isinstance(v, dict)}
    op = line.get("operators")
    if op:
        out["operators_ms"] = {k: {"fused": v["fused_ms"], "operators": v["operators_ms"]} for k, v in op.items()
                               if isinstance(v, dict)}
    jo = line.get("join")
    if jo:
        out["join_ms"] = {k: jo[k]["ms"] for k in jo if isinstance(jo[k], dict) and "ms" in jo[k]}
    return out


def run_serve_only(args):
    """The serving part alone on a --rows fact table and a --budget-gb arena."""
    import torch

    import datagen as G
    import paper_2502_09541_gb300 as vx
    vx.load()
    t = time.perf_counter()
    fact, dims = make_data(args.rows, pinned=True)
    gen = time.perf_counter() - t
    budget = int(args.budget_gb * (1 << 30))
    arena = torch.empty(budget, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    ctx = vx.vx_open_ex(arena.data_ptr(), budget, stream.cuda_stream)
    fid = {c: vx.vx_register_host_column(ctx, c, fact[c]) for c in fact}
    did = {d: {a: vx.vx_register_host_column(ctx, f"{d}.{a}", arr) for a, arr in dims[d].items()} for d in dims}
    out = {"workload": "serve", "rows": args.rows, "budget_gib": args.budget_gb, "generate_s": round(gen, 1),
           "serving": run_serving(vx, G, ctx, fid, did, args)}
    vx.vx_close(ctx)
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "star":
        run_ours(args)
    elif args.workload == "serve":
        run_serve_only(args)
    elif args.workload == "ops":
        import datagen as G
        import paper_2502_09541_gb300 as vx
        vx.load()
        print(json.dumps({"workload": "ops", "operators": run_ops_extra(vx, G, args)}), flush=True)
    else:  # one out-of-core operator alone (profiling, or a user's own sizes)
        import datagen as G
        import paper_2502_09541_gb300 as vx
        vx.load()
        fn = run_sort_extra if args.workload == "sort" else run_join_extra
        print(json.dumps({"workload": args.workload, args.workload: fn(vx, G, args)}), flush=True)


if __name__ == "__main__":
    main()
