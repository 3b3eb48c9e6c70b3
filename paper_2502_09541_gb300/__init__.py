"""Python binding of libvx (include/vx.h): argument marshalling only.

Every function here has the name of the C entry point it calls; all work runs
in the CUDA library.  Loading fails loudly if the library is missing or no
CUDA device is present — there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvx.so")
_lib = None
_lock = threading.Lock()

# ---- constants (vx.h)
VX_OK, VX_E_INVAL, VX_E_NOMEM, VX_E_CUDA, VX_E_CAPACITY, VX_E_TIMEOUT, VX_E_BUSY, VX_E_UNSUPPORTED, \
    VX_E_DUPKEY, VX_E_RANGE = 0, -1, -2, -3, -4, -5, -6, -7, -8, -9
VX_I32, VX_U32, VX_I64, VX_U64 = 0, 1, 2, 3
VX_SCHED_IMMEDIATE, VX_SCHED_DAG = 0, 1
VX_LATE_AUTO, VX_LATE_FORCE_EARLY, VX_LATE_FORCE_LATE, VX_LATE_PER_CHUNK = 0, 1, 2, 3
VX_BETWEEN, VX_EQ, VX_NE, VX_LT, VX_LE, VX_GT, VX_GE = range(7)
VX_AGG_COUNT, VX_AGG_SUM, VX_AGG_MUL, VX_AGG_SUB = range(4)
VX_MAX_DIMS, VX_MAX_PREDS, VX_MAX_GKEYS = 8, 8, 4
I32MIN = -2**31

_NP_DTYPE = {np.dtype(np.int32): VX_I32, np.dtype(np.uint32): VX_U32, np.dtype(np.int64): VX_I64,
             np.dtype(np.uint64): VX_U64}


class VxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"vx status {status}: {msg}")
        self.status = status


# ---- structs (vx.h)
class vx_config(ctypes.Structure):
    _fields_ = [("chunk_bytes", ctypes.c_uint64), ("n_slots", ctypes.c_int32), ("sched", ctypes.c_int32),
                ("late_mat", ctypes.c_int32), ("zc_threshold", ctypes.c_double), ("use_graphs", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("wait_timeout_ms", ctypes.c_uint32), ("log_chunk_stats", ctypes.c_int32),
                ("log_timeline", ctypes.c_int32), ("kernel_rows", ctypes.c_int32),
                ("lookback_spin_limit", ctypes.c_uint32), ("h2d_copy_blocks", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class vx_pred(ctypes.Structure):
    _fields_ = [("col", ctypes.c_int32), ("op", ctypes.c_int32), ("lo", ctypes.c_int32), ("hi", ctypes.c_int32)]


class vx_plan_dim(ctypes.Structure):
    _fields_ = [("key_col", ctypes.c_int32), ("fact_fk_col", ctypes.c_int32), ("n_attr", ctypes.c_int32),
                ("attr_col", ctypes.c_int32 * 4), ("n_preds", ctypes.c_int32), ("pred_attr", ctypes.c_int32 * 4),
                ("pred_op", ctypes.c_int32 * 4), ("pred_lo", ctypes.c_int32 * 4), ("pred_hi", ctypes.c_int32 * 4)]


class vx_plan_gkey(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("attr", ctypes.c_int32), ("card", ctypes.c_int32),
                ("fact_col", ctypes.c_int32)]


class vx_plan(ctypes.Structure):
    _fields_ = [("n_dims", ctypes.c_int32), ("dims", vx_plan_dim * VX_MAX_DIMS), ("n_fact_preds", ctypes.c_int32),
                ("fact_preds", vx_pred * VX_MAX_PREDS), ("n_group_keys", ctypes.c_int32),
                ("group_keys", vx_plan_gkey * VX_MAX_GKEYS), ("agg_op", ctypes.c_int32), ("agg_a", ctypes.c_int32),
                ("agg_b", ctypes.c_int32), ("late_mat", ctypes.c_int32), ("row_begin", ctypes.c_uint64),
                ("row_end", ctypes.c_uint64)]


class vx_query_stats(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_uint64), ("survivors", ctypes.c_uint64), ("chunks", ctypes.c_uint64),
                ("bytes_h2d", ctypes.c_uint64), ("bytes_d2h", ctypes.c_uint64), ("bytes_zero_copy", ctypes.c_uint64),
                ("bytes_logical", ctypes.c_uint64), ("late_mask", ctypes.c_uint32),
                ("overflow_retries", ctypes.c_uint32), ("est_selectivity", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_kernel", ctypes.c_double), ("kernel_launches", ctypes.c_uint64),
                ("late_chunks", ctypes.c_uint64), ("ms_gather", ctypes.c_double),
                ("ms_features", ctypes.c_double), ("surv_list_bytes", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class vx_result(ctypes.Structure):
    _fields_ = [("cap", ctypes.c_uint64), ("gid", ctypes.c_void_p), ("sum", ctypes.c_void_p),
                ("cnt", ctypes.c_void_p), ("n_out", ctypes.c_uint64), ("stats", vx_query_stats)]


VX_PART_SAMPLE, VX_PART_LEARNED_PL, VX_PART_LEARNED_MLP = 0, 1, 2
VX_JOIN_DIRECT, VX_JOIN_RADIX = 0, 1
VX_SORT_PARTITION, VX_SORT_MERGE = 0, 1


class vx_sort_opts(ctypes.Structure):
    _fields_ = [("partitioner", ctypes.c_int32), ("n_partitions", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("sample_size", ctypes.c_uint64), ("mlp_steps", ctypes.c_uint32), ("region_slack_pct", ctypes.c_uint32),
                ("host_scratch", ctypes.c_void_p), ("host_scratch_bytes", ctypes.c_uint64),
                ("max_slot_pairs", ctypes.c_uint64), ("splitters_out", ctypes.c_void_p), ("plan", ctypes.c_int32),
                ("runs_mode", ctypes.c_int32)]


class vx_sort_stats(ctypes.Structure):
    _fields_ = [("n_partitions", ctypes.c_uint32), ("passthrough_partitions", ctypes.c_uint32),
                ("overflow_retries", ctypes.c_uint32), ("contiguous_layout", ctypes.c_uint32),
                ("max_partition", ctypes.c_uint64), ("min_partition", ctypes.c_uint64),
                ("slot_pairs", ctypes.c_uint64), ("imbalance", ctypes.c_double), ("ms_sample", ctypes.c_double),
                ("ms_train", ctypes.c_double), ("ms_partition", ctypes.c_double), ("ms_sort", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("bytes_h2d", ctypes.c_uint64), ("bytes_d2h", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("ms_sort_kernel", ctypes.c_double),
                ("radix_pass_pairs", ctypes.c_uint64), ("out_of_region_pairs", ctypes.c_uint64),
                ("spill_buffers", ctypes.c_uint64), ("plan", ctypes.c_uint32), ("n_runs", ctypes.c_uint32),
                ("ms_merge_kernel", ctypes.c_double), ("merge_pass_pairs", ctypes.c_uint64),
                ("natural_runs", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class vx_join_opts(ctypes.Structure):
    _fields_ = [("partitioner", ctypes.c_int32), ("n_partitions", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("sample_size", ctypes.c_uint64), ("load_factor", ctypes.c_double), ("count_pass", ctypes.c_int32),
                ("algorithm", ctypes.c_int32), ("radix_bits", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class vx_join_result(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("payload_sum", ctypes.c_uint64), ("pair_fp", ctypes.c_uint64),
                ("n_partitions", ctypes.c_uint32), ("overflow_retries", ctypes.c_uint32),
                ("max_partition", ctypes.c_uint64), ("bytes_h2d", ctypes.c_uint64),
                ("kernel_launches", ctypes.c_uint64), ("ms_sample", ctypes.c_double), ("ms_train", ctypes.c_double),
                ("ms_build", ctypes.c_double), ("ms_probe", ctypes.c_double), ("ms_kernel", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_probe_kernel", ctypes.c_double), ("bytes_d2h", ctypes.c_uint64),
                ("algorithm", ctypes.c_uint32), ("ranges", ctypes.c_uint32), ("ms_partition", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class vx_serve_opts(ctypes.Structure):
    _fields_ = [("chunk_rows", ctypes.c_uint64), ("max_active", ctypes.c_uint32), ("n_slots", ctypes.c_uint32)]


class vx_serve_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("cycles", ctypes.c_uint64), ("bytes_h2d", ctypes.c_uint64), ("active_peak", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("wall_ms", ctypes.c_double), ("work_rows", ctypes.c_uint64),
                ("ms_kernel", ctypes.c_double), ("ms_admit", ctypes.c_double), ("ms_cycle", ctypes.c_double),
                ("ms_wait", ctypes.c_double), ("completed_kind", ctypes.c_uint64 * 3),
                ("p50_kind_ms", ctypes.c_double * 3), ("p99_kind_ms", ctypes.c_double * 3)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if k.endswith("_kind") or k.endswith("_kind_ms") else getattr(self, k))
                for k, _ in self._fields_}


VX_QUERY_STAR, VX_QUERY_SORT, VX_QUERY_JOIN = 0, 1, 2


class vx_op_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("key_col", ctypes.c_int32), ("val_col", ctypes.c_int32),
                ("probe_col", ctypes.c_int32), ("row_begin", ctypes.c_uint64), ("row_end", ctypes.c_uint64),
                ("out_keys", ctypes.c_void_p), ("out_rowids", ctypes.c_void_p), ("device_budget", ctypes.c_uint64),
                ("sort", vx_sort_opts), ("join", vx_join_opts)]


class vx_op_result(ctypes.Structure):
    _fields_ = [("sort", vx_sort_stats), ("join", vx_join_result), ("ms_total", ctypes.c_double),
                ("ms_queued", ctypes.c_double)]


_P = ctypes.POINTER
_vp, _u64, _i32, _u32, _dbl = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_double
_f32 = ctypes.c_float
SIGNATURES = {
    "vx_open": ([_u64, _P(_vp)], _i32),
    "vx_open_ex": ([_vp, _u64, _vp, _P(_vp)], _i32),
    "vx_close": ([_vp], _i32),
    "vx_last_error": ([], ctypes.c_char_p),
    "vx_get_config": ([_vp, _P(vx_config)], _i32),
    "vx_set_config": ([_vp, _P(vx_config)], _i32),
    "vx_register_host_column": ([_vp, ctypes.c_char_p, _i32, _vp, _u64, _u32, _P(_i32)], _i32),
    "vx_unregister_host_column": ([_vp, _i32], _i32),
    "vx_filter": ([_vp, _P(vx_pred), _i32, _u64, _u64, _vp, _u64, _P(_u64)], _i32),
    "vx_run_plan": ([_vp, _P(vx_plan), _P(vx_result)], _i32),
    "vx_run_plan_operators": ([_vp, _P(vx_plan), _P(vx_result)], _i32),
    "vx_groupby": ([_vp, _P(vx_plan_gkey), _i32, _i32, _i32, _i32, _P(vx_pred), _i32, _P(vx_result)], _i32),
    "vx_last_stats": ([_vp, _P(vx_query_stats)], _i32),
    "vx_last_timeline": ([_vp, _vp, _u64, _P(_u64)], _i32),
    "vx_drop_resident": ([_vp], _i32),
    "vx_probe_link": ([_vp, _u64, _u64, _P(_dbl), _P(_dbl), _P(_dbl)], _i32),
    "vx_probe_hbm_random": ([_vp, _u64, _u64, _P(_dbl)], _i32),
    "vx_probe_stream": ([_vp, _u64, _i32, _P(_dbl)], _i32),
    "vx_probe_zero_copy": ([_vp, _u64, _vp, _i32, _vp, _vp, _vp], _i32),
    "vx_probe_zero_copy_gather": ([_vp, _u64, _u32, _u64, _P(_dbl), _P(_dbl), _P(_u64)], _i32),
    "vx_probe_stream_copying": ([_vp, _u64, _i32, _u64, _P(_dbl)], _i32),
    "vx_sort": ([_vp, _i32, _i32, _vp, _vp, _P(vx_sort_opts), _P(vx_sort_stats)], _i32),
    "vx_radix_sort_pairs": ([_vp, _vp, _vp, _u64, _vp, _vp], _i32),
    "vx_range_partition": ([_vp, _vp, _vp, _u64, _vp, _u32, _vp, _vp, _vp], _i32),
    "vx_sort_splitters": ([_vp, _i32, _i32, _u32, _u64, _u64, _vp, _P(_u32)], _i32),
    "vx_mlp_loss_grad": ([_vp, _vp, _i32, _vp, _vp, _u64, _vp, _vp], _i32),
    "vx_mlp_train": ([_vp, _vp, _i32, _vp, _vp, _u64, _u32, _f32, _vp], _i32),
    "vx_join": ([_vp, _i32, _i32, _i32, _P(vx_join_opts), _P(vx_join_result)], _i32),
    "vx_autotune": ([_vp, _P(vx_plan), _u64, _P(vx_config)], _i32),
    "vx_regressor_fit": ([_vp, _vp, _vp, _u64, _i32, _f32, _vp], _i32),
    "vx_regressor_train": ([_vp, _f32, _vp, _P(_u64)], _i32),
    "vx_chunk_log": ([_vp, _vp, _vp, _u64, _P(_u64)], _i32),
    "vx_regressor_set": ([_vp, _vp, _i32], _i32),
    "vx_chunk_log_clear": ([_vp], _i32),
    "vx_serve_start": ([_vp, _P(vx_serve_opts)], _i32),
    "vx_submit": ([_vp, _P(vx_plan), _P(_u64)], _i32),
    "vx_poll": ([_vp, _u64, _P(vx_result), _P(_i32)], _i32),
    "vx_wait": ([_vp, _u64, _P(vx_result), _u32], _i32),
    "vx_serve_stats_get": ([_vp, _P(vx_serve_stats)], _i32),
    "vx_serve_stop": ([_vp], _i32),
    "vx_submit_op": ([_vp, _P(vx_op_request), _P(_u64)], _i32),
    "vx_wait_op": ([_vp, _u64, _P(vx_op_result), _u32], _i32),
    "vx_radix_cluster": ([_vp, _vp, _u64, _i32, _vp, _vp, _vp], _i32),
    "vx_exact_splits": ([_vp, _vp, _vp, _u32, _vp, _u32, _vp], _i32),
    "vx_merge_runs": ([_vp, _vp, _vp, _vp, _u32, _vp, _vp], _i32),
    "vx_filter_device_static": ([_vp, _i32, _P(vx_pred), _i32, _u64, _u64, _vp, _u64, _P(_u64), _vp], _i32),
}


def load(build_if_missing: bool = True):
    """Loads libvx.so (building it in-tree first if asked).  Raises if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                from . import build as _b
                _b.build()
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libvx.so not built at {LIB_PATH}")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(st):
    if st != VX_OK:
        raise VxError(st, load().vx_last_error().decode(errors="replace"))
    return st


def vx_last_error() -> str:
    return load().vx_last_error().decode(errors="replace")


# ------------------------------------------------------------------ thin wrappers
def vx_open(device_budget_bytes: int):
    h = ctypes.c_void_p()
    _check(load().vx_open(device_budget_bytes, ctypes.byref(h)))
    return h


def vx_open_ex(dev_ptr: int, nbytes: int, stream: int | None = None):
    h = ctypes.c_void_p()
    _check(load().vx_open_ex(dev_ptr, nbytes, stream, ctypes.byref(h)))
    return h


def vx_close(ctx):
    _check(load().vx_close(ctx))


def vx_get_config(ctx) -> vx_config:
    c = vx_config()
    _check(load().vx_get_config(ctx, ctypes.byref(c)))
    return c


def vx_set_config(ctx, cfg: vx_config):
    _check(load().vx_set_config(ctx, ctypes.byref(cfg)))


def vx_register_host_column(ctx, name: str, array: np.ndarray) -> int:
    assert array.flags["C_CONTIGUOUS"]
    cid = ctypes.c_int32()
    _check(load().vx_register_host_column(ctx, name.encode(), _NP_DTYPE[array.dtype], array.ctypes.data,
                                          len(array), 0, ctypes.byref(cid)))
    return cid.value


def vx_unregister_host_column(ctx, col_id: int):
    _check(load().vx_unregister_host_column(ctx, col_id))


def vx_filter(ctx, preds, row_begin=0, row_end=0, out: np.ndarray | None = None):
    """preds: list of (col_id, op, lo, hi).  Returns (status, count); writes out."""
    arr = (vx_pred * len(preds))(*[vx_pred(*p) for p in preds])
    cnt = ctypes.c_uint64()
    st = load().vx_filter(ctx, arr, len(preds), row_begin, row_end, None if out is None else out.ctypes.data,
                          0 if out is None else len(out), ctypes.byref(cnt))
    if st not in (VX_OK, VX_E_CAPACITY):
        _check(st)
    return st, cnt.value


def vx_filter_device_static(col_ptrs, preds, n_rows: int, row0: int, out_ptr: int, cap: int, stream: int = 0):
    """Allocation-free filter over device columns (col_ptrs: device addresses;
    preds: (index into col_ptrs, op, lo, hi)).  Returns (status, count)."""
    cols = (ctypes.c_void_p * len(col_ptrs))(*col_ptrs)
    arr = (vx_pred * len(preds))(*[vx_pred(*p) for p in preds])
    cnt = ctypes.c_uint64()
    st = load().vx_filter_device_static(cols, len(col_ptrs), arr, len(preds), n_rows, row0, out_ptr or None, cap,
                                        ctypes.byref(cnt), stream or None)
    if st not in (VX_OK, VX_E_CAPACITY):
        _check(st)
    return st, cnt.value


def vx_run_plan(ctx, plan: vx_plan, cap: int = 1 << 16):
    """Returns (status, gid, sum, cnt, stats) with arrays trimmed to n_out."""
    gid = np.zeros(cap, np.uint64)
    s = np.zeros(cap, np.int64)
    c = np.zeros(cap, np.uint64)
    res = vx_result(cap, gid.ctypes.data, s.ctypes.data, c.ctypes.data, 0, vx_query_stats())
    st = load().vx_run_plan(ctx, ctypes.byref(plan), ctypes.byref(res))
    if st not in (VX_OK, VX_E_CAPACITY):
        _check(st)
    n = min(res.n_out, cap)
    return st, gid[:n], s[:n], c[:n], res.stats.as_dict()


def vx_run_plan_operators(ctx, plan: vx_plan, cap: int = 1 << 16):
    """The plan one operator at a time with host intermediates; returns
    (status, gid, sum, cnt, stats) like vx_run_plan."""
    gid = np.zeros(cap, np.uint64)
    s = np.zeros(cap, np.int64)
    c = np.zeros(cap, np.uint64)
    res = vx_result(cap, gid.ctypes.data, s.ctypes.data, c.ctypes.data, 0, vx_query_stats())
    st = load().vx_run_plan_operators(ctx, ctypes.byref(plan), ctypes.byref(res))
    if st not in (VX_OK, VX_E_CAPACITY):
        _check(st)
    n = min(res.n_out, cap)
    return st, gid[:n], s[:n], c[:n], res.stats.as_dict()


def vx_groupby(ctx, keys, agg_op, agg_a, agg_b, preds, cap: int = 1 << 16):
    """keys: list of (col_id, card)."""
    karr = (vx_plan_gkey * max(1, len(keys)))(*[vx_plan_gkey(-1, 0, card, col) for col, card in keys])
    parr = (vx_pred * max(1, len(preds)))(*[vx_pred(*p) for p in preds])
    gid = np.zeros(cap, np.uint64)
    s = np.zeros(cap, np.int64)
    c = np.zeros(cap, np.uint64)
    res = vx_result(cap, gid.ctypes.data, s.ctypes.data, c.ctypes.data, 0, vx_query_stats())
    st = load().vx_groupby(ctx, karr, len(keys), agg_op, agg_a, agg_b, parr, len(preds), ctypes.byref(res))
    if st not in (VX_OK, VX_E_CAPACITY):
        _check(st)
    n = min(res.n_out, cap)
    return st, gid[:n], s[:n], c[:n], res.stats.as_dict()


def vx_drop_resident(ctx):
    _check(load().vx_drop_resident(ctx))


def vx_regressor_fit(ctx, X, y, lam=0.0):
    X = np.ascontiguousarray(X, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    w = np.zeros(X.shape[1], np.float32)
    _check(load().vx_regressor_fit(ctx, X.ctypes.data, y.ctypes.data, X.shape[0], X.shape[1], lam, w.ctypes.data))
    return w


def vx_regressor_train(ctx, lam=1e-6):
    w = np.zeros(4, np.float32)
    n = ctypes.c_uint64()
    _check(load().vx_regressor_train(ctx, lam, w.ctypes.data, ctypes.byref(n)))
    return w, n.value


def vx_regressor_set(ctx, w):
    w = np.ascontiguousarray(w, np.float32)
    _check(load().vx_regressor_set(ctx, w.ctypes.data, len(w)))


def vx_chunk_log(ctx):
    n = ctypes.c_uint64()
    _check(load().vx_chunk_log(ctx, None, None, 0, ctypes.byref(n)))
    X = np.zeros((n.value, 4), np.float32)
    y = np.zeros(n.value, np.float32)
    _check(load().vx_chunk_log(ctx, X.ctypes.data, y.ctypes.data, n.value, ctypes.byref(n)))
    return X, y


def vx_chunk_log_clear(ctx):
    _check(load().vx_chunk_log_clear(ctx))


def vx_serve_start(ctx, chunk_rows=0, max_active=0, n_slots=0):
    o = vx_serve_opts(chunk_rows, max_active, n_slots)
    _check(load().vx_serve_start(ctx, ctypes.byref(o)))


def vx_submit(ctx, plan: vx_plan) -> int:
    t = ctypes.c_uint64()
    _check(load().vx_submit(ctx, ctypes.byref(plan), ctypes.byref(t)))
    return t.value


def _result_arrays(cap):
    gid = np.zeros(cap, np.uint64)
    s = np.zeros(cap, np.int64)
    c = np.zeros(cap, np.uint64)
    return gid, s, c, vx_result(cap, gid.ctypes.data, s.ctypes.data, c.ctypes.data, 0, vx_query_stats())


def vx_poll(ctx, ticket: int, cap: int = 1 << 13):
    """Returns None while running, else (status, gid, sum, cnt, stats)."""
    gid, s, c, res = _result_arrays(cap)
    done = ctypes.c_int32()
    st = load().vx_poll(ctx, ticket, ctypes.byref(res), ctypes.byref(done))
    if not done.value:
        if st != VX_OK:
            _check(st)
        return None
    n = min(res.n_out, cap)
    return st, gid[:n], s[:n], c[:n], res.stats.as_dict()


def vx_wait(ctx, ticket: int, timeout_ms: int = 600_000, cap: int = 1 << 13):
    gid, s, c, res = _result_arrays(cap)
    st = load().vx_wait(ctx, ticket, ctypes.byref(res), timeout_ms)
    if st not in (VX_OK, VX_E_CAPACITY):
        _check(st)
    n = min(res.n_out, cap)
    return st, gid[:n], s[:n], c[:n], res.stats.as_dict()


def vx_submit_op(ctx, req: vx_op_request) -> int:
    t = ctypes.c_uint64()
    _check(load().vx_submit_op(ctx, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def vx_wait_op(ctx, ticket: int, timeout_ms: int = 600_000) -> dict:
    """Waits for a sort / join ticket; returns {"sort": ..., "join": ...,
    "ms_total": ..., "ms_queued": ...}."""
    r = vx_op_result()
    _check(load().vx_wait_op(ctx, ticket, ctypes.byref(r), timeout_ms))
    return {"sort": r.sort.as_dict(), "join": r.join.as_dict(), "ms_total": r.ms_total, "ms_queued": r.ms_queued}


def vx_serve_stats_get(ctx) -> dict:
    s = vx_serve_stats()
    _check(load().vx_serve_stats_get(ctx, ctypes.byref(s)))
    return s.as_dict()


def vx_serve_stop(ctx):
    _check(load().vx_serve_stop(ctx))


def vx_autotune(ctx, plan: vx_plan, sample_rows: int) -> vx_config:
    c = vx_config()
    _check(load().vx_autotune(ctx, ctypes.byref(plan), sample_rows, ctypes.byref(c)))
    return c


TIMELINE_COLS = ("chunk", "issue", "h2d_start", "h2d_end", "kernel_start", "kernel_end", "d2h_start", "d2h_end")


def vx_last_timeline(ctx) -> np.ndarray:
    """(chunks, 8) float32 rows: chunk, load issue, h2d start/end, kernel
    start/end, d2h start/end in ms from the pipeline's start (-1: none)."""
    n = ctypes.c_uint64()
    _check(load().vx_last_timeline(ctx, None, 0, ctypes.byref(n)))
    out = np.zeros((n.value, len(TIMELINE_COLS)), np.float32)
    _check(load().vx_last_timeline(ctx, out.ctypes.data, n.value, ctypes.byref(n)))
    return out


def vx_last_stats(ctx) -> dict:
    s = vx_query_stats()
    _check(load().vx_last_stats(ctx, ctypes.byref(s)))
    return s.as_dict()


def vx_probe_zero_copy(ctx, n: int, sels):
    """Returns (ms_zero_copy[k], ms_copy[k], checksums[k]) per SEL."""
    s = np.ascontiguousarray(sels, np.int32)
    zc = np.zeros(len(s), np.float64)
    ce = np.zeros(len(s), np.float64)
    ck = np.zeros(len(s), np.uint64)
    _check(load().vx_probe_zero_copy(ctx, n, s.ctypes.data, len(s), zc.ctypes.data, ce.ctypes.data, ck.ctypes.data))
    return zc, ce, ck


def vx_probe_zero_copy_gather(ctx, window_bytes: int, n_reads: int, seed: int = 1):
    """(us_first, us_warm, checksum) of one sparse gather launch over mapped
    host memory: n_reads 4-byte reads at sorted uniform positions of a window."""
    a, b, c = _dbl(), _dbl(), _u64()
    _check(load().vx_probe_zero_copy_gather(ctx, window_bytes, n_reads, seed, ctypes.byref(a), ctypes.byref(b),
                                            ctypes.byref(c)))
    return a.value, b.value, c.value


def vx_probe_stream(ctx, nbytes: int, reps: int) -> float:
    """GB/s of one coalesced read of nbytes right after their host-to-device
    copy (median of reps launches)."""
    r = _dbl()
    _check(load().vx_probe_stream(ctx, nbytes, reps, ctypes.byref(r)))
    return r.value


def vx_probe_stream_copying(ctx, nbytes: int, reps: int, copy_bytes: int) -> float:
    """GB/s of the same read with a host-to-device copy of copy_bytes in flight."""
    r = _dbl()
    _check(load().vx_probe_stream_copying(ctx, nbytes, reps, copy_bytes, ctypes.byref(r)))
    return r.value


def vx_probe_hbm_random(ctx, table_bytes: int, n_reads: int) -> float:
    """1e9 random 16-byte reads per second from 32-byte buckets of a table."""
    r = _dbl()
    _check(load().vx_probe_hbm_random(ctx, table_bytes, n_reads, ctypes.byref(r)))
    return r.value


def vx_probe_link(ctx, nbytes: int, chunk: int):
    a, b, c = _dbl(), _dbl(), _dbl()
    _check(load().vx_probe_link(ctx, nbytes, chunk, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


# ------------------------------------------------------------------ sort / partition / learned
def _np(a, dt):
    a = np.ascontiguousarray(a, dtype=dt)
    return a


def vx_sort(ctx, key_col: int, rowid_col: int, out_keys: np.ndarray, out_rowids: np.ndarray,
            opts: vx_sort_opts | None = None):
    """Returns the stats dict; fills out_keys/out_rowids."""
    st = vx_sort_stats()
    _check(load().vx_sort(ctx, key_col, rowid_col, out_keys.ctypes.data, out_rowids.ctypes.data,
                          None if opts is None else ctypes.byref(opts), ctypes.byref(st)))
    return st.as_dict()


def vx_join(ctx, build_key: int, build_payload: int, probe_key: int, opts: vx_join_opts | None = None) -> dict:
    r = vx_join_result()
    _check(load().vx_join(ctx, build_key, build_payload, probe_key, None if opts is None else ctypes.byref(opts),
                          ctypes.byref(r)))
    return r.as_dict()


def vx_radix_sort_pairs(ctx, keys, vals):
    keys, vals = _np(keys, np.uint64), _np(vals, np.uint32)
    ok, ov = np.empty_like(keys), np.empty_like(vals)
    _check(load().vx_radix_sort_pairs(ctx, keys.ctypes.data, vals.ctypes.data, len(keys), ok.ctypes.data,
                                      ov.ctypes.data))
    return ok, ov


def vx_range_partition(ctx, keys, vals, splitters):
    keys, vals = _np(keys, np.uint64), _np(vals, np.uint32)
    spl = _np(splitters, np.uint64)
    P = len(spl) + 1
    ok, ov = np.empty_like(keys), np.empty_like(vals)
    b = np.zeros(P + 1, np.uint64)
    _check(load().vx_range_partition(ctx, keys.ctypes.data, vals.ctypes.data, len(keys),
                                     spl.ctypes.data if len(spl) else None, P, ok.ctypes.data, ov.ctypes.data,
                                     b.ctypes.data))
    return ok, ov, b


def vx_sort_splitters(ctx, key_col: int, partitioner: int, n_partitions: int, sample_size=0, seed=0):
    out = np.zeros(2 * (n_partitions - 1), np.uint64)
    k = ctypes.c_uint32()
    _check(load().vx_sort_splitters(ctx, key_col, partitioner, n_partitions, sample_size, seed, out.ctypes.data,
                                    ctypes.byref(k)))
    return out[:k.value].copy()


def vx_radix_cluster(ctx, keys, bits):
    """(clustered keys, chunk-local rows, boundary array of 2^bits + 1)."""
    keys = _np(keys, np.uint64)
    ok = np.empty_like(keys)
    rows = np.empty(len(keys), np.uint32)
    bnd = np.zeros((1 << bits) + 1, np.uint32)
    _check(load().vx_radix_cluster(ctx, keys.ctypes.data, len(keys), bits, ok.ctypes.data, rows.ctypes.data,
                                   bnd.ctypes.data))
    return ok, rows, bnd


def vx_exact_splits(ctx, keys, run_off, ranks):
    """Per rank, the elements of each sorted run left of the exact cut:
    array (len(ranks), n_runs)."""
    keys = _np(keys, np.uint64)
    ro = _np(run_off, np.uint64)
    rk = _np(ranks, np.uint64)
    out = np.zeros((len(rk), len(ro) - 1), np.uint64)
    _check(load().vx_exact_splits(ctx, keys.ctypes.data, ro.ctypes.data, len(ro) - 1,
                                  rk.ctypes.data if len(rk) else None, len(rk), out.ctypes.data))
    return out


def vx_merge_runs(ctx, keys, vals, run_off):
    """Stable in-HBM merge of the sorted runs [run_off[r], run_off[r+1])."""
    keys, vals = _np(keys, np.uint64), _np(vals, np.uint32)
    ro = _np(run_off, np.uint64)
    ok, ov = np.empty_like(keys), np.empty_like(vals)
    _check(load().vx_merge_runs(ctx, keys.ctypes.data, vals.ctypes.data, ro.ctypes.data, len(ro) - 1,
                                ok.ctypes.data, ov.ctypes.data))
    return ok, ov


def vx_mlp_loss_grad(ctx, theta, H, x, t):
    th, x, t = _np(theta, np.float32), _np(x, np.float32), _np(t, np.float32)
    g = np.zeros(3 * H + 1, np.float32)
    loss = np.zeros(1, np.float32)
    _check(load().vx_mlp_loss_grad(ctx, th.ctypes.data, H, x.ctypes.data, t.ctypes.data, len(x), g.ctypes.data,
                                   loss.ctypes.data))
    return float(loss[0]), g


def vx_mlp_train(ctx, theta, H, x, t, steps, lr):
    th = np.array(theta, dtype=np.float32, copy=True)
    x, t = _np(x, np.float32), _np(t, np.float32)
    loss = np.zeros(1, np.float32)
    _check(load().vx_mlp_train(ctx, th.ctypes.data, H, x.ctypes.data, t.ctypes.data, len(x), steps, lr,
                               loss.ctypes.data))
    return th, float(loss[0])


# ------------------------------------------------------------------ plan marshalling
def make_plan(tmpl: dict, fact_ids: dict, dim_ids: dict, attr_cards: dict, late_mat=VX_LATE_AUTO,
              row_begin=0, row_end=0) -> vx_plan:
    """Marshals a template dict (dims / fact_preds / group / agg, predicates as
    inclusive int32 ranges) into a vx_plan.  fact_ids: fact column -> id;
    dim_ids: dim -> {"key": id, attr: id}; attr_cards: dim -> {attr: card} in
    attribute order."""
    attr_names = {d: list(v.keys()) for d, v in attr_cards.items()}
    p = vx_plan()
    p.n_dims = len(tmpl["dims"])
    dindex = {}
    for d, spec in enumerate(tmpl["dims"]):
        attrs = attr_names[spec["dim"]]
        pd = p.dims[d]
        pd.key_col = dim_ids[spec["dim"]]["key"]
        pd.fact_fk_col = fact_ids[spec["fk"]]
        pd.n_attr = len(attrs)
        for k, a in enumerate(attrs):
            pd.attr_col[k] = dim_ids[spec["dim"]][a]
        pd.n_preds = len(spec["preds"])
        for k, (a, lo, hi) in enumerate(spec["preds"]):
            pd.pred_attr[k] = attrs.index(a)
            pd.pred_op[k] = VX_BETWEEN
            pd.pred_lo[k] = lo
            pd.pred_hi[k] = hi
        dindex[spec["dim"]] = d
    p.n_fact_preds = len(tmpl["fact_preds"])
    for k, (c, lo, hi) in enumerate(tmpl["fact_preds"]):
        p.fact_preds[k] = vx_pred(fact_ids[c], VX_BETWEEN, lo, hi)
    p.n_group_keys = len(tmpl["group"])
    for k, g in enumerate(tmpl["group"]):
        dname, a = g
        p.group_keys[k] = vx_plan_gkey(dindex[dname], attr_names[dname].index(a), attr_cards[dname][a], -1)
    op, a, b = tmpl["agg"]
    p.agg_op = {"sum": VX_AGG_SUM, "mul": VX_AGG_MUL, "sub": VX_AGG_SUB, "count": VX_AGG_COUNT}[op]
    p.agg_a = fact_ids[a] if a else -1
    p.agg_b = fact_ids[b] if b else -1
    p.late_mat = late_mat
    p.row_begin = row_begin
    p.row_end = row_end
    return p
