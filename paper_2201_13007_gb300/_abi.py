"""ctypes declarations of the C ABI in include/ann.h (libann.so).

Names match the C entry points. Every function raises ``AnnError`` with the
library's message when the C call returns a non-zero status. There is no
fallback: if libann.so is missing the first call fails loudly.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

ANN_OK = 0
ANN_ERR_ARG, ANN_ERR_OOM, ANN_ERR_CUDA, ANN_ERR_BUSY, ANN_ERR_TIMEOUT, ANN_ERR_STATE = -1, -2, -3, -4, -5, -6
STORAGE = {"f32": 0, "bf16": 1, "f16": 2, "e4m3": 3}
METRIC = {"l2": 0, "ip": 1}
MODE = {"sync": 0, "async": 1}
ANN_INDEX_DEVICE_INPUT = 0x1
ANN_INDEX_KEEP_F32 = 0x2
ANN_NOALLOC_SCRATCH_BYTES = 16 << 20


class AnnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libann error {code}: {msg}")
        self.code = code


class IndexInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("d_pad", ctypes.c_int32),
                ("R", ctypes.c_int32), ("storage", ctypes.c_int32), ("metric", ctypes.c_int32),
                ("has_f32", ctypes.c_int32), ("entry", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("n_hot", ctypes.c_int64)]


class QueryStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("expansions", ctypes.c_int64), ("evals", ctypes.c_int64),
                ("hash_resets", ctypes.c_int64), ("dup_dropped", ctypes.c_int64),
                ("merges", ctypes.c_int64), ("t_start_ns", ctypes.c_int64), ("t_end_ns", ctypes.c_int64)]


STATS_FIELDS = [f for f, _ in QueryStats._fields_]


class SearchParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("M0", ctypes.c_int32), ("t", ctypes.c_int32),
                ("R_ratio", ctypes.c_float), ("rerank", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("hash_bits", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("k_per_query", ctypes.c_void_p), ("L_per_query", ctypes.c_void_p),
                ("M_per_query", ctypes.c_void_p), ("stats", ctypes.c_void_p),
                ("order", ctypes.c_void_p), ("cluster", ctypes.c_int32), ("phase_cycles", ctypes.c_void_p),
                ("visited_mode", ctypes.c_int32), ("l2_prefetch", ctypes.c_int32),
                ("team_lanes", ctypes.c_int32), ("merge_rule", ctypes.c_int32), ("patience", ctypes.c_float),
                ("gather", ctypes.c_int32)]


class BucketConfig(ctypes.Structure):
    _fields_ = [("L_max", ctypes.c_int32), ("threads", ctypes.c_int32), ("hash_bits", ctypes.c_int32)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("streams", ctypes.c_int32),
                ("max_k", ctypes.c_int32), ("max_L", ctypes.c_int32), ("max_M", ctypes.c_int32),
                ("mode", ctypes.c_int32), ("rerank", ctypes.c_int32), ("scratch_bytes", ctypes.c_int64)]


class Result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("k", ctypes.c_int32), ("status", ctypes.c_int32),
                ("latency_us", ctypes.c_double), ("device_us", ctypes.c_double),
                ("device_start_ns", ctypes.c_int64), ("device_end_ns", ctypes.c_int64)]


class LaunchInfo(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("smem_bytes", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("hash_bits", ctypes.c_int32), ("cluster", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("visited_slot_bytes", ctypes.c_int32), ("visited_ways", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libann.so (compiling it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if _build.needs_build():
                path = _build.build()
            if not os.path.exists(path):
                raise AnnError(ANN_ERR_STATE, f"{path} is missing; run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            L.ann_index_create.argtypes = [vp, i64, i32, i32, vp, i32, i64, i32, i32, ctypes.POINTER(vp)]
            L.ann_index_destroy.argtypes = [vp]
            L.ann_index_destroy.restype = None
            L.ann_index_get_info.argtypes = [vp, ctypes.POINTER(IndexInfo)]
            L.ann_index_group_neighbors.argtypes = [vp, ctypes.c_float, i32]
            L.ann_knn_bf16.argtypes = [vp, i64, i32, vp, i64, i64, i32, i32, vp, vp, vp]
            L.ann_search.argtypes = [vp, vp, i64, i32, i32, i32, vp, vp, vp]
            L.ann_search_ex.argtypes = [vp, vp, i64, i32, i32, i32, vp, vp, ctypes.POINTER(SearchParams), vp]
            L.ann_search_host.argtypes = [vp, vp, i64, i32, i32, i32, vp, vp, ctypes.POINTER(SearchParams), vp]
            L.ann_search_host_noalloc.argtypes = [vp, vp, i64, i32, i32, i32, vp, vp,
                                                  ctypes.POINTER(SearchParams), vp]
            L.ann_search_describe.argtypes = [vp, i64, i32, i32, i32, ctypes.POINTER(SearchParams),
                                              ctypes.POINTER(LaunchInfo)]
            L.ann_batch_create.argtypes = [vp, i64, vp, vp, vp, ctypes.POINTER(BucketConfig), i32,
                                           ctypes.POINTER(SearchParams), ctypes.POINTER(vp)]
            L.ann_batch_search.argtypes = [vp, vp, vp, vp, vp]
            L.ann_batch_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
            L.ann_batch_destroy.argtypes = [vp]
            L.ann_batch_destroy.restype = None
            L.ann_serve_create.argtypes = [vp, ctypes.POINTER(ServeConfig), ctypes.POINTER(vp)]
            L.ann_serve_destroy.argtypes = [vp]
            L.ann_serve_destroy.restype = None
            L.ann_serve_submit.argtypes = [vp, vp, i32, i32, i32, ctypes.c_uint64]
            L.ann_serve_poll.argtypes = [vp, ctypes.POINTER(Result), vp, vp, i32, i32]
            L.ann_serve_replay.argtypes = [vp, vp, i64, vp, vp, vp, vp, vp, i64, vp, vp, vp, vp, vp]
            L.ann_last_error.restype = ctypes.c_char_p
            L.ann_last_error.argtypes = []
            _lib = L
    return _lib


def ann_last_error() -> str:
    return lib().ann_last_error().decode(errors="replace")


def _check(rc):
    if rc != ANN_OK:
        raise AnnError(rc, ann_last_error())


def ann_index_create(base, n, d, storage, adj, R, entry, metric, flags) -> int:
    out = ctypes.c_void_p()
    _check(lib().ann_index_create(base, n, d, storage, adj, R, entry, metric, flags, ctypes.byref(out)))
    return out.value


def ann_index_destroy(index) -> None:
    lib().ann_index_destroy(index)


def ann_index_get_info(index) -> IndexInfo:
    info = IndexInfo()
    _check(lib().ann_index_get_info(index, ctypes.byref(info)))
    return info


def ann_index_group_neighbors(index, hot_fraction, prefetch) -> None:
    _check(lib().ann_index_group_neighbors(index, float(hot_fraction), int(prefetch)))


def ann_knn_bf16(base, n, d, queries, nq, self_offset, metric, k, out_ids, out_dists, stream) -> None:
    _check(lib().ann_knn_bf16(base, n, d, queries, nq, self_offset, metric, k, out_ids, out_dists, stream))


def ann_search(index, queries, nq, k, L, M, out_ids, out_dists, stream) -> None:
    _check(lib().ann_search(index, queries, nq, k, L, M, out_ids, out_dists, stream))


def ann_search_ex(index, queries, nq, k, L, M, out_ids, out_dists, params, stream) -> None:
    p = ctypes.byref(params) if params is not None else None
    _check(lib().ann_search_ex(index, queries, nq, k, L, M, out_ids, out_dists, p, stream))


def ann_search_host(index, queries, nq, k, L, M, out_ids, out_dists, params, stream) -> None:
    p = ctypes.byref(params) if params is not None else None
    _check(lib().ann_search_host(index, queries, nq, k, L, M, out_ids, out_dists, p, stream))


def ann_search_host_noalloc(index, queries, nq, k, L, M, out_ids, out_dists, params, stream) -> None:
    p = ctypes.byref(params) if params is not None else None
    _check(lib().ann_search_host_noalloc(index, queries, nq, k, L, M, out_ids, out_dists, p, stream))


def ann_serve_create(index, cfg) -> int:
    out = ctypes.c_void_p()
    _check(lib().ann_serve_create(index, ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(out)))
    return out.value


def ann_serve_destroy(server) -> None:
    lib().ann_serve_destroy(server)


def ann_serve_submit(server, query, k, L, M, tag) -> int:
    """Returns ANN_OK or ANN_ERR_BUSY (a full server is not an error for the
    caller); raises on any other status."""
    rc = lib().ann_serve_submit(server, query, k, L, M, tag)
    if rc not in (ANN_OK, ANN_ERR_BUSY):
        _check(rc)
    return rc


def ann_serve_poll(server, results, out_ids, out_dists, max_n, timeout_us) -> int:
    """Returns the number of completions (0 on timeout); raises on errors."""
    rc = lib().ann_serve_poll(server, results, out_ids, out_dists, max_n, timeout_us)
    if rc == ANN_ERR_TIMEOUT:
        return 0
    if rc < 0:
        _check(rc)
    return rc


def ann_serve_replay(server, queries, qi, k, L, M, arrival_us=None):
    """Drive the server with a request trace from native threads
    (ann_serve_replay). queries: host float32 (n, d); qi, k, L, M: one entry
    per request; arrival_us: submit times after the start (None = flood).
    Returns (latency_us, device_us, status, wall_us, busy_retries)."""
    import numpy as np
    q = np.ascontiguousarray(queries, np.float32)
    qi = np.ascontiguousarray(qi, np.int64)
    k = np.ascontiguousarray(k, np.int32)
    L = np.ascontiguousarray(L, np.int32)
    M = np.ascontiguousarray(M, np.int32)
    n = qi.shape[0]
    arr = None if arrival_us is None else np.ascontiguousarray(arrival_us, np.float64)
    lat = np.empty(n, np.float64)
    dev = np.empty(n, np.float64)
    st = np.empty(n, np.int32)
    wall = ctypes.c_double(0.0)
    busy = ctypes.c_int64(0)
    p = lambda a: ctypes.c_void_p(a.ctypes.data)
    _check(lib().ann_serve_replay(server, p(q), q.shape[0], p(qi), p(k), p(L), p(M),
                                  None if arr is None else p(arr), n, p(lat), p(dev), p(st),
                                  ctypes.byref(wall), ctypes.byref(busy)))
    return lat, dev, st, wall.value, busy.value


def ann_batch_create(index, nq, k, L, M, buckets, n_buckets, params) -> int:
    out = ctypes.c_void_p()
    _check(lib().ann_batch_create(index, nq, k, L, M, buckets, n_buckets,
                                  ctypes.byref(params) if params is not None else None, ctypes.byref(out)))
    return out.value


def ann_batch_search(batch, queries, out_ids, out_dists, stream) -> None:
    _check(lib().ann_batch_search(batch, queries, out_ids, out_dists, stream))


def ann_batch_info(batch):
    nb, km = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().ann_batch_info(batch, ctypes.byref(nb), ctypes.byref(km)))
    return nb.value, km.value


def ann_batch_destroy(batch) -> None:
    lib().ann_batch_destroy(batch)


def ann_search_describe(index, nq, k, L, M, params) -> dict:
    out = LaunchInfo()
    p = ctypes.byref(params) if params is not None else None
    _check(lib().ann_search_describe(index, nq, k, L, M, p, ctypes.byref(out)))
    return {f: getattr(out, f) for f, _ in LaunchInfo._fields_}
