"""FP64 CPU oracle for graph-based best-first ANN search (Speed-ANN, arXiv 2201.13007).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline and reference legs may import this package. The
product library ``paper_2201_13007_gb300`` never imports it, and the two share
no code.

The arithmetic lives in ``oracle.c`` (plain C, FP64); this module compiles it
with gcc and marshals numpy arrays through ctypes. Function-to-passage map:

- :func:`exact_knn`  -- Def. 1 (K-NNS), Sec. 2.1, brute force.
- :func:`exact_knn_gemm`, :func:`exact_knn_blocked` -- Def. 1 through FP64
  matrix products (whole, or by blocks of base rows for 10M-point sets).
- :func:`search` with ``algo="bfis"``  -- Algorithm 1 (BFiS).
- :func:`search` with ``algo="topm"``  -- Sec. 4.1 top-M parallel neighbour
  expansion (BSP) with the Sec. 4.2 staged schedule.
- :func:`search` with ``algo="speedann"`` -- Algorithm 3 + Algorithm 2
  (update-position CheckMetrics), deterministic lock-step simulation.
- :func:`round_bf16`, :func:`round_fp16`, :func:`round_e4m3`,
  :func:`fp8_scaled` -- storage formats of the reduced-precision variant.
- :func:`rerank` -- exact FP32-row re-rank of a candidate list.
- :func:`recall` -- Eq. (recall), Sec. 2.1: |R' n R| / K.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ALGOS = {"bfis": 0, "topm": 1, "speedann": 2}
METRICS = {"l2": 0, "ip": 1}


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so with gcc (no fast-math, so
    IEEE double arithmetic is kept as written)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
             "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Graph(ctypes.Structure):
    _fields_ = [("base", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32),
                ("adj", ctypes.c_void_p), ("R", ctypes.c_int32), ("entry", ctypes.c_int64),
                ("metric", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("K", ctypes.c_int32), ("M0", ctypes.c_int32),
                ("M_max", ctypes.c_int32), ("t", ctypes.c_int32), ("R_ratio", ctypes.c_double),
                ("merge_rule", ctypes.c_int32), ("patience", ctypes.c_double),
                ("max_steps", ctypes.c_int64), ("tie_tol", ctypes.c_double),
                ("tie_abs", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("expansions", ctypes.c_int64),
                ("evals", ctypes.c_int64), ("merges", ctypes.c_int64),
                ("substeps", ctypes.c_int64), ("tie_events", ctypes.c_int64)]


class Trace(ctypes.Structure):
    _fields_ = [("queue_ids", ctypes.c_void_p), ("queue_keys", ctypes.c_void_p),
                ("queue_checked", ctypes.c_void_p), ("queue_len", ctypes.c_int32),
                ("visited", ctypes.c_void_p), ("n_visited", ctypes.c_int64),
                ("visited_cap", ctypes.c_int64), ("expanded", ctypes.c_void_p),
                ("n_expanded", ctypes.c_int64), ("expanded_cap", ctypes.c_int64)]


STATS_FIELDS = [f for f, _ in Stats._fields_]
_STATS_DTYPE = np.dtype([(f, np.int64) for f in STATS_FIELDS])


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ANN_ORACLE_LIB lets the planted-mistake tests load a mutated copy
            path = os.environ.get("ANN_ORACLE_LIB") or build()
            L = ctypes.CDLL(path)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            L.orc_search.argtypes = [i32, ctypes.POINTER(Graph), ctypes.POINTER(Params), vp, i64,
                                     vp, vp, vp, i32]
            L.orc_search_trace.argtypes = [i32, ctypes.POINTER(Graph), ctypes.POINTER(Params), vp,
                                           vp, vp, ctypes.POINTER(Stats), ctypes.POINTER(Trace)]
            L.orc_exact_knn.argtypes = [ctypes.POINTER(Graph), vp, i64, i32, vp, vp, i32]
            L.orc_rerank.argtypes = [ctypes.POINTER(Graph), vp, i64, vp, i32, i32, vp, vp]
            for f in ("orc_round_bf16", "orc_round_fp16", "orc_round_e4m3"):
                getattr(L, f).argtypes = [vp, i64, vp]
            L.orc_fp8_scaled.argtypes = [vp, i64, i32, vp, vp]
            _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _graph(base, adj, entry, metric):
    base = _f32(base)
    adj = np.ascontiguousarray(adj, dtype=np.int32)
    if base.ndim != 2 or adj.ndim != 2 or adj.shape[0] != base.shape[0]:
        raise ValueError("base must be n x d and adj n x R")
    g = Graph(base=base.ctypes.data, n=base.shape[0], d=base.shape[1], adj=adj.ctypes.data,
              R=adj.shape[1], entry=int(entry), metric=METRICS[metric])
    return g, (base, adj)


def _params(L, K, M0=1, M_max=1, t=1, R_ratio=float("inf"), max_steps=-1, tie_tol=1e-5, tie_abs=0.0,
            patience=None):
    """patience=None: Algorithm 2's merge test (R_ratio); a number: the stall-count test."""
    return Params(L=int(L), K=int(K), M0=int(M0), M_max=int(M_max), t=int(t),
                  R_ratio=float(R_ratio), merge_rule=0 if patience is None else 1,
                  patience=0.0 if patience is None else float(patience), max_steps=int(max_steps),
                  tie_tol=float(tie_tol), tie_abs=float(tie_abs))


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc}")


def search(base, adj, entry, queries, *, algo="topm", metric="l2", L, K, M0=1, M_max=1, t=1,
           R_ratio=float("inf"), max_steps=-1, tie_tol=1e-5, tie_abs=0.0, nthreads=1, patience=None):
    """Run one of the paper's searches for every query. Returns (ids int64
    nq x K, keys float64 nq x K, stats structured array nq). For "speedann",
    patience=None merges by Algorithm 2 (R_ratio); a number merges by the
    stall count against that patience."""
    g, keep = _graph(base, adj, entry, metric)
    q = _f32(queries)
    if q.ndim == 1:
        q = q[None, :]
    nq = q.shape[0]
    ids = np.empty((nq, K), np.int64)
    keys = np.empty((nq, K), np.float64)
    st = np.zeros(nq, _STATS_DTYPE)
    p = _params(L, K, M0, M_max, t, R_ratio, max_steps, tie_tol, tie_abs, patience)
    rc = lib().orc_search(ALGOS[algo], ctypes.byref(g), ctypes.byref(p), _ptr(q), nq,
                          _ptr(ids), _ptr(keys), _ptr(st), int(nthreads))
    _check(rc, "search")
    del keep
    return ids, keys, st


def search_trace(base, adj, entry, query, *, algo="topm", metric="l2", L, K, M0=1, M_max=1, t=1,
                 R_ratio=float("inf"), max_steps=-1, tie_tol=1e-5, tie_abs=0.0, patience=None):
    """One query with its full final state: dict with ids, keys, stats, the
    final queue (ids, keys, checked), the visited set in visit order and the
    expansion order."""
    g, keep = _graph(base, adj, entry, metric)
    q = _f32(query).reshape(-1)
    n = g.n
    qi = np.empty(L, np.int64)
    qk = np.empty(L, np.float64)
    qc = np.empty(L, np.uint8)
    vis = np.empty(n, np.int64)
    exp_cap = n + 1
    ex = np.empty(exp_cap, np.int64)
    tr = Trace(queue_ids=qi.ctypes.data, queue_keys=qk.ctypes.data, queue_checked=qc.ctypes.data,
               queue_len=0, visited=vis.ctypes.data, n_visited=0, visited_cap=n,
               expanded=ex.ctypes.data, n_expanded=0, expanded_cap=exp_cap)
    ids = np.empty(K, np.int64)
    keys = np.empty(K, np.float64)
    st = Stats()
    p = _params(L, K, M0, M_max, t, R_ratio, max_steps, tie_tol, tie_abs, patience)
    rc = lib().orc_search_trace(ALGOS[algo], ctypes.byref(g), ctypes.byref(p), _ptr(q), _ptr(ids),
                                _ptr(keys), ctypes.byref(st), ctypes.byref(tr))
    _check(rc, "search_trace")
    del keep
    ql = tr.queue_len
    return {
        "ids": ids, "keys": keys,
        "stats": {f: getattr(st, f) for f in STATS_FIELDS},
        "queue_ids": qi[:ql].copy(), "queue_keys": qk[:ql].copy(),
        "queue_checked": qc[:ql].astype(bool),
        "visited": vis[:tr.n_visited].copy(),
        "expanded": ex[:min(tr.n_expanded, exp_cap)].copy(),
    }


def exact_knn(base, queries, K, metric="l2", nthreads=1):
    """Def. 1: brute-force K nearest neighbours in FP64; (key, id) order."""
    base = _f32(base)
    dummy_adj = np.zeros((base.shape[0], 1), np.int32)
    g, keep = _graph(base, dummy_adj, 0, metric)
    q = _f32(queries)
    if q.ndim == 1:
        q = q[None, :]
    nq = q.shape[0]
    ids = np.empty((nq, K), np.int64)
    keys = np.empty((nq, K), np.float64)
    rc = lib().orc_exact_knn(ctypes.byref(g), _ptr(q), nq, int(K), _ptr(ids), _ptr(keys), int(nthreads))
    _check(rc, "exact_knn")
    del keep
    return ids, keys


def exact_knn_gemm(base, queries, K, metric="l2", chunk=256):
    """Def. 1 through an FP64 matrix product: key = |x|^2 - 2 <q, x> (+ |q|^2)
    for l2, -<q, x> for inner product, then the K smallest by (key, id).
    When every coordinate is an integer the products and sums stay below
    2^53, so every key is exact and the answer is exactly exact_knn's; on
    other data keys differ from the direct sum only by FP64 rounding. A
    library GEMM serves as the step that forms the dot products; everything
    else is written out. Returns (ids int64 nq x K, keys float64 nq x K)."""
    X = np.ascontiguousarray(base, np.float64)
    Q = np.ascontiguousarray(queries, np.float64)
    if Q.ndim == 1:
        Q = Q[None, :]
    n = X.shape[0]
    xn = np.einsum("ij,ij->i", X, X)
    ids = np.empty((Q.shape[0], K), np.int64)
    keys = np.empty((Q.shape[0], K), np.float64)
    for a in range(0, Q.shape[0], chunk):
        q = Q[a:a + chunk]
        dot = q @ X.T
        if metric == "l2":
            D = xn[None, :] - 2.0 * dot + np.einsum("ij,ij->i", q, q)[:, None]
        else:
            D = -dot
        kk = min(K, n)
        part = np.argpartition(D, kk - 1, axis=1)[:, :kk]
        for r in range(q.shape[0]):
            kth = D[r, part[r]].max()
            cand = np.flatnonzero(D[r] <= kth)          # every id tied with the K-th key takes part
            o = np.lexsort((cand, D[r, cand]))[:kk]
            ids[a + r, :kk] = cand[o]
            keys[a + r, :kk] = D[r, cand[o]]
        if kk < K:
            ids[a:a + chunk, kk:] = -1
            keys[a:a + chunk, kk:] = np.inf
    return ids, keys


def exact_knn_blocked(base, queries, K, metric="l2", block=1 << 20, qchunk=256):
    """Def. 1 over base sets too large for one distance matrix, in plain
    PyTorch CPU ops (FP64): the keys of exact_knn_gemm, formed block by
    block of ``block`` base rows. Within a block, every id whose key is at
    most the block's K-th smallest key becomes a candidate, so ids tied at a
    block's cut all take part; the answer is the K smallest candidates by
    (key, id). The library matrix product and top-k selection serve as steps.
    Returns (ids int64 nq x K, keys float64 nq x K), padded with (-1, +inf)."""
    import torch
    Q = torch.from_numpy(np.ascontiguousarray(queries, np.float64))
    if Q.ndim == 1:
        Q = Q[None, :]
    nq = Q.shape[0]
    n = base.shape[0]
    qn = (Q * Q).sum(1)
    cand_i = [[] for _ in range(nq)]
    cand_k = [[] for _ in range(nq)]
    for a in range(0, n, block):
        Xb = torch.from_numpy(np.ascontiguousarray(base[a:a + block], np.float64))
        xn = (Xb * Xb).sum(1)
        kk = min(K, Xb.shape[0])
        for c in range(0, nq, qchunk):
            q = Q[c:c + qchunk]
            if metric == "l2":
                # |x|^2 - 2<q, x> in one product; |q|^2 is added to the selected keys
                # only (the same two roundings as |x|^2 - 2<q, x> + |q|^2)
                D = torch.addmm(xn[None, :].expand(q.shape[0], -1), q, Xb.T, beta=1.0, alpha=-2.0)
            else:
                D = torch.mm(q, Xb.T).neg_()
            kth = torch.topk(D, kk, dim=1, largest=False, sorted=True).values[:, -1]
            rows, cols = torch.nonzero(D <= kth[:, None], as_tuple=True)
            vals = D[rows, cols]
            if metric == "l2":
                vals = vals + qn[c:c + qchunk][rows]
            vals = vals.numpy()
            rows, cols = rows.numpy(), cols.numpy()
            for r in np.unique(rows):
                m = rows == r
                cand_i[c + r].append(cols[m].astype(np.int64) + a)
                cand_k[c + r].append(vals[m])
            del D
    ids = np.full((nq, K), -1, np.int64)
    keys = np.full((nq, K), np.inf)
    for r in range(nq):
        ci = np.concatenate(cand_i[r])
        ck = np.concatenate(cand_k[r])
        o = np.lexsort((ci, ck))[:K]
        ids[r, :o.size] = ci[o]
        keys[r, :o.size] = ck[o]
    return ids, keys


def rerank(base32, queries, cand, K, metric="l2"):
    """Recompute candidate keys from FP32 rows, sort by (key, id), keep K."""
    base32 = _f32(base32)
    dummy_adj = np.zeros((base32.shape[0], 1), np.int32)
    g, keep = _graph(base32, dummy_adj, 0, metric)
    q = _f32(queries)
    if q.ndim == 1:
        q = q[None, :]
    cand = np.ascontiguousarray(cand, dtype=np.int64)
    if cand.ndim == 1:
        cand = cand[None, :]
    nq = q.shape[0]
    ids = np.empty((nq, K), np.int64)
    keys = np.empty((nq, K), np.float64)
    rc = lib().orc_rerank(ctypes.byref(g), _ptr(q), nq, _ptr(cand), cand.shape[1], int(K),
                          _ptr(ids), _ptr(keys))
    _check(rc, "rerank")
    del keep
    return ids, keys


def _round(fn, x):
    x = _f32(x)
    out = np.empty_like(x)
    getattr(lib(), fn)(_ptr(x), x.size, _ptr(out))
    return out


def round_bf16(x):
    """bfloat16 value of each float32 (round to nearest even), as float32."""
    return _round("orc_round_bf16", x)


def round_fp16(x):
    """IEEE binary16 value of each float32 (round to nearest even), as float32."""
    return _round("orc_round_fp16", x)


def round_e4m3(x):
    """OCP FP8 E4M3 value (round to nearest even, saturating at +-448)."""
    return _round("orc_round_e4m3", x)


def fp8_scaled(x):
    """Per-vector scaled E4M3: returns (dequantised float32 rows, scales)."""
    x = _f32(x)
    n, d = x.shape
    deq = np.empty_like(x)
    sc = np.empty(n, np.float32)
    lib().orc_fp8_scaled(_ptr(x), n, d, _ptr(deq), _ptr(sc))
    return deq, sc


def stored_values(base, storage):
    """The float32 values a search over ``storage`` sees for FP32 rows ``base``."""
    if storage == "f32":
        return _f32(base)
    if storage == "bf16":
        return round_bf16(base)
    if storage == "f16":
        return round_fp16(base)
    if storage == "e4m3":
        return fp8_scaled(base)[0]
    raise ValueError(storage)


def recall(found_ids, true_ids):
    """Eq. (recall), Sec. 2.1: |R' n R| / K per query, K = true_ids.shape[1]."""
    found_ids = np.asarray(found_ids)
    true_ids = np.asarray(true_ids)
    K = true_ids.shape[1]
    out = np.empty(true_ids.shape[0])
    for i in range(true_ids.shape[0]):
        f = set(int(v) for v in found_ids[i, :K] if v >= 0)
        out[i] = len(f & set(int(v) for v in true_ids[i])) / K
    return out
