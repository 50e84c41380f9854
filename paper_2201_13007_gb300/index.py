"""Torch-tensor convenience over the C ABI: torch provides device memory and
the stream; every step of the search runs in libann's kernels."""
from __future__ import annotations

import numpy as np
import torch

from . import _abi


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes_void(s.cuda_stream)


def ctypes_void(v):
    import ctypes
    return ctypes.c_void_p(int(v))


def _ptr(t):
    return ctypes_void(t.data_ptr()) if t is not None else None


class Index:
    """A graph index on the current CUDA device (ann_index_create)."""

    def __init__(self, base, adj, entry, *, storage="f32", metric="l2", keep_f32=False):
        base_t = torch.as_tensor(base).to(torch.float32).contiguous()
        adj_t = torch.as_tensor(adj).to(torch.int32).contiguous()
        if base_t.dim() != 2 or adj_t.dim() != 2 or adj_t.shape[0] != base_t.shape[0]:
            raise ValueError("base must be n x d and adj n x R")
        flags = _abi.ANN_INDEX_KEEP_F32 if keep_f32 else 0
        if base_t.is_cuda != adj_t.is_cuda:
            base_t, adj_t = base_t.cuda(), adj_t.cuda()
        if base_t.is_cuda:
            flags |= _abi.ANN_INDEX_DEVICE_INPUT
        self.n, self.d = base_t.shape
        self.R = adj_t.shape[1]
        self.metric = metric
        self.storage = storage
        self._h = _abi.ann_index_create(_ptr(base_t), self.n, self.d, _abi.STORAGE[storage], _ptr(adj_t),
                                        self.R, int(entry), _abi.METRIC[metric], flags)

    @property
    def handle(self):
        return ctypes_void(self._h)

    def info(self):
        i = _abi.ann_index_get_info(self.handle)
        return {f: getattr(i, f) for f, _ in _abi.IndexInfo._fields_}

    def group_neighbors(self, hot_fraction, prefetch="block"):
        """Neighbour groups for the hottest vertices by in-degree
        (ann_index_group_neighbors); prefetch "block" or "rows"."""
        _abi.ann_index_group_neighbors(self.handle, hot_fraction, {"block": 0, "rows": 1}[prefetch])

    def close(self):
        if getattr(self, "_h", None):
            _abi.ann_index_destroy(self.handle)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def params(mode="sync", M0=1, t=1, R_ratio=0.8, rerank=False, threads=0, hash_bits=0,
               persistent=False, k_per_query=None, L_per_query=None, M_per_query=None, stats=None,
               order=None, cluster=0, phase_cycles=None, visited_mode=0,
               l2_prefetch=0, team_lanes=0, patience=None, gather=0):
        """patience=None: async walkers merge by Algorithm 2 (R_ratio); a number: by the stall count."""
        return _abi.SearchParams(mode=_abi.MODE[mode], M0=M0, t=t, R_ratio=R_ratio, rerank=int(rerank),
                                 threads=threads, hash_bits=hash_bits, persistent=int(persistent),
                                 k_per_query=_ptr(k_per_query), L_per_query=_ptr(L_per_query),
                                 M_per_query=_ptr(M_per_query), stats=_ptr(stats), order=_ptr(order),
                                 cluster=cluster, phase_cycles=_ptr(phase_cycles), visited_mode=visited_mode,
                                 l2_prefetch=l2_prefetch,
                                 team_lanes=team_lanes, merge_rule=0 if patience is None else 1,
                                 patience=0.0 if patience is None else float(patience), gather=gather)

    def describe(self, nq, k, L, M, **kw):
        """Launch configuration of a search with these arguments (ann_search_describe)."""
        return _abi.ann_search_describe(self.handle, nq, k, L, M, self.params(**kw))

    def search(self, queries, k, L, M, *, out=None, stream=None, with_stats=False, stats=None, **kw):
        """queries: CUDA float32 nq x d. Returns (ids int64, dists float32[, stats int64 nq x 8]).
        ``stats`` may be a preallocated CUDA int64 nq x 8 tensor for the per-query counters."""
        q = queries.contiguous()
        if not q.is_cuda or q.dtype != torch.float32 or q.dim() != 2 or q.shape[1] != self.d:
            raise ValueError("queries must be a CUDA float32 tensor of shape nq x d")
        nq = q.shape[0]
        if out is None:
            ids = torch.empty((nq, k), dtype=torch.int64, device=q.device)
            dists = torch.empty((nq, k), dtype=torch.float32, device=q.device)
        else:
            ids, dists = out
        if stats is None and with_stats:
            stats = torch.empty((nq, 8), dtype=torch.int64, device=q.device)
        p = self.params(stats=stats, **kw)
        _abi.ann_search_ex(self.handle, _ptr(q), nq, k, L, M, _ptr(ids), _ptr(dists), p,
                           _stream_handle(stream))
        return (ids, dists, stats) if with_stats else (ids, dists)

    def search_host(self, queries, k, L, M, *, out=None, stream=None, **kw):
        """Host-buffer search (ann_search_host): queries host float32 nq x d
        (numpy or a CPU tensor, ideally pinned); returns host ids / dists."""
        q = torch.as_tensor(queries)
        if q.is_cuda or q.dtype != torch.float32:
            raise ValueError("queries must be host float32")
        q = q.contiguous()
        nq = q.shape[0]
        if out is None:
            ids = torch.empty((nq, k), dtype=torch.int64)
            dists = torch.empty((nq, k), dtype=torch.float32)
        else:
            ids, dists = out
        p = self.params(**kw)
        _abi.ann_search_host(self.handle, _ptr(q), nq, k, L, M, _ptr(ids), _ptr(dists), p,
                             _stream_handle(stream))
        return ids, dists


class Batch:
    """A planned batch of queries with uneven k, L, M (ann_batch_create).
    k, L, M: host integer arrays; buckets: None or a list of
    (L_max, threads, hash_bits) tuples (e.g. from autotune.tune_buckets)."""

    def __init__(self, index, k, L, M, *, buckets=None, stats=None, **params):
        self.k = np.ascontiguousarray(k, np.int32)
        self.L = np.ascontiguousarray(L, np.int32)
        self.M = np.ascontiguousarray(M, np.int32)
        self.nq = self.k.shape[0]
        self.index = index
        nb = 0
        cfg = None
        if buckets:
            nb = len(buckets)
            cfg = (_abi.BucketConfig * nb)(*[_abi.BucketConfig(int(a), int(b), int(c)) for a, b, c in buckets])
        p = Index.params(stats=stats, **params)
        vp = lambda a: ctypes_void(a.ctypes.data)
        self._h = _abi.ann_batch_create(index.handle, self.nq, vp(self.k), vp(self.L), vp(self.M), cfg, nb, p)
        self.n_buckets, self.k_max = _abi.ann_batch_info(ctypes_void(self._h))

    def search(self, queries, out=None, stream=None):
        q = queries.contiguous()
        if out is None:
            ids = torch.empty((self.nq, self.k_max), dtype=torch.int64, device=q.device)
            dists = torch.empty((self.nq, self.k_max), dtype=torch.float32, device=q.device)
        else:
            ids, dists = out
        _abi.ann_batch_search(ctypes_void(self._h), _ptr(q), _ptr(ids), _ptr(dists), _stream_handle(stream))
        return ids, dists

    def close(self):
        if getattr(self, "_h", None):
            _abi.ann_batch_destroy(ctypes_void(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stats_dict(stats):
    s = stats.cpu().numpy() if isinstance(stats, torch.Tensor) else np.asarray(stats)
    return {f: s[:, i] for i, f in enumerate(_abi.STATS_FIELDS)}
