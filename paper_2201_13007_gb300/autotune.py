"""Autotuner for planned batches: per L bucket, the block size and visited
table size that run that bucket fastest on this GPU.

For every bucket of the L ladder that the batch uses, a sample of its
queries (up to ``sample``) is planned alone with each candidate
(threads, hash_bits), timed with CUDA events after a warm-up, and the fastest
candidate kept. Results are cached in a JSON file keyed by the index shape,
storage, metric, search params and the sample's k / L / M mix. The tuner only
chooses launch configurations; every search it times is the library's.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from .index import Batch

LADDER = (32, 64, 128, 256, 512, 1024, 2048)
# (threads, hash_bits); (0, 0) is the library's own choice for the bucket, so the tuner never does worse than it
CANDIDATES = ((0, 0), (128, 11), (128, 12), (128, 14), (256, 12), (256, 13), (256, 14), (512, 13), (512, 14))


def _key(index, k, L, M, params, ladder):
    h = hashlib.sha1()
    info = index.info()
    h.update(json.dumps([info["n"], info["d"], info["R"], info["storage"], info["metric"], sorted(params.items()),
                         list(ladder)], default=str).encode())
    for a in (k, L, M):
        h.update(np.bincount(np.asarray(a, np.int64)).tobytes())
    return h.hexdigest()[:16]


def tune_buckets(index, queries, k, L, M, *, ladder=LADDER, candidates=CANDIDATES, sample=2000, reps=3,
                 cache_path=None, **params):
    """Returns a list of (L_max, threads, hash_bits), one per ladder rung (0 = the library's choice)."""
    k = np.asarray(k, np.int32)
    L = np.asarray(L, np.int32)
    M = np.asarray(M, np.int32)
    key = _key(index, k, L, M, params, ladder)
    if cache_path and os.path.exists(cache_path):
        cache = json.load(open(cache_path))
        if key in cache:
            return [tuple(v) for v in cache[key]]
    out = []
    lo = 0
    for hi in ladder:
        sel = np.flatnonzero((L > lo) & (L <= hi))
        lo = hi
        if sel.size == 0:
            out.append((hi, 0, 0))
            continue
        sel = sel[np.linspace(0, sel.size - 1, min(sample, sel.size)).astype(np.int64)]
        qs = queries[torch.from_numpy(sel).to(queries.device)].contiguous()
        best = None
        for th, hb in candidates:
            try:
                b = Batch(index, k[sel], L[sel], M[sel], buckets=[(hi, th, hb)], **params)
            except Exception:
                continue
            ids, d = b.search(qs)
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                b.search(qs, out=(ids, d))
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            b.close()
            t = min(ts)
            if best is None or t < best[0]:
                best = (t, th, hb)
        out.append((hi, best[1], best[2]) if best else (hi, 0, 0))
    if cache_path:
        cache = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
        cache[key] = out
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        json.dump(cache, open(cache_path, "w"), indent=1)
    return out
