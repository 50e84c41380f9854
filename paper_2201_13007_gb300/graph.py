"""Similarity-graph construction on the GPU for base sets too large for a
materialised distance matrix (10M points and up).

The search takes its graph as given (Sec. 2.2 builds on proximity graphs
such as NSG). This builder produces the same kind of graph as the smaller
workloads use: the exact k nearest neighbours of every point (Def. 1, here
by the library's brute-force tensor-core kernel ``ann_knn_bf16`` over BF16
rows), united with the reverse k-NN edges, cut by the NSG-style occlusion
rule to degree R, widened with reverse edges, and repaired so that every
vertex is reachable from the entry vertex (the medoid). Every step after
the k-NN kernel is plain torch on the device.
"""
from __future__ import annotations

import numpy as np

from . import _abi


def knn_bf16(xb, k: int = 64, metric: str = "l2", chunk: int = 1 << 20):
    """Exact k nearest other rows of every row of ``xb`` ((n, d) torch
    bfloat16 CUDA tensor, d in {32, 64, 96, 128}); ties by id. Returns
    (ids int32 (n, k), keys float32 (n, k)) on the device: squared l2 or
    -<q, x>, products exact in FP32, sums in FP32."""
    import torch
    xb = xb.contiguous()
    n, d = xb.shape
    bits = xb.view(torch.int16)
    ids = torch.empty((n, k), dtype=torch.int32, device=xb.device)
    keys = torch.empty((n, k), dtype=torch.float32, device=xb.device)
    stream = torch.cuda.current_stream().cuda_stream
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        _abi.ann_knn_bf16(bits.data_ptr(), n, d, bits[a:b].data_ptr(), b - a, a, 0 if metric == "l2" else 1, k,
                          ids[a:b].data_ptr(), keys[a:b].data_ptr(), stream)
    return ids, keys


def union_candidates(ids, keys, cap: int):
    """Per vertex, its k-NN list united with the vertices that list it,
    deduplicated, ordered by (distance, id) and cut to ``cap``. Device
    tensors in and out: (cand int64 (n, cap), dist float32 (n, cap)); empty
    slots hold id 0 at distance +inf."""
    import torch
    n, k = ids.shape
    dev = ids.device
    own = torch.arange(n, device=dev).repeat_interleave(k)
    c = ids.reshape(-1).long()
    w = keys.reshape(-1)
    o2 = torch.cat([own, c])
    c2 = torch.cat([c, own])
    w2 = torch.cat([w, w])
    del own, c, w
    key = o2 * n + c2
    del o2, c2
    key, order = torch.sort(key)
    w2 = w2[order]
    del order
    keep = torch.ones_like(key, dtype=torch.bool)
    keep[1:] = key[1:] != key[:-1]
    key, w2 = key[keep], w2[keep]
    del keep
    # (owner, distance, candidate): stable sorts from the last key to the first
    order = torch.argsort(w2, stable=True)
    key, w2 = key[order], w2[order]
    o2 = key // n
    order = torch.argsort(o2, stable=True)
    key, w2, o2 = key[order], w2[order], o2[order]
    del order
    c2 = key % n
    del key
    counts = torch.bincount(o2, minlength=n)
    first = torch.cumsum(counts, 0) - counts
    rank = torch.arange(o2.shape[0], device=dev) - first[o2]
    if o2.numel() and int(rank.min()) < 0:
        raise RuntimeError("union_candidates: owners not grouped")
    m = rank < cap
    cand = torch.zeros((n, cap), dtype=torch.int64, device=dev)
    cdist = torch.full((n, cap), float("inf"), dtype=torch.float32, device=dev)
    cand[o2[m], rank[m]] = c2[m]
    cdist[o2[m], rank[m]] = w2[m]
    return cand, cdist


def occlusion_prune(X, cand, cdist, R: int, batch: int = 1 << 17):
    """NSG occlusion rule over each sorted candidate list: keep candidate c_j
    unless a kept c_i is closer to c_j than the vertex is; stop at R kept.
    X is the (n, d) FP32 device tensor. Returns int32 (n, R), -1 padded."""
    import torch
    n, k = cand.shape
    dev = X.device
    out = torch.full((n, R), -1, dtype=torch.int32, device=dev)
    ar = torch.arange(k, device=dev)
    for a in range(0, n, batch):
        b = min(n, a + batch)
        C = cand[a:b]
        dpc = cdist[a:b]
        V = X[C]
        nv = (V * V).sum(-1)
        D = nv[:, :, None] + nv[:, None, :] - 2.0 * torch.bmm(V, V.transpose(1, 2))
        del V
        kept = torch.zeros((b - a, k), dtype=torch.bool, device=dev)
        cnt = torch.zeros(b - a, dtype=torch.int32, device=dev)
        for j in range(k):
            occl = (kept & (D[:, :, j] < dpc[:, j:j + 1])).any(1)
            keep = (~occl) & (cnt < R) & torch.isfinite(dpc[:, j])
            kept[:, j] = keep
            cnt += keep.to(torch.int32)
        del D
        order = torch.where(kept, ar[None, :].expand(b - a, k), torch.full_like(C, k))
        order, _ = torch.sort(order, dim=1)
        order = order[:, :R]
        valid = order < k
        sel = torch.gather(C, 1, order.clamp(max=k - 1))
        out[a:b] = torch.where(valid, sel, torch.full_like(sel, -1)).to(torch.int32)
    return out


def reverse_fill(X, fwd, R: int, chunk: int = 1 << 22):
    """Fill the free slots of each vertex c with reverse edges c -> p (for
    forward edges p -> c) by ascending FP64 distance, then id, skipping ones
    already present. Device tensors; returns int32 (n, R)."""
    import torch
    n = fwd.shape[0]
    dev = fwd.device
    adj = torch.full((n, R), -1, dtype=torch.int32, device=dev)
    w = min(R, fwd.shape[1])
    adj[:, :w] = fwd[:, :w]
    deg = (adj >= 0).sum(1).long()
    src = torch.arange(n, device=dev).repeat_interleave(R)
    dst = adj.reshape(-1).long()
    m = dst >= 0
    src, dst = src[m], dst[m]
    fwd_keys = src * n + dst
    owner, target = dst, src
    keep = ~torch.isin(owner * n + target, fwd_keys)
    del fwd_keys
    owner, target = owner[keep], target[keep]
    dist = torch.empty(owner.shape[0], dtype=torch.float64, device=dev)
    for a in range(0, owner.shape[0], chunk):
        b = min(owner.shape[0], a + chunk)
        diff = X[owner[a:b]].double() - X[target[a:b]].double()
        dist[a:b] = (diff * diff).sum(1)
    # lexicographic (owner, dist, target): stable sorts from the last key to the first
    order = torch.argsort(target, stable=True)
    owner, target, dist = owner[order], target[order], dist[order]
    order = torch.argsort(dist, stable=True)
    owner, target, dist = owner[order], target[order], dist[order]
    order = torch.argsort(owner, stable=True)
    owner, target, dist = owner[order], target[order], dist[order]
    del order
    first = torch.searchsorted(owner, owner, side="left")
    rank = torch.arange(owner.shape[0], device=dev) - first
    if owner.numel() and int(rank.min()) < 0:
        raise RuntimeError("reverse_fill: owners not grouped")
    free = R - deg[owner]
    take = rank < free
    owner, target, rank = owner[take], target[take], rank[take]
    adj[owner, deg[owner] + rank] = target.to(torch.int32)
    return adj


def reachable(adj, entry: int):
    """Vertices reachable from ``entry`` (frontier BFS on the device); adj
    is an (n, R) int32 array or device tensor. Returns a numpy bool mask."""
    import torch
    if isinstance(adj, torch.Tensor):
        A = adj
    else:
        A = torch.from_numpy(np.ascontiguousarray(adj))
        if torch.cuda.is_available():
            A = A.cuda()
    n = A.shape[0]
    seen = torch.zeros(n, dtype=torch.bool, device=A.device)
    seen[entry] = True
    frontier = torch.tensor([entry], dtype=torch.int64, device=A.device)
    while frontier.numel():
        nb = A[frontier].reshape(-1).long()
        nb = nb[nb >= 0]
        nb = torch.unique(nb[~seen[nb]])
        seen[nb] = True
        frontier = nb
    return seen.cpu().numpy()


def medoid(X) -> int:
    """Base point nearest (FP64 l2) to the mean of the base set; ties to the
    smaller id."""
    import torch
    mean = X.double().mean(0)
    best, best_i = float("inf"), 0
    for a in range(0, X.shape[0], 1 << 20):
        diff = X[a:a + (1 << 20)].double() - mean
        dd = (diff * diff).sum(1)
        i = int(torch.argmin(dd))
        if float(dd[i]) < best:
            best, best_i = float(dd[i]), a + i
    return best_i


def build(base: np.ndarray, R: int = 32, k: int = 64, cap: int = 128, log=None):
    """Graph over ``base`` (n x d float32 whose values are BF16-representable,
    d in {32, 64, 96, 128}): returns (adj int32 n x R, entry, repaired links,
    the k-NN ids (n x k int32 numpy) and seconds per stage)."""
    import time
    import torch
    from . import synth
    t = {}
    t0 = time.perf_counter()
    X = torch.from_numpy(np.ascontiguousarray(base, np.float32)).cuda()
    xb = X.to(torch.bfloat16)
    if not torch.equal(xb.float(), X):
        raise ValueError("base values must be BF16-representable")
    ids, keys = knn_bf16(xb, k)
    torch.cuda.synchronize()
    if int(ids.min()) < 0 or int(ids.max()) >= X.shape[0]:
        raise RuntimeError("k-NN lists hold ids outside the base set")
    t["knn"] = time.perf_counter() - t0
    del xb
    if log:
        log(f"graph: k-NN of {X.shape[0]} rows in {t['knn']:.1f}s")
    t0 = time.perf_counter()
    cand, cdist = union_candidates(ids, keys, cap)
    knn_np = ids.cpu().numpy()
    del ids, keys
    pruned = occlusion_prune(X, cand, cdist, R)
    del cand, cdist
    adj = reverse_fill(X, pruned, R)
    del pruned
    entry = medoid(X)
    torch.cuda.synchronize()
    t["prune"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    adj_np = adj.cpu().numpy()
    del adj
    adj_np, added = synth.repair_reachability(adj_np, entry, None, base, reach=reachable)
    t["repair"] = time.perf_counter() - t0
    if log:
        log(f"graph: prune {t['prune']:.1f}s, repair {t['repair']:.1f}s ({added} links)")
    return adj_np, entry, added, knn_np, t
