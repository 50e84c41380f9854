"""Seeded synthetic workloads: base vectors, queries and the similarity graph.

This module builds the INPUTS of the search and nothing of the search itself:
Gaussian-mixture point sets shaped like the paper's datasets (Table 3: SIFT1M
128-d, GIST1M 960-d, DEEP 96-d) and a fixed-degree similarity graph over them.
Graph construction is not the paper's method (Sec. 2.2 takes a prebuilt NSG
index and says construction is not its focus), so the builder here is plain
index preparation: an exact k-NN list, an occlusion prune of the kind NSG uses,
reverse edges to fill the degree, and a reachability repair from the entry.

Both the CUDA path and the CPU oracle consume what this module returns; it
imports neither. Every random draw is a numpy PCG64 stream with a fixed seed.

Workload recipes (n x d, components, distribution):

- ``tiny``   10,000 x 32 float32, 16-component mixture, means U[-1,1]^32,
  isotropic sigma 0.15, equal weights; graph = exact 16-NN (L2, self
  excluded) + reverse edges by ascending distance, degree cap 24.
- ``sift``   n x 128 integer-valued (0..255) vectors: 64 components, means
  U[0,255]^128 * 0.5 + 64, sigma 60, rounded to nearest and clipped to
  [0, 255]; graph = occlusion prune to 32 of the union of each vertex's 64-NN
  and reverse 64-NN lists (first 128 by distance), then reverse fill to 32. (With
  sigma 30 the components are disjoint islands and no pruned k-NN graph over
  them is navigable: recall@10 stays below 0.75 at L = 256.)
- ``gist``   n x 960 non-negative: 32 components, x = exp(mu_c + 0.5 z),
  mu_c ~ N(-2, 0.5)^960; graph as ``sift``.
- ``deep``   n x 96 L2-normalised, low intrinsic dimension: a
  ``components``-component (128 by default) mixture in a 32-d latent space
  mapped to 96-d by a fixed random matrix, plus noise 0.1, normalised;
  inner-product search; graph built with L2 on the unit vectors (the same
  ordering as -IP). (An isotropic 96-d mixture is either islands (small
  sigma) or nearly uniform on the sphere (large sigma); neither is navigable
  like DEEP descriptors: recall@10 stays below 0.6 at L = 512.)

The entry point is the base point nearest (FP64 L2) to the mean of the base
set, ties to the smaller id (a cheap stand-in for the medoid).
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass, field

import numpy as np

_REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cache_dir() -> str:
    return os.environ.get("ANN_SYNTH_CACHE", os.path.join(_REPO, ".synth_cache"))


@dataclass
class Workload:
    name: str
    base: np.ndarray          # n x d float32
    queries: np.ndarray       # nq x d float32
    adj: np.ndarray           # n x R int32, -1 padded
    entry: int
    metric: str               # "l2" or "ip"
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.base.shape[0]

    @property
    def d(self):
        return self.base.shape[1]

    @property
    def R(self):
        return self.adj.shape[1]


# --------------------------------------------------------------- point sets

def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _labels(rng, count, C):
    return rng.integers(0, C, size=count)


def mixture_tiny(n, nq, d=32, C=16, sigma=0.15, seed=100):
    means = _rng(seed + 7).uniform(-1.0, 1.0, size=(C, d))
    def draw(count, s):
        r = _rng(s)
        lab = _labels(r, count, C)
        return (means[lab] + sigma * r.standard_normal((count, d))).astype(np.float32)
    return draw(n, seed + 1), draw(nq, seed + 2)


def mixture_sift(n, nq, d=128, C=64, sigma=60.0, seed=200):
    means = _rng(seed + 7).uniform(0.0, 255.0, size=(C, d)) * 0.5 + 64.0
    def draw(count, s):
        r = _rng(s)
        lab = _labels(r, count, C)
        out = np.empty((count, d), np.float32)
        step = 1 << 16
        for a in range(0, count, step):
            b = min(count, a + step)
            v = means[lab[a:b]] + sigma * r.standard_normal((b - a, d))
            out[a:b] = np.clip(np.rint(v), 0.0, 255.0)
        return out
    return draw(n, seed + 1), draw(nq, seed + 2)


def mixture_gist(n, nq, d=960, C=32, seed=300):
    mus = _rng(seed + 7).normal(-2.0, 0.5, size=(C, d))
    def draw(count, s):
        r = _rng(s)
        lab = _labels(r, count, C)
        out = np.empty((count, d), np.float32)
        step = 1 << 14
        for a in range(0, count, step):
            b = min(count, a + step)
            out[a:b] = np.exp(mus[lab[a:b]] + 0.5 * r.standard_normal((b - a, d)))
        return out
    return draw(n, seed + 1), draw(nq, seed + 2)


def mixture_deep(n, nq, d=96, C=128, r=32, spread=1.0, noise=0.1, seed=400):
    """Unit vectors with low intrinsic dimension: a C-component mixture in an
    r-dimensional latent space (means N(0, spread^2), unit spread around
    them), mapped to d dimensions by a fixed random matrix, plus isotropic
    noise, then L2-normalised."""
    g = _rng(seed + 7)
    means = g.standard_normal((C, r)) * spread
    A = g.standard_normal((d, r)) / np.sqrt(r)
    def draw(count, s):
        rr = _rng(s)
        lab = _labels(rr, count, C)
        out = np.empty((count, d), np.float32)
        step = 1 << 16
        for a in range(0, count, step):
            b = min(count, a + step)
            z = means[lab[a:b]] + rr.standard_normal((b - a, r))
            v = z @ A.T + noise * rr.standard_normal((b - a, d))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            out[a:b] = v
        return out
    return draw(n, seed + 1), draw(nq, seed + 2)


# ------------------------------------------------------------ graph builder

def _torch_device(device=None):
    import torch
    if device is not None:
        return torch.device(device)
    return torch.device("cuda") if torch.cuda.is_available() else torch.device("cpu")


def knn_lists(x: np.ndarray, k: int, exact64: bool = False, chunk_elems: int = 1 << 31):
    """k nearest other points of every point by L2 (self excluded), sorted by
    ascending distance. Returns (ids int32 n x k, squared distances float32).
    Chunked ||a||^2 + ||b||^2 - 2 a.b on whatever torch device is present;
    ``exact64`` computes in float64 (small sets)."""
    import torch
    dev = torch.device("cpu") if exact64 else _torch_device()
    dt = torch.float64 if exact64 else torch.float32
    n = x.shape[0]
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        X = torch.from_numpy(np.ascontiguousarray(x)).to(dev, dt)
        nrm = (X * X).sum(1)
        ids = torch.empty((n, k), dtype=torch.int32, device=dev)
        dst = torch.empty((n, k), dtype=torch.float32, device=dev)
        step = max(1, min(8192, chunk_elems // max(n, 1)))
        for a in range(0, n, step):
            b = min(n, a + step)
            D = nrm[a:b, None] + nrm[None, :] - 2.0 * (X[a:b] @ X.T)
            D.clamp_(min=0)
            D[torch.arange(b - a, device=dev), torch.arange(a, b, device=dev)] = float("inf")
            v, i = torch.topk(D, k, dim=1, largest=False, sorted=True)
            ids[a:b] = i.to(torch.int32)
            dst[a:b] = v.to(torch.float32)
            del D
        return ids.cpu().numpy(), dst.cpu().numpy()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def occlusion_prune(x: np.ndarray, cand: np.ndarray, cand_d: np.ndarray, R: int, batch: int = 16384):
    """NSG-style occlusion rule over each point's sorted candidate list: keep
    candidate c_j unless an already kept c_i is closer to c_j than the point
    itself is; stop at R kept. Returns int32 n x R, -1 padded."""
    import torch
    dev = _torch_device()
    n, k = cand.shape
    X = torch.from_numpy(np.ascontiguousarray(x)).to(dev, torch.float32)
    out = np.full((n, R), -1, np.int32)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for a in range(0, n, batch):
            b = min(n, a + batch)
            C = torch.from_numpy(cand[a:b].astype(np.int64)).to(dev)
            dpc = torch.from_numpy(cand_d[a:b]).to(dev)
            V = X[C]                                     # B x k x d
            nv = (V * V).sum(-1)                         # B x k
            D = nv[:, :, None] + nv[:, None, :] - 2.0 * torch.bmm(V, V.transpose(1, 2))
            kept = torch.zeros((b - a, k), dtype=torch.bool, device=dev)
            cnt = torch.zeros(b - a, dtype=torch.int32, device=dev)
            for j in range(k):
                occl = (kept & (D[:, :, j] < dpc[:, j:j + 1])).any(1)
                keep = (~occl) & (cnt < R)
                kept[:, j] = keep
                cnt += keep.to(torch.int32)
            # gather kept ids in order
            order = torch.where(kept, torch.arange(k, device=dev)[None, :].expand(b - a, k),
                                torch.full_like(C, k))
            order, _ = torch.sort(order, dim=1)
            order = order[:, :R]
            valid = order < k
            sel = torch.gather(C, 1, order.clamp(max=k - 1))
            sel = torch.where(valid, sel, torch.full_like(sel, -1))
            w = sel.shape[1]
            out[a:b, :w] = sel.cpu().numpy().astype(np.int32)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def _edge_dist(x, src, dst):
    out = np.empty(src.shape[0], np.float64)
    step = 1 << 20
    for a in range(0, src.shape[0], step):
        b = min(src.shape[0], a + step)
        diff = x[src[a:b]].astype(np.float64) - x[dst[a:b]].astype(np.float64)
        out[a:b] = np.einsum("ij,ij->i", diff, diff)
    return out


def reverse_fill(x: np.ndarray, fwd: np.ndarray, R: int) -> np.ndarray:
    """Widen a -1 padded forward list to R columns and fill free slots of
    each vertex c with reverse edges c -> p (for forward edges p -> c), by
    ascending distance, skipping ones already present."""
    n = fwd.shape[0]
    adj = np.full((n, R), -1, np.int32)
    w = min(R, fwd.shape[1])
    adj[:, :w] = fwd[:, :w]
    deg = (adj >= 0).sum(1).astype(np.int64)
    src = np.repeat(np.arange(n, dtype=np.int64), R)
    dst = adj.reshape(-1).astype(np.int64)
    m = dst >= 0
    src, dst = src[m], dst[m]
    fwd_keys = src * n + dst
    # candidate reverse edge: owner = dst, target = src
    owner, target = dst, src
    rev_keys = owner * n + target
    keep = ~np.isin(rev_keys, fwd_keys)
    owner, target = owner[keep], target[keep]
    dist = _edge_dist(x, owner, target)
    order = np.lexsort((target, dist, owner))
    owner, target = owner[order], target[order]
    first = np.searchsorted(owner, owner, side="left")
    rank = np.arange(owner.shape[0]) - first
    free = R - deg[owner]
    take = rank < free
    owner, target, rank = owner[take], target[take], rank[take]
    adj[owner, deg[owner] + rank] = target.astype(np.int32)
    return adj


def entry_point(x: np.ndarray) -> int:
    """Base point nearest (FP64 L2) to the mean of the base set; ties to the
    smaller id."""
    mean = x.astype(np.float64).mean(0)
    best, best_i = np.inf, 0
    step = 1 << 16
    for a in range(0, x.shape[0], step):
        b = min(x.shape[0], a + step)
        diff = x[a:b].astype(np.float64) - mean
        dd = np.einsum("ij,ij->i", diff, diff)
        i = int(np.argmin(dd))
        if dd[i] < best:
            best, best_i = float(dd[i]), a + i
    return best_i


def reachable_from(adj: np.ndarray, entry: int) -> np.ndarray:
    """Boolean mask of vertices reachable from ``entry`` along directed edges."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order
    n, R = adj.shape
    rows = np.repeat(np.arange(n), R)
    cols = adj.reshape(-1)
    m = cols >= 0
    g = sp.csr_matrix((np.ones(int(m.sum()), np.int8), (rows[m], cols[m])), shape=(n, n))
    order = breadth_first_order(g, entry, directed=True, return_predecessors=False)
    mask = np.zeros(n, bool)
    mask[order] = True
    return mask


def _nearest_among(x, targets, pool, device=None):
    """For each row index in ``targets``, the index in ``pool`` of the nearest
    point by L2 (chunked GEMM on the torch device, or on ``device``)."""
    import torch
    dev = _torch_device(device)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        T = torch.from_numpy(np.ascontiguousarray(x[targets])).to(dev, torch.float32)
        tn = (T * T).sum(1)
        best_d = torch.full((T.shape[0],), float("inf"), device=dev)
        best_i = torch.zeros(T.shape[0], dtype=torch.int64, device=dev)
        step = 1 << 18
        for a in range(0, pool.shape[0], step):
            P = torch.from_numpy(np.ascontiguousarray(x[pool[a:a + step]])).to(dev, torch.float32)
            D = tn[:, None] + (P * P).sum(1)[None, :] - 2.0 * (T @ P.T)
            v, i = D.min(1)
            upd = v < best_d
            best_d = torch.where(upd, v, best_d)
            best_i = torch.where(upd, i + a, best_i)
        return pool[best_i.cpu().numpy()]
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def repair_reachability(adj: np.ndarray, entry: int, knn: np.ndarray, x: np.ndarray,
                        max_rounds: int = 256, per_round: int = 1024, device=None, reach=None):
    """Make every vertex reachable from ``entry``. Each round finds the
    unreachable set by BFS and links up to ``per_round`` of its vertices
    (evenly spaced by id) from their nearest reachable vertex that still has
    room (a free slot, else one of its last slots; at most R/2 slots of a row
    are given to such links); a link makes the whole part of the graph behind
    that vertex reachable. ``device`` forces the torch device of the
    nearest-vertex search ("cpu" keeps the repair off the GPU); ``reach``
    replaces the BFS (same contract as reachable_from). Returns (adj, number
    of links added)."""
    adj = adj.copy()
    n, R = adj.shape
    protected = np.zeros((n, R), bool)
    added = 0
    for _ in range(max_rounds):
        mask = (reach or reachable_from)(adj, entry)
        un = np.flatnonzero(~mask)
        if un.size == 0:
            return adj, added
        pick = un[np.linspace(0, un.size - 1, min(per_round, un.size)).astype(np.int64)]
        pick = np.unique(pick)
        room = mask & (protected.sum(1) < max(1, R // 2))
        if not room.any():
            break
        src = _nearest_among(x, pick, np.flatnonzero(room), device)
        for s_, u in zip(src.tolist(), pick.tolist()):
            row = adj[s_]
            if u in row or protected[s_].sum() >= max(1, R // 2):
                continue
            free = np.flatnonzero(row < 0)
            if free.size:
                slot = int(free[0])
            else:
                slot = int(np.flatnonzero(~protected[s_])[-1])
            row[slot] = u
            protected[s_, slot] = True
            added += 1
    raise RuntimeError("graph repair did not converge")


# ---------------------------------------------------------------- builders

def build_knn_reverse_graph(x, k=16, cap=24):
    """Exact k-NN (FP64, L2, self excluded) then reverse edges to ``cap``."""
    ids, _ = knn_lists(x, k, exact64=True)
    return reverse_fill(x, ids, cap), ids


def union_candidates(ids: np.ndarray, dd: np.ndarray, cap: int):
    """Per vertex, the union of its k-NN list and of the vertices that list it
    (reverse k-NN), deduplicated, sorted by (distance, id) and cut to ``cap``.
    Returns (ids int32 n x cap, squared distances float32 n x cap; padding
    has distance +inf). Runs on the torch device."""
    import torch
    dev = _torch_device()
    n, k = ids.shape
    I = torch.from_numpy(ids.astype(np.int64)).to(dev)
    W = torch.from_numpy(dd.astype(np.float32)).to(dev)
    own = torch.arange(n, device=dev).repeat_interleave(k)
    c = I.reshape(-1)
    w = W.reshape(-1)
    o2 = torch.cat([own, c])
    c2 = torch.cat([c, own])
    w2 = torch.cat([w, w])
    del I, W, own, c, w
    # dedupe (owner, candidate) pairs
    key = o2 * n + c2
    key, order = torch.sort(key)
    w2 = w2[order]
    keep = torch.ones_like(key, dtype=torch.bool)
    keep[1:] = key[1:] != key[:-1]
    key, w2 = key[keep], w2[keep]
    o2 = key // n
    c2 = key % n
    # sort by (owner, distance, candidate): stable sorts from the last key to the first
    order = torch.argsort(w2, stable=True)          # (ties keep ascending candidate order from above)
    o2, c2, w2 = o2[order], c2[order], w2[order]
    order = torch.argsort(o2, stable=True)
    o2, c2, w2 = o2[order], c2[order], w2[order]
    counts = torch.bincount(o2, minlength=n)
    first = torch.cumsum(counts, 0) - counts
    rank = torch.arange(o2.shape[0], device=dev) - first[o2]
    m = rank < cap
    cand = torch.zeros((n, cap), dtype=torch.int32, device=dev)
    cdist = torch.full((n, cap), float("inf"), dtype=torch.float32, device=dev)
    cand[o2[m], rank[m]] = c2[m].to(torch.int32)
    cdist[o2[m], rank[m]] = w2[m]
    return cand.cpu().numpy(), cdist.cpu().numpy()


def build_pruned_graph(x, R=32, k=64, cap=128):
    """Occlusion prune (to R) of the union of forward and reverse k-NN
    candidates, then reverse fill to R."""
    ids, dd = knn_lists(x, k)
    cand, cdist = union_candidates(ids, dd, cap)
    pruned = occlusion_prune(x, cand, cdist, R)
    return reverse_fill(x, pruned, R), ids


def _key(d):
    return hashlib.sha1(json.dumps(d, sort_keys=True).encode()).hexdigest()[:16]


def _load_or_build(spec: dict, fn):
    cdir = _cache_dir()
    path = os.path.join(cdir, spec["kind"] + "_" + _key(spec) + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        return {k: z[k] for k in z.files}
    out = fn()
    os.makedirs(cdir, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, **out)
    os.replace(tmp, path)
    return out


def make_workload(kind: str, n: int, nq: int, *, d: int | None = None, R: int | None = None,
                  components: int | None = None, cache: bool = True) -> Workload:
    """Build (or load from the cache) a seeded workload of the given shape."""
    spec = {"kind": kind, "n": n, "nq": nq, "d": d, "R": R, "components": components, "v": 5}

    def gen():
        if kind == "tiny":
            base, q = mixture_tiny(n, nq, d=d or 32, C=components or 16)
            adj, knn = build_knn_reverse_graph(base, k=16, cap=R or 24)
        elif kind == "sift":
            base, q = mixture_sift(n, nq, d=d or 128, C=components or 64)
            adj, knn = build_pruned_graph(base, R=R or 32)
        elif kind == "gist":
            base, q = mixture_gist(n, nq, d=d or 960, C=components or 32)
            adj, knn = build_pruned_graph(base, R=R or 32)
        elif kind == "deep":
            base, q = mixture_deep(n, nq, d=d or 96, C=components or 128)
            adj, knn = build_pruned_graph(base, R=R or 32)
        else:
            raise ValueError(kind)
        entry = entry_point(base)
        adj, added = repair_reachability(adj, entry, knn, base)
        return {"base": base, "queries": q, "adj": adj, "entry": np.array(entry),
                "repaired": np.array(added)}

    z = _load_or_build(spec, gen) if cache else gen()
    metric = "ip" if kind == "deep" else "l2"
    return Workload(name=kind, base=z["base"], queries=z["queries"], adj=z["adj"],
                    entry=int(z["entry"]), metric=metric,
                    meta={"repaired_links": int(z["repaired"]), **spec})


def deep_bf16(n: int, nq: int, components: int = 256, cache: bool = True):
    """The serving point set: mixture_deep unit vectors (``components``
    mixture components) rounded to BF16, so that BF16 storage holds them
    exactly; queries stay FP32. No graph: large sets get theirs from the
    library's GPU builder. Returns (base n x d float32, queries nq x d
    float32)."""
    import torch
    spec = {"kind": "deep_bf16", "n": n, "nq": nq, "components": components, "v": 1}

    def gen():
        base, q = mixture_deep(n, nq, C=components)
        step = 1 << 20
        for a in range(0, n, step):
            blk = torch.from_numpy(base[a:a + step])
            base[a:a + step] = blk.to(torch.bfloat16).to(torch.float32).numpy()
        return {"base": base, "queries": q}

    z = _load_or_build(spec, gen) if cache else gen()
    return z["base"], z["queries"]


def graph_quality(adj: np.ndarray, entry: int, knn: np.ndarray | None = None, sample: int = 2000,
                  seed: int = 9) -> dict:
    """Structure of a fixed-degree graph, as input preparation reports it:
    out-degree and in-degree distributions, the share of vertices reachable
    from the entry, the share of directed edges whose reverse edge also
    exists, and, given the exact k-NN lists, how many of each sampled
    vertex's exact k nearest neighbours are its direct out-neighbours (the
    "k-NN coverage" of the pruned graph)."""
    n, R = adj.shape
    valid = adj >= 0
    outdeg = valid.sum(1)
    indeg = np.bincount(adj[valid].ravel(), minlength=n)
    reach = reachable_from(adj, entry)
    r = _rng(seed)
    src = r.choice(n, size=min(sample, n), replace=False)
    back = 0
    edges = 0
    for v in src:
        for u in adj[v][adj[v] >= 0]:
            edges += 1
            back += int(v in adj[u])
    out = {"n": int(n), "R": int(R),
           "out_degree": {"mean": float(outdeg.mean()), "min": int(outdeg.min()), "max": int(outdeg.max()),
                          "full_rows": float((outdeg == R).mean())},
           "in_degree": {"mean": float(indeg.mean()), "max": int(indeg.max()),
                         "p99": float(np.percentile(indeg, 99)), "zero": float((indeg == 0).mean())},
           "reachable_from_entry": float(reach.mean()),
           "reciprocal_edges": back / max(edges, 1)}
    if knn is not None:
        k = knn.shape[1]
        cov = [len(set(knn[v].tolist()) & set(adj[v][adj[v] >= 0].tolist())) / k for v in src]
        out[f"exact_{k}nn_in_out_edges"] = float(np.mean(cov))
    return out


def random_graph(n, d, R, seed, metric="l2", nq=8, pad_frac=0.0, dup_frac=0.0):
    """Small adversarial inputs for tests: uniform random points, R random
    out-edges per vertex (with optional -1 padding and duplicated vectors)."""
    r = _rng(seed)
    base = r.standard_normal((n, d)).astype(np.float32)
    if dup_frac > 0:
        k = int(n * dup_frac)
        src = r.integers(0, n, size=k)
        dst = r.integers(0, n, size=k)
        base[dst] = base[src]
    adj = np.empty((n, R), np.int32)
    for i in range(n):
        adj[i] = r.choice(np.delete(np.arange(n), i), size=R, replace=R > n - 1)
    if pad_frac > 0:
        adj[r.random((n, R)) < pad_frac] = -1
    if metric == "ip":
        base /= np.linalg.norm(base, axis=1, keepdims=True)
    q = r.standard_normal((nq, d)).astype(np.float32)
    if metric == "ip":
        q /= np.linalg.norm(q, axis=1, keepdims=True)
    return base, adj, q
