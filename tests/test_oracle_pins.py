"""Pins of the FP64 CPU oracle against things other than itself.

What pins what:
- hand-derived traces of Algorithm 1, top-M (Sec. 4.1-4.2) and Algorithm 3 on a
  tiny line graph (tests/golden/line_graph_traces.json);
- the exact K-NN (Def. 1) against scipy's cdist + a lexicographic sort, and a
  hand-derived tie case (tests/golden/ties_knn.json);
- exhaustive queue (L >= n, every vertex reachable): all three searches return
  the exact K-NN (every vertex is visited and nothing is truncated);
- BFiS is top-M with M = 1 (Sec. 4.1 states it);
- after every step the queue is the first min(L, |V|) of the visited set in
  (key, id) order, keys recomputed with scipy; the queue is sorted and
  duplicate-free and the L-th key never increases;
- the visited set is exactly {P} plus every neighbour of every expanded vertex,
  and the distance count equals |V|;
- each top-M step expands the first min(M_s, #unchecked) unchecked entries of
  the previous queue with M_s = min(M_max, M0 * 2^floor(s/t)) (Sec. 4.2);
- Algorithm 3 with R = 0 merges after every sub-step and reduces to top-M with
  t = 1; with one walker and no early merge (R = inf) it reduces to Algorithm 1.
"""
import json
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

from paper_2201_13007_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _keys(base, q, ids, metric="l2"):
    ids = np.asarray(ids, dtype=np.int64)
    if ids.size == 0:
        return np.zeros(0)
    x = base[ids].astype(np.float64)
    qq = np.asarray(q, np.float64).reshape(1, -1)
    if metric == "l2":
        return cdist(qq, x, "sqeuclidean")[0]
    return -(x @ qq[0])


def _lex(ids, keys):
    order = np.lexsort((ids, keys))
    return np.asarray(ids)[order], np.asarray(keys)[order]


# ----------------------------------------------------------------- golden

def test_golden_line_graph_traces(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "line_graph_traces.json")))
    base = np.array(g["base"], np.float32)
    adj = np.array(g["adj"], np.int32)
    q = np.array(g["query"], np.float32)
    for case in g["cases"]:
        kw = {k: case[k] for k in ("L", "K", "M0", "M_max", "t", "R_ratio", "patience") if k in case}
        tr = oracle_mod.search_trace(base, adj, g["entry"], q, algo=case["algo"], **kw)
        assert tr["ids"].tolist() == case["ids"], case["algo"]
        np.testing.assert_allclose(tr["keys"], case["keys"], rtol=1e-12)
        assert tr["expanded"].tolist() == case["expanded"], case["algo"]
        for f in ("steps", "evals", "expansions", "merges", "substeps"):
            if f in case:
                assert tr["stats"][f] == case[f], (case["algo"], f)
        if "final_queue" in case:
            assert tr["queue_ids"].tolist() == case["final_queue"]
        for s, want in enumerate(case.get("queue_after_each_step", []), start=1):
            trs = oracle_mod.search_trace(base, adj, g["entry"], q, algo=case["algo"], max_steps=s, **kw)
            assert trs["queue_ids"].tolist() == want, (case["algo"], s)


def test_golden_ties(oracle_mod):
    g = json.load(open(os.path.join(GOLD, "ties_knn.json")))
    ids, keys = oracle_mod.exact_knn(np.array(g["base"], np.float32), np.array(g["query"], np.float32), g["K"])
    assert ids[0].tolist() == g["ids"]
    np.testing.assert_array_equal(keys[0], g["keys"])


# ------------------------------------------------------------- exact k-NN

@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_exact_knn_matches_scipy(oracle_mod, metric):
    r = np.random.default_rng(5)
    base = r.standard_normal((300, 7)).astype(np.float32)
    base[10] = base[20]  # exact tie
    q = r.standard_normal((9, 7)).astype(np.float32)
    q[0] = base[10]
    K = 12
    ids, keys = oracle_mod.exact_knn(base, q, K, metric=metric, nthreads=3)
    if metric == "l2":
        D = cdist(q.astype(np.float64), base.astype(np.float64), "sqeuclidean")
    else:
        D = -(q.astype(np.float64) @ base.astype(np.float64).T)
    for i in range(q.shape[0]):
        order = np.lexsort((np.arange(base.shape[0]), D[i]))[:K]
        assert ids[i].tolist() == order.tolist()
        np.testing.assert_allclose(keys[i], D[i][order], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_exact_knn_gemm_equals_the_plain_sum_on_integer_data(oracle_mod, metric):
    """The GEMM form of Def. 1 is exact when the coordinates are integers
    (0..255 here, d = 128, with duplicated rows for exact ties): ids and keys
    equal the plain per-coordinate sum's bit for bit, ties included."""
    r = np.random.default_rng(6)
    base = r.integers(0, 256, (3000, 128)).astype(np.float32)
    base[100:140] = base[0:40]                       # exact key ties, broken by id
    q = r.integers(0, 256, (37, 128)).astype(np.float32)
    q[3] = base[5]
    ids, keys = oracle_mod.exact_knn(base, q, 15, metric=metric, nthreads=4)
    gi, gk = oracle_mod.exact_knn_gemm(base, q, 15, metric=metric, chunk=8)
    np.testing.assert_array_equal(gi, ids)
    np.testing.assert_array_equal(gk, keys)


def test_exact_knn_gemm_float_data_within_fp64_rounding(oracle_mod):
    r = np.random.default_rng(7)
    base = r.standard_normal((2000, 24)).astype(np.float32)
    q = r.standard_normal((20, 24)).astype(np.float32)
    ids, keys = oracle_mod.exact_knn(base, q, 10)
    gi, gk = oracle_mod.exact_knn_gemm(base, q, 10)
    np.testing.assert_array_equal(gi, ids)  # no near-ties at this size
    np.testing.assert_allclose(gk, keys, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_exact_knn_blocked_equals_the_plain_sum_on_integer_data(oracle_mod, metric):
    """The block-by-block form of Def. 1 on integer data (exact keys) equals
    the plain per-coordinate sum bit for bit, with blocks small enough that
    runs of tied keys straddle block cuts, query chunks that do not divide
    the query count, and a last block shorter than K."""
    r = np.random.default_rng(16)
    base = r.integers(0, 256, (1003, 96)).astype(np.float32)
    base[500:560] = base[10:70]                      # ties across blocks
    base[990:1003] = base[0]                         # a run of 13 equal rows, one split by a cut
    q = r.integers(0, 256, (23, 96)).astype(np.float32)
    q[2] = base[15]
    q[4] = base[0]
    ids, keys = oracle_mod.exact_knn(base, q, 20, metric=metric, nthreads=4)
    gi, gk = oracle_mod.exact_knn_blocked(base, q, 20, metric=metric, block=97, qchunk=5)
    np.testing.assert_array_equal(gi, ids)
    np.testing.assert_array_equal(gk, keys)


def test_exact_knn_blocked_float_data_and_padding(oracle_mod):
    r = np.random.default_rng(17)
    base = r.standard_normal((1500, 32)).astype(np.float32)
    q = r.standard_normal((9, 32)).astype(np.float32)
    ids, keys = oracle_mod.exact_knn(base, q, 12)
    gi, gk = oracle_mod.exact_knn_blocked(base, q, 12, block=256)
    np.testing.assert_array_equal(gi, ids)
    np.testing.assert_allclose(gk, keys, rtol=1e-12, atol=1e-12)
    small = base[:5]
    gi, gk = oracle_mod.exact_knn_blocked(small, q[:2], 8, block=2)
    ids, keys = oracle_mod.exact_knn(small, q[:2], 8)
    np.testing.assert_array_equal(gi, ids)
    assert np.isinf(gk[:, 5:]).all()


def test_exact_knn_pads_when_k_exceeds_n(oracle_mod):
    base = np.arange(3, dtype=np.float32).reshape(3, 1)
    ids, keys = oracle_mod.exact_knn(base, np.array([[0.2]], np.float32), 5)
    assert ids[0].tolist() == [0, 1, 2, -1, -1]
    assert np.isinf(keys[0, 3:]).all()


# --------------------------------------------------------- search invariants

ALGO_KW = [
    ("bfis", {}),
    ("topm", {"M0": 1, "M_max": 4, "t": 1}),
    ("topm", {"M0": 2, "M_max": 8, "t": 2}),
    ("speedann", {"M0": 1, "M_max": 4, "R_ratio": 0.8}),
    ("speedann", {"M0": 1, "M_max": 8, "R_ratio": float("inf")}),
]


@pytest.mark.parametrize("algo,kw", ALGO_KW)
@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_exhaustive_queue_returns_exact_knn(oracle_mod, algo, kw, metric):
    n = 120
    base, adj, q = synth.random_graph(n, 6, 5, seed=11, metric=metric, nq=6)
    adj[:, 0] = (np.arange(n) + 1) % n  # a ring makes every vertex reachable
    assert synth.reachable_from(adj, 0).all()
    K = 10
    ids, keys, st = oracle_mod.search(base, adj, 0, q, algo=algo, metric=metric, L=n, K=K, **kw)
    gt_ids, gt_keys = oracle_mod.exact_knn(base, q, K, metric=metric)
    np.testing.assert_array_equal(ids, gt_ids)
    np.testing.assert_allclose(keys, gt_keys, rtol=1e-12)
    assert (st["evals"] == n).all()


def test_bfis_is_topm_with_m1(oracle_mod):
    base, adj, q = synth.random_graph(400, 8, 6, seed=3, nq=20, pad_frac=0.2)
    for L in (1, 4, 16, 50):
        a = oracle_mod.search(base, adj, 0, q, algo="bfis", L=L, K=1)
        b = oracle_mod.search(base, adj, 0, q, algo="topm", L=L, K=1, M0=1, M_max=1)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])
        for f in ("steps", "evals", "expansions"):
            np.testing.assert_array_equal(a[2][f], b[2][f])


def _state_checks(oracle_mod, base, adj, entry, q, algo, L, kw):
    full = oracle_mod.search_trace(base, adj, entry, q, algo=algo, L=L, K=1, **kw)
    n_steps = full["stats"]["steps"]
    prev_lth = np.inf
    prev = None
    for s in range(0, n_steps + 1):
        tr = oracle_mod.search_trace(base, adj, entry, q, algo=algo, L=L, K=1, max_steps=s, **kw)
        V = tr["visited"]
        assert len(set(V.tolist())) == len(V)
        assert tr["stats"]["evals"] == len(V)
        # V = {P} + neighbours of every expanded vertex
        want = {entry}
        for v in tr["expanded"]:
            want.update(int(u) for u in adj[v] if u >= 0)
        assert set(V.tolist()) == want
        # queue = first min(L, |V|) of V in (key, id) order
        vk = _keys(base, q, V)
        sid, skey = _lex(V, vk)
        m = min(L, len(V))
        assert tr["queue_ids"].tolist() == sid[:m].tolist()
        np.testing.assert_allclose(tr["queue_keys"], skey[:m], rtol=1e-12, atol=1e-300)
        if m == L:
            assert skey[L - 1] <= prev_lth
            prev_lth = skey[L - 1]
        if algo == "topm" and prev is not None:
            # this step expanded the first M_s unchecked entries of the previous queue
            s0 = s - 1
            Ms = min(kw["M_max"], kw["M0"] * 2 ** (s0 // kw["t"]))
            unchecked = prev["queue_ids"][~prev["queue_checked"]]
            new_exp = tr["expanded"][len(prev["expanded"]):]
            assert new_exp.tolist() == unchecked[:Ms].tolist()
        prev = tr
    # converged: nothing unchecked remains
    assert full["queue_checked"].all()


@pytest.mark.parametrize("algo,kw", [
    ("bfis", {}),
    ("topm", {"M0": 1, "M_max": 4, "t": 1}),
    ("topm", {"M0": 1, "M_max": 3, "t": 2}),
    ("topm", {"M0": 2, "M_max": 16, "t": 1}),
])
@pytest.mark.parametrize("L", [1, 3, 8, 24])
def test_queue_is_top_l_of_visited_every_step(oracle_mod, algo, kw, L):
    base, adj, q = synth.random_graph(150, 5, 6, seed=L, nq=2, pad_frac=0.15, dup_frac=0.1)
    for qi in range(q.shape[0]):
        _state_checks(oracle_mod, base, adj, 7, q[qi], algo, L, kw)


def test_speedann_visited_and_sorted(oracle_mod):
    base, adj, q = synth.random_graph(300, 6, 8, seed=9, nq=10, pad_frac=0.1)
    for qi in range(q.shape[0]):
        tr = oracle_mod.search_trace(base, adj, 0, q[qi], algo="speedann", L=20, K=5, M0=1, M_max=8,
                                     R_ratio=0.9)
        V = tr["visited"]
        want = {0}
        for v in tr["expanded"]:
            want.update(int(u) for u in adj[v] if u >= 0)
        assert set(V.tolist()) == want
        assert tr["stats"]["evals"] == len(V)
        qk = tr["queue_keys"]
        assert (np.diff(qk) >= 0).all()
        assert len(set(tr["queue_ids"].tolist())) == len(qk)
        assert tr["queue_checked"].all()
        np.testing.assert_allclose(qk, _keys(base, q[qi], tr["queue_ids"]), rtol=1e-12)


@pytest.mark.parametrize("L,Mmax", [(1, 2), (5, 4), (16, 8), (40, 32)])
def test_speedann_r0_is_topm_t1(oracle_mod, L, Mmax):
    base, adj, q = synth.random_graph(500, 6, 8, seed=L + Mmax, nq=16, pad_frac=0.1)
    a = oracle_mod.search(base, adj, 0, q, algo="speedann", L=L, K=1, M0=1, M_max=Mmax, R_ratio=0.0)
    b = oracle_mod.search(base, adj, 0, q, algo="topm", L=L, K=1, M0=1, M_max=Mmax, t=1)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    for f in ("steps", "evals", "expansions"):
        np.testing.assert_array_equal(a[2][f], b[2][f])
    np.testing.assert_array_equal(a[2]["substeps"], a[2]["steps"])


@pytest.mark.parametrize("L,Mmax", [(8, 2), (16, 4), (40, 8)])
def test_stall_rule_limits(oracle_mod, L, Mmax):
    """Patience 0 merges at the checker's first expansion, as Algorithm 2 with
    R = 0 does (which is top-M with t = 1); an infinite patience never merges
    early, as R = infinity; with one walker, patience 1 is R = 1."""
    base, adj, q = synth.random_graph(300, 6, 5, seed=L + Mmax, nq=12)
    cases = [(0.0, 0.0, Mmax), (float("inf"), float("inf"), Mmax),
             # one walker: patience 1 merges at its first expansion since the deal that inserted nothing into
             # its top L, which is when its update position first reaches L, i.e. Algorithm 2 with R = 1
             (1.0, 1.0, 1)]
    for pat, R, Mw in cases:
        a = oracle_mod.search(base, adj, 0, q, algo="speedann", L=L, K=3, M0=1, M_max=Mw, patience=pat)
        b = oracle_mod.search(base, adj, 0, q, algo="speedann", L=L, K=3, M0=1, M_max=Mw, R_ratio=R)
        np.testing.assert_array_equal(a[0], b[0])
        for f in ("steps", "expansions", "evals", "merges", "substeps"):
            np.testing.assert_array_equal(a[2][f], b[2][f])


@pytest.mark.parametrize("L", [1, 6, 32])
def test_speedann_single_walker_nosync_is_bfis(oracle_mod, L):
    base, adj, q = synth.random_graph(500, 6, 8, seed=L, nq=16, pad_frac=0.1)
    a = oracle_mod.search(base, adj, 0, q, algo="speedann", L=L, K=1, M0=1, M_max=1,
                          R_ratio=float("inf"))
    b = oracle_mod.search(base, adj, 0, q, algo="bfis", L=L, K=1)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2]["evals"], b[2]["evals"])
    np.testing.assert_array_equal(a[2]["expansions"], b[2]["expansions"])


def test_padding_when_fewer_than_k_reachable(oracle_mod):
    base = np.arange(6, dtype=np.float32).reshape(6, 1)
    adj = np.array([[1, -1], [2, -1], [-1, -1], [4, 5], [5, -1], [3, -1]], np.int32)
    for algo, kw in ALGO_KW:
        ids, keys, st = oracle_mod.search(base, adj, 0, np.array([[0.0]], np.float32), algo=algo,
                                          L=8, K=5, **kw)
        assert ids[0].tolist() == [0, 1, 2, -1, -1]
        assert np.isinf(keys[0, 3:]).all()
        assert st["evals"][0] == 3


def test_rejects_invalid_input(oracle_mod):
    base = np.zeros((4, 2), np.float32)
    adj = np.array([[1], [2], [9], [0]], np.int32)  # 9 out of range
    with pytest.raises(ValueError):
        oracle_mod.search(base, adj, 0, np.zeros((1, 2), np.float32), algo="bfis", L=2, K=1)
    adj[2, 0] = 3
    with pytest.raises(ValueError):  # K > L
        oracle_mod.search(base, adj, 0, np.zeros((1, 2), np.float32), algo="bfis", L=2, K=3)
    with pytest.raises(ValueError):  # entry out of range
        oracle_mod.search(base, adj, 4, np.zeros((1, 2), np.float32), algo="bfis", L=2, K=1)


def test_threads_do_not_change_results(oracle_mod):
    base, adj, q = synth.random_graph(300, 6, 8, seed=1, nq=33)
    a = oracle_mod.search(base, adj, 0, q, algo="topm", L=16, K=4, M_max=4, nthreads=1)
    b = oracle_mod.search(base, adj, 0, q, algo="topm", L=16, K=4, M_max=4, nthreads=5)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[2], b[2])


def test_rerank_matches_sorted_fp32_keys(oracle_mod):
    r = np.random.default_rng(2)
    base = r.standard_normal((50, 4)).astype(np.float32)
    q = r.standard_normal((3, 4)).astype(np.float32)
    cand = np.array([[5, 9, 1, -1, 30], [0, 1, 2, 3, 4], [7, -1, -1, -1, -1]], np.int64)
    ids, keys = oracle_mod.rerank(base, q, cand, 3)
    for i in range(3):
        c = cand[i][cand[i] >= 0]
        k = _keys(base, q[i], c)
        sid, sk = _lex(c, k)
        want = list(sid[:3]) + [-1] * (3 - min(3, len(sid)))
        assert ids[i].tolist() == want
