"""Planned batches of queries with uneven k, L, M (ann_batch_*): per-query
results, CUDA-graph capture and the autotuner."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_13007_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_13007_gb300.index import Batch, Index
    w = synth.make_workload("deep", 20000, 1000, components=32)
    ix = Index(w.base, w.adj, w.entry, metric="ip")
    g = np.random.default_rng(11)
    nq = w.queries.shape[0]
    k = g.choice([1, 10, 100], nq).astype(np.int32)
    L = np.maximum(k, g.choice([32, 64, 128, 256, 512, 1024], nq)).astype(np.int32)
    M = g.choice([1, 2, 4, 8, 16, 32], nq).astype(np.int32)
    yield ix, Batch, w, k, L, M
    ix.close()


def _check_rows(ix, q, ids, dists, k, L, M, rows):
    for i in rows:
        a, b = ix.search(q[i:i + 1], int(k[i]), int(L[i]), int(M[i]))
        assert torch.equal(ids[i, :k[i]], a[0]) and torch.equal(dists[i, :k[i]], b[0]), i
        assert (ids[i, k[i]:] == -1).all()


def test_batch_rows_equal_single_searches(setup):
    ix, Batch, w, k, L, M = setup
    q = torch.from_numpy(w.queries).cuda()
    b = Batch(ix, k, L, M)
    assert b.n_buckets >= 5 and b.k_max == 100
    ids, dists = b.search(q)
    torch.cuda.synchronize()
    _check_rows(ix, q, ids, dists, k, L, M, range(0, q.shape[0], 3))
    b.close()


def test_batch_rows_equal_the_oracle(oracle_mod):
    """A planned batch on integer-valued data (1..255 values, d = 128: every
    FP32 sum is exact) with uneven k, L, M: every row's ids and keys equal
    the oracle's top-M search of that query with its own k, L, M bit for
    bit, and so do its steps and expansions (the forgetful visited cache can
    only add distance evaluations)."""
    from paper_2201_13007_gb300.index import Batch, Index, stats_dict
    from parity_util import oracle_rows
    w = synth.make_workload("sift", 20000, 600)
    ix = Index(w.base, w.adj, w.entry, storage="bf16", keep_f32=True)
    g = np.random.default_rng(12)
    nq = w.queries.shape[0]
    k = g.choice([1, 10, 100], nq).astype(np.int32)
    L = np.maximum(k, g.choice([32, 64, 128, 256, 512], nq)).astype(np.int32)
    M = g.choice([1, 2, 4, 8, 16, 32], nq).astype(np.int32)
    st = torch.empty((nq, 8), dtype=torch.int64, device="cuda")
    b = Batch(ix, k, L, M, stats=st, rerank=True)
    ids, dists = b.search(torch.from_numpy(w.queries).cuda())
    torch.cuda.synchronize()
    ids, dists, s = ids.cpu().numpy(), dists.cpu().numpy(), stats_dict(st)
    o_ids, o_keys, o_steps, o_exps, o_evals = oracle_rows(oracle_mod, w.base, w.adj, w.entry, w.queries, k, L, M)
    for i in range(nq):
        np.testing.assert_array_equal(ids[i, :k[i]], o_ids[i], err_msg=f"row {i}")
        np.testing.assert_array_equal(dists[i, :k[i]].astype(np.float64), o_keys[i], err_msg=f"row {i}")
        assert (ids[i, k[i]:] == -1).all()
    np.testing.assert_array_equal(s["steps"], o_steps)
    np.testing.assert_array_equal(s["expansions"], o_exps)
    assert (s["evals"] >= o_evals).all()
    b.close()
    ix.close()


def test_batch_under_cuda_graph_capture(setup):
    ix, Batch, w, k, L, M = setup
    q = torch.from_numpy(w.queries).cuda()
    b = Batch(ix, k, L, M)
    ref = b.search(q)
    torch.cuda.synchronize()
    ids = torch.full_like(ref[0], -5)
    dists = torch.zeros_like(ref[1])
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside capture on the capture stream
        b.search(q, out=(ids, dists), stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    ids.fill_(-5)
    with torch.cuda.graph(g):
        b.search(q, out=(ids, dists))
    for _ in range(3):
        ids.fill_(-5)
        dists.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(ids, ref[0]) and torch.equal(dists, ref[1])
    b.close()


def test_autotuned_buckets_same_answers(setup, tmp_path):
    ix, Batch, w, k, L, M = setup
    from paper_2201_13007_gb300 import autotune
    q = torch.from_numpy(w.queries).cuda()
    cache = str(tmp_path / "tune.json")
    cfg = autotune.tune_buckets(ix, q, k, L, M, sample=200, reps=1, cache_path=cache)
    assert len(cfg) == len(autotune.LADDER)
    assert autotune.tune_buckets(ix, q, k, L, M, sample=200, reps=1, cache_path=cache) == cfg  # cached
    ref = Batch(ix, k, L, M).search(q)
    got = Batch(ix, k, L, M, buckets=cfg).search(q)
    torch.cuda.synchronize()
    assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])


def test_work_list_runs_only_listed_queries(setup):
    ix, Batch, w, k, L, M = setup
    q = torch.from_numpy(w.queries).cuda()
    order = torch.tensor([5, 3, 900, 17], dtype=torch.int32, device="cuda")
    ids = torch.full((q.shape[0], 10), -7, dtype=torch.int64, device="cuda")
    dists = torch.zeros((q.shape[0], 10), device="cuda")
    from paper_2201_13007_gb300 import _abi
    from paper_2201_13007_gb300.index import _ptr, _stream_handle
    p = ix.params(order=order, persistent=True)
    _abi.ann_search_ex(ix.handle, _ptr(q), 4, 10, 64, 4, _ptr(ids), _ptr(dists), p, _stream_handle(None))
    torch.cuda.synchronize()
    ref = ix.search(q, 10, 64, 4)
    for r in (5, 3, 900, 17):
        assert torch.equal(ids[r], ref[0][r])
    untouched = torch.ones(q.shape[0], dtype=torch.bool)
    untouched[[5, 3, 900, 17]] = False
    assert (ids[untouched.cuda()] == -7).all()
