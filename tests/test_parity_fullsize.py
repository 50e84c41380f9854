"""Parity at the benchmark's full size and launch: the sift-like 1M x 128
workload with all 10,000 queries in one call, in the two forms the benchmark
times (batched persistent BF16 + FP32 re-rank at L = 640, M = 32; plain FP32,
one CTA per query, at L = 160, M = 8), with the launch shape the library
chooses for that batch. The oracle recomputes a sample of the queries one by
one. The data are integers 0..255 in 128 dimensions, so every FP32 sum is
exact and BF16 holds every value: ids, keys, steps and expansions must equal
the oracle's bit for bit (the visited cache may forget, which only adds
distance evaluations)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_13007_gb300 import synth  # noqa: E402
from parity_util import compare_exact  # noqa: E402

pytestmark = pytest.mark.gpu

SAMPLE = np.linspace(0, 9999, 64).astype(np.int64)


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_13007_gb300.index import Index, stats_dict
    w = synth.make_workload("sift", 1_000_000, 10_000)
    return w, Index, stats_dict


@pytest.mark.parametrize("form,L,M", [("batched_bf16_rerank", 640, 32), ("plain_f32", 160, 8)])
def test_full_size_sampled_queries_equal_the_oracle(full, oracle_mod, form, L, M):
    w, Index, stats_dict = full
    if form == "batched_bf16_rerank":
        ix = Index(w.base, w.adj, w.entry, storage="bf16", keep_f32=True)
        kw = dict(rerank=True, persistent=True)
    else:
        ix = Index(w.base, w.adj, w.entry, storage="f32")
        kw = {}
    q = torch.from_numpy(w.queries).cuda()
    ids, dists, st = ix.search(q, 10, L, M, with_stats=True, **kw)
    torch.cuda.synchronize()
    launch = ix.describe(q.shape[0], 10, L, M, **kw)
    ix.close()
    ids, dists, st = ids.cpu().numpy(), dists.cpu().numpy(), stats_dict(st.cpu().numpy())
    o_ids, o_keys, o_st = oracle_mod.search(w.base, w.adj, w.entry, w.queries[SAMPLE], algo="topm", L=L, K=10,
                                            M0=1, M_max=M, t=1, nthreads=8)
    compare_exact(ids[SAMPLE], dists[SAMPLE], o_ids, o_keys)
    np.testing.assert_array_equal(st["steps"][SAMPLE], o_st["steps"])
    np.testing.assert_array_equal(st["expansions"][SAMPLE], o_st["expansions"])
    assert (st["evals"][SAMPLE] >= o_st["evals"]).all()
    assert launch["grid"] >= 152, launch  # the whole GPU is in use, as in the benchmark


# ----------------------------------------------------------------- clusters

@pytest.fixture(scope="module")
def ix32(full):
    w, Index, _ = full
    ix = Index(w.base, w.adj, w.entry, storage="f32")
    yield ix
    ix.close()


_ORC = {}


def _oracle_sample(oracle_mod, w, L, M):
    if (L, M) not in _ORC:
        _ORC[(L, M)] = oracle_mod.search(w.base, w.adj, w.entry, w.queries[SAMPLE], algo="topm", L=L, K=10,
                                         M0=1, M_max=M, t=1, nthreads=8)
    return _ORC[(L, M)]


@pytest.mark.parametrize("C", [2, 4, 8])
@pytest.mark.parametrize("L,M", [(640, 32), (1024, 32)])
def test_cluster_at_full_size_equals_the_oracle(full, ix32, oracle_mod, C, L, M):
    """The clustered search on the 1M x 128 workload at the queue lengths and
    widths where clusters are used (L = 640 and 1024, M = 32), with the
    launch shape of the benchmark's one-query-per-launch form (the same
    threads, shared memory and visited table for 64 queries as for one):
    ids, keys, steps and expansions equal the oracle's bit for bit."""
    w, _, stats_dict = full
    one = ix32.describe(1, 10, L, M, cluster=C)
    many = ix32.describe(SAMPLE.size, 10, L, M, cluster=C)
    for f in ("threads", "smem_bytes", "hash_bits", "cluster", "visited_slot_bytes"):
        assert one[f] == many[f], (f, one, many)
    q = torch.from_numpy(w.queries[SAMPLE]).cuda()
    ids, d, st = ix32.search(q, 10, L, M, cluster=C, with_stats=True)
    torch.cuda.synchronize()
    o_ids, o_keys, o_st = _oracle_sample(oracle_mod, w, L, M)
    compare_exact(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_keys)
    s = stats_dict(st.cpu().numpy())
    np.testing.assert_array_equal(s["steps"], o_st["steps"])
    np.testing.assert_array_equal(s["expansions"], o_st["expansions"])
    assert (s["evals"] >= o_st["evals"]).all()


# ------------------------------------------------------------ async walkers

@pytest.fixture(scope="module")
def gt_full(full, oracle_mod):
    """Exact top-10 of all 10,000 queries (the oracle's FP64 GEMM form of
    Def. 1, exact on this integer data)."""
    w = full[0]
    return oracle_mod.exact_knn_gemm(w.base, w.queries, 10)[0]


@pytest.mark.parametrize("L,M,R", [(128, 4, 0.8), (512, 8, 0.8)])
def test_async_recall_at_full_size(full, gt_full, oracle_mod, L, M, R):
    """The asynchronous walkers (Algorithm 3 + Algorithm 2) at the points the
    benchmark times, in its launch (BF16 + FP32 re-rank, persistent grid) on
    the 1M x 128 workload, all 10,000 queries: recall@10 against the exact
    top-10 within 0.002 of the oracle's simulation of Algorithm 3 (BF16 holds
    these integers exactly, so the re-rank changes no key); every answer has
    distinct ids with exact keys in (key, id) order."""
    w, Index, stats_dict = full
    ix = Index(w.base, w.adj, w.entry, storage="bf16", keep_f32=True)
    q = torch.from_numpy(w.queries).cuda()
    ids, d, st = ix.search(q, 10, L, M, mode="async", R_ratio=R, rerank=True, persistent=True, with_stats=True)
    torch.cuda.synchronize()
    ix.close()
    ids, d = ids.cpu().numpy(), d.cpu().numpy()
    for i in range(0, ids.shape[0], 7):
        r = ids[i]
        assert len(set(r.tolist())) == r.size and (r >= 0).all()
        k64 = ((w.base[r].astype(np.float64) - w.queries[i].astype(np.float64)) ** 2).sum(1)
        np.testing.assert_array_equal(d[i].astype(np.float64), k64)
        assert (np.lexsort((r, k64)) == np.arange(r.size)).all()
    o_ids, _, o_st = oracle_mod.search(w.base, w.adj, w.entry, w.queries, algo="speedann", L=L, K=10, M0=1,
                                       M_max=M, R_ratio=R, nthreads=os.cpu_count() or 8)
    r_gpu = oracle_mod.recall(ids, gt_full).mean()
    r_orc = oracle_mod.recall(o_ids, gt_full).mean()
    print(f"async L={L} M={M} R={R}: recall GPU {r_gpu:.5f} oracle {r_orc:.5f} gap {r_gpu - r_orc:+.5f}")
    assert abs(r_gpu - r_orc) <= 0.002, (r_gpu, r_orc)
    assert (stats_dict(st.cpu().numpy())["merges"] >= 1).all()
