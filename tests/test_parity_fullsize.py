"""Parity at the benchmark's full size and launch: the sift-like 1M x 128
workload with all 10,000 queries in one call, in the two forms the benchmark
times (batched persistent BF16 + FP32 re-rank at L = 640, M = 32; plain FP32,
one CTA per query, at L = 160, M = 8), with the launch shape the library
chooses for that batch. The oracle recomputes a sample of the queries one by
one. The data are integers 0..255 in 128 dimensions, so every FP32 sum is
exact and BF16 holds every value: ids, keys, steps and expansions must equal
the oracle's bit for bit (the visited cache may forget, which only adds
distance evaluations)."""
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
