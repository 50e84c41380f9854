"""The clustered search (one query over a thread-block cluster sharing its
step work through distributed shared memory) against the one-CTA kernel and
the FP64 oracle: identical ids and keys."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_13007_gb300 import synth  # noqa: E402
from parity_util import compare_exact  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_13007_gb300.index import Index
    w = synth.make_workload("sift", 20000, 64)
    return Index, w


@pytest.mark.parametrize("C", [2, 4, 8])
@pytest.mark.parametrize("L,M", [(16, 1), (64, 4), (200, 16), (128, 32)])
def test_cluster_equals_single_cta_and_oracle(env, oracle_mod, C, L, M):
    Index, w = env
    ix = Index(w.base, w.adj, w.entry)
    q = torch.from_numpy(w.queries).cuda()
    a_ids, a_d, a_st = ix.search(q, 10, L, M, hash_bits=15, visited_mode=1, with_stats=True)
    b_ids, b_d, b_st = ix.search(q, 10, L, M, hash_bits=15, cluster=C, with_stats=True)
    torch.cuda.synchronize()
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d)
    # same trajectory: same steps and the same number of distance evaluations
    assert torch.equal(a_st[:, 0], b_st[:, 0]) and torch.equal(a_st[:, 2], b_st[:, 2])
    o_ids, o_keys, _ = oracle_mod.search(w.base, w.adj, w.entry, w.queries, algo="topm", L=L, K=10, M0=1,
                                         M_max=M, t=1, nthreads=8)
    compare_exact(b_ids.cpu().numpy(), b_d.cpu().numpy(), o_ids, o_keys)
    ix.close()


@pytest.mark.parametrize("C", [2, 8])
def test_cluster_with_forgetful_tables_rerank_and_work_list(env, oracle_mod, C):
    Index, w = env
    ix = Index(w.base, w.adj, w.entry, storage="bf16", keep_f32=True)
    q = torch.from_numpy(w.queries).cuda()
    ref = ix.search(q, 10, 128, 8, rerank=True)
    got = ix.search(q, 10, 128, 8, rerank=True, cluster=C, hash_bits=8)  # many resets per CTA
    torch.cuda.synchronize()
    assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])
    # per-query k / L / M and a work list
    g = np.random.default_rng(3)
    nq = q.shape[0]
    ks = torch.from_numpy(g.choice([1, 5, 10], nq).astype(np.int32)).cuda()
    Ls = torch.from_numpy(np.maximum(ks.cpu().numpy(), g.choice([16, 64, 128], nq)).astype(np.int32)).cuda()
    Ms = torch.from_numpy(g.choice([1, 4, 8], nq).astype(np.int32)).cuda()
    order = torch.arange(nq - 1, -1, -2, dtype=torch.int32, device="cuda")
    ids = torch.full((nq, 10), -9, dtype=torch.int64, device="cuda")
    d = torch.zeros((nq, 10), device="cuda")
    from paper_2201_13007_gb300 import _abi
    from paper_2201_13007_gb300.index import _ptr, _stream_handle
    p = ix.params(k_per_query=ks, L_per_query=Ls, M_per_query=Ms, order=order, cluster=C)
    _abi.ann_search_ex(ix.handle, _ptr(q), order.numel(), 10, 128, 8, _ptr(ids), _ptr(d), p, _stream_handle(None))
    torch.cuda.synchronize()
    for i in order.cpu().numpy():
        a, b = ix.search(q[i:i + 1], int(ks[i]), int(Ls[i]), int(Ms[i]))
        assert torch.equal(ids[i, :ks[i]], a[0]) and torch.equal(d[i, :ks[i]], b[0])
    assert (ids[0::2] == -9).all() if nq % 2 == 0 else True
    ix.close()


def test_cluster_inner_product(env, oracle_mod):
    Index, _ = env
    w = synth.make_workload("deep", 20000, 64, components=32)
    ix = Index(w.base, w.adj, w.entry, metric="ip")
    q = torch.from_numpy(w.queries).cuda()
    a = ix.search(q, 10, 96, 8)
    b = ix.search(q, 10, 96, 8, cluster=4)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    ix.close()
