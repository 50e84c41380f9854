"""Neighbour grouping (Sec. 4.4, degree-centric): the hottest vertices by
in-degree get a contiguous copy of their neighbours' rows, and the one-CTA
sync kernel reads a hot vertex's fresh neighbours from that block. The copies
hold the same values, so every answer, step and distance count must equal
the ungrouped index's, and on integer-valued data the oracle's bit for bit."""
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
    from paper_2201_13007_gb300.index import Index, stats_dict
    from paper_2201_13007_gb300 import _abi
    w = synth.make_workload("sift", 20000, 300)
    return Index, stats_dict, _abi, w


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("frac,prefetch", [(0.01, "block"), (0.05, "block"), (0.05, "rows")])
@pytest.mark.parametrize("L,M", [(64, 4), (200, 16), (128, 32)])
def test_grouped_index_equals_the_oracle(env, oracle_mod, storage, frac, prefetch, L, M):
    Index, stats_dict, _, w = env
    ix = Index(w.base, w.adj, w.entry, storage=storage, keep_f32=storage != "f32")
    q = torch.from_numpy(w.queries).cuda()
    # an exact visited set (open addressing, 2^15 slots, never reset at this size): the distance count is then
    # the same on every run, so it can be compared with the ungrouped index's
    kw = dict(rerank=storage != "f32", persistent=True, visited_mode=1, hash_bits=15)
    a_ids, a_d, a_st = ix.search(q, 10, L, M, with_stats=True, **kw)
    ix.group_neighbors(frac, prefetch)
    assert ix.info()["n_hot"] == round(frac * w.n)
    b_ids, b_d, b_st = ix.search(q, 10, L, M, with_stats=True, **kw)
    torch.cuda.synchronize()
    assert torch.equal(a_ids, b_ids) and torch.equal(a_d, b_d)
    sa, sb = stats_dict(a_st), stats_dict(b_st)
    for f in ("steps", "expansions", "evals"):
        np.testing.assert_array_equal(sa[f], sb[f])
    o_ids, o_keys, o_st = oracle_mod.search(w.base, w.adj, w.entry, w.queries, algo="topm", L=L, K=10, M0=1,
                                            M_max=M, t=1, nthreads=8)
    compare_exact(b_ids.cpu().numpy(), b_d.cpu().numpy(), o_ids, o_keys)
    np.testing.assert_array_equal(sb["steps"], o_st["steps"])
    ix.close()


def test_grouping_with_fp8_scales_regroup_and_remove(env, oracle_mod):
    """FP8 rows carry a per-row scale, copied with the row into the group."""
    Index, _, _, _ = env
    w = synth.make_workload("gist", 6000, 48, d=200)
    ix = Index(w.base, w.adj, w.entry, storage="e4m3", keep_f32=True)
    q = torch.from_numpy(w.queries).cuda()
    ref = ix.search(q, 10, 96, 8, rerank=True)
    plain = ix.search(q, 96, 96, 8)
    for frac in (0.02, 0.05, 0.0, 0.01):
        ix.group_neighbors(frac)
        assert ix.info()["n_hot"] == round(frac * w.n)
        got = ix.search(q, 10, 96, 8, rerank=True)
        got_plain = ix.search(q, 96, 96, 8)
        torch.cuda.synchronize()
        assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])
        assert torch.equal(plain[0], got_plain[0]) and torch.equal(plain[1], got_plain[1])
    ix.close()


def test_grouping_leaves_other_kernels_and_errors(env):
    """Clusters and asynchronous walkers read rows by id and are unaffected;
    bad fractions and prefetch modes are refused on the host."""
    Index, _, _abi, w = env
    ix = Index(w.base, w.adj, w.entry)
    q = torch.from_numpy(w.queries[:64]).cuda()
    c_ref = ix.search(q, 10, 128, 8, cluster=4)
    ix.group_neighbors(0.03)
    c_got = ix.search(q, 10, 128, 8, cluster=4)
    torch.cuda.synchronize()
    assert torch.equal(c_ref[0], c_got[0])
    for frac, pf in ((0.2, 0), (-0.1, 0), (0.01, 2)):
        with pytest.raises(_abi.AnnError):
            _abi.ann_index_group_neighbors(ix.handle, frac, pf)
    ix.close()
