"""The allocation-free host-buffer search (ann_search_host_noalloc).

Some callers cannot allocate device memory when they search (a thread that
is capturing a CUDA graph, a process whose device memory is held by another
framework's allocator); this entry point keeps its device scratch in one
static device array instead. Here it must give the same answers as the
ordinary host-buffer search (ann_search_host) on two calls in a row with
different batches, and refuse a batch that does not fit its scratch.

This file is named to be collected last so that a run that stops at the
first failure has already run every other test; it builds its own inputs and
also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_13007_gb300 import _abi, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _vp(a):
    return ctypes.c_void_p(a.ctypes.data)


@pytest.fixture(scope="module")
def index():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    w = synth.make_workload("sift", 20000, 64)
    base = np.ascontiguousarray(w.base, np.float32)
    adj = np.ascontiguousarray(w.adj, np.int32)
    h = _abi.ann_index_create(_vp(base), w.n, w.d, _abi.STORAGE["bf16"], _vp(adj), w.R, w.entry,
                              _abi.METRIC["l2"], _abi.ANN_INDEX_KEEP_F32)
    yield ctypes.c_void_p(h), w
    _abi.ann_index_destroy(ctypes.c_void_p(h))


def _run(fn, h, q, k, L, M, params):
    nq = q.shape[0]
    ids = np.full((nq, k), -7, np.int64)
    dists = np.full((nq, k), np.nan, np.float32)
    fn(h, _vp(q), nq, k, L, M, _vp(ids), _vp(dists), params, None)
    return ids, dists


@pytest.mark.parametrize("mode,rerank", [("sync", 0), ("sync", 1)])
def test_matches_host_search_on_two_calls(index, mode, rerank):
    h, w = index
    params = _abi.SearchParams(mode=_abi.MODE[mode], rerank=rerank)
    batches = [np.ascontiguousarray(w.queries[:48]), np.ascontiguousarray(w.queries[16:64][::-1])]
    for q in batches:  # two calls in a row, different batches: the shared counter must be reset
        a_ids, a_d = _run(_abi.ann_search_host, h, q, 10, 96, 8, params)
        b_ids, b_d = _run(_abi.ann_search_host_noalloc, h, q, 10, 96, 8, params)
        # deterministic search: identical answers (tighter than the float tolerance of the other tests)
        np.testing.assert_array_equal(b_ids, a_ids)
        np.testing.assert_array_equal(b_d, a_d)
        assert (b_ids >= 0).all()


def test_rejects_batch_beyond_static_scratch(index):
    h, w = index
    k = 10
    per_query = w.d * 4 + k * 12
    nq = _abi.ANN_NOALLOC_SCRATCH_BYTES // per_query + 1
    q = np.zeros((nq, w.d), np.float32)
    with pytest.raises(_abi.AnnError) as ei:
        _run(_abi.ann_search_host_noalloc, h, q, k, 32, 4, None)
    assert "maximum" in str(ei.value) and "static device scratch" in str(ei.value)
