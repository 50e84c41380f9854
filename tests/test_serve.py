"""Continuous-batching server (ann_serve_*), through the C ABI."""
import ctypes
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_13007_gb300 import _abi, synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _vp(a):
    return ctypes.c_void_p(a.ctypes.data)


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_13007_gb300.index import Index
    w = synth.make_workload("sift", 20000, 2000)
    ix = Index(w.base, w.adj, w.entry)
    yield ix, w
    ix.close()


def _server(ix, **kw):
    cfg = _abi.ServeConfig(**kw)
    return ctypes.c_void_p(_abi.ann_serve_create(ix.handle, cfg))


def _collect(srv, out, kmax, timeout_us):
    res = (_abi.Result * 64)()
    ids = np.zeros((64, kmax), np.int64)
    dists = np.zeros((64, kmax), np.float32)
    got = _abi.ann_serve_poll(srv, res, _vp(ids), _vp(dists), 64, timeout_us)
    for i in range(got):
        r = res[i]
        out[r.tag] = (r.status, r.k, ids[i, :r.k].copy(), dists[i, :r.k].copy(), r.latency_us, r.device_us,
                      r.device_start_ns, r.device_end_ns)
    return got


def _drain(srv, n, kmax, timeout_s=60.0, out=None):
    out = {} if out is None else out
    t0 = time.time()
    while len(out) < n and time.time() - t0 < timeout_s:
        _collect(srv, out, kmax, 100000)
    return out


def test_each_result_equals_its_standalone_search(setup):
    ix, w = setup
    g = np.random.default_rng(7)
    n = 600
    qi = g.integers(0, w.queries.shape[0], n)
    ks = g.choice([1, 10, 20], n)
    Ls = np.maximum(ks, g.choice([16, 32, 64, 128], n))
    Ms = g.choice([1, 2, 4, 8], n)
    srv = _server(ix, max_batch=8, streams=4, max_k=20, max_L=128, max_M=8)
    out = {}
    try:
        for t in range(n):
            q = np.ascontiguousarray(w.queries[qi[t]])
            # a full server (every slot submitted and not yet collected) answers BUSY: collect, then retry
            while _abi.ann_serve_submit(srv, _vp(q), int(ks[t]), int(Ls[t]), int(Ms[t]), t) == _abi.ANN_ERR_BUSY:
                _collect(srv, out, 20, 1000)
        _drain(srv, n, 20, out=out)
    finally:
        _abi.ann_serve_destroy(srv)
    assert len(out) == n
    # each answer equals the oracle's search of that query with its own k, L, M: integer-valued data, so
    # ids and keys are bit-exact
    from parity_util import oracle_rows
    import oracle
    oracle.build()
    o_ids, o_keys = oracle_rows(oracle, w.base, w.adj, w.entry, w.queries[qi], ks, Ls, Ms)[:2]
    for t in range(n):
        np.testing.assert_array_equal(out[t][2], o_ids[t], err_msg=f"request {t}")
        np.testing.assert_array_equal(out[t][3].astype(np.float64), o_keys[t], err_msg=f"request {t}")
    # each answer equals the same query searched alone with its own k, L, M
    qd = torch.from_numpy(w.queries).cuda()
    for t in range(n):
        status, k, rid, rd = out[t][:4]
        assert status == 0 and k == ks[t]
        a_ids, a_d = ix.search(qd[qi[t]:qi[t] + 1], int(ks[t]), int(Ls[t]), int(Ms[t]))
        np.testing.assert_array_equal(rid, a_ids[0].cpu().numpy())
        np.testing.assert_array_equal(rd, a_d[0].cpu().numpy())
    # launches overlapped on the device: more requests were active at once than one launch holds
    ev = sorted([(v[6], 1) for v in out.values()] + [(v[7], -1) for v in out.values()])
    cur = peak = 0
    for _, d in ev:
        cur += d
        peak = max(peak, cur)
    assert peak > 8, peak
    lat = np.array([v[4] for v in out.values()])
    assert (lat > 0).all()


def test_busy_timeout_and_argument_errors(setup):
    ix, w = setup
    srv = _server(ix, max_batch=4, streams=1, max_k=10, max_L=64, max_M=4, slots=6)
    try:
        q = np.ascontiguousarray(w.queries[0])
        codes = [_abi.ann_serve_submit(srv, _vp(q), 10, 64, 4, t) for t in range(10)]
        assert codes.count(_abi.ANN_ERR_BUSY) == 4 and codes[:6] == [0] * 6
        out = _drain(srv, 6, 10)
        assert sorted(out) == list(range(6))
        # nothing left: a poll waits about its timeout and returns nothing
        res = (_abi.Result * 4)()
        ids = np.zeros((4, 10), np.int64)
        d = np.zeros((4, 10), np.float32)
        t0 = time.time()
        assert _abi.ann_serve_poll(srv, res, _vp(ids), _vp(d), 4, 20000) == 0
        assert time.time() - t0 >= 0.015
        with pytest.raises(_abi.AnnError):
            _abi.ann_serve_submit(srv, _vp(q), 11, 64, 4, 99)  # k above max_k
        with pytest.raises(_abi.AnnError):
            _abi.ann_serve_submit(srv, _vp(q), 10, 8, 4, 99)  # L < k
    finally:
        _abi.ann_serve_destroy(srv)


def test_scratch_budget_limits_groups(setup):
    ix, w = setup
    per_group = 8 * (w.d * 4 + 12 + 10 * 12 + 64)
    srv = _server(ix, max_batch=8, streams=8, max_k=10, max_L=32, max_M=2, scratch_bytes=3 * per_group)
    try:
        q = np.ascontiguousarray(w.queries[1])
        out = {}
        for t in range(40):
            while _abi.ann_serve_submit(srv, _vp(q), 10, 32, 2, t) == _abi.ANN_ERR_BUSY:
                _collect(srv, out, 10, 1000)
        _drain(srv, 40, 10, out=out)
        assert len(out) == 40
        first = out[0][2]
        for v in out.values():
            np.testing.assert_array_equal(v[2], first)
    finally:
        _abi.ann_serve_destroy(srv)
    with pytest.raises(_abi.AnnError):
        _server(ix, max_batch=8, streams=2, max_k=10, max_L=32, max_M=2, scratch_bytes=per_group // 2)


def test_trace_replay_completes_every_request(setup):
    """ann_serve_replay drives the server from native threads: every request
    of a flood trace and of a Poisson trace completes with ANN_OK, each
    latency is at least its device time, and the timed window covers the
    last arrival. The results themselves are the server's (compared with
    standalone searches above)."""
    ix, w = setup
    srv = _server(ix, max_batch=64, streams=2, max_k=10, max_L=128, max_M=8, slots=256)
    try:
        g = np.random.default_rng(3)
        n = 600
        qi = g.integers(0, w.queries.shape[0], n)
        k = np.full(n, 10, np.int32)
        L = g.choice([32, 64, 128], n).astype(np.int32)
        M = g.choice([1, 4, 8], n).astype(np.int32)
        lat, dev, st, wall, busy = _abi.ann_serve_replay(srv, w.queries, qi, k, L, M)
        assert (st == 0).all() and np.isfinite(lat).all() and (lat >= dev).all() and wall > 0
        arr = np.cumsum(g.exponential(1e6 / 20000.0, n))
        lat, dev, st, wall, busy = _abi.ann_serve_replay(srv, w.queries, qi, k, L, M, arr)
        assert (st == 0).all() and np.isfinite(lat).all() and wall >= arr[-1]
        with pytest.raises(_abi.AnnError):
            _abi.ann_serve_replay(srv, w.queries, qi, k, L, M, arr[::-1].copy())  # arrivals must not decrease
        with pytest.raises(_abi.AnnError):
            _abi.ann_serve_replay(srv, w.queries, qi + w.queries.shape[0], k, L, M)  # rows out of range
    finally:
        _abi.ann_serve_destroy(srv)
