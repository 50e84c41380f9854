"""Persistent searches on one index from several streams at once.

A persistent grid pulls its queries from a device work counter that the call
resets first. The index keeps one counter per stream, so searches on
different streams can overlap on the GPU without resetting or draining each
other's counter: every result must equal the same search run alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_13007_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_13007_gb300.index import Index
    w = synth.make_workload("sift", 20000, 1200)
    ix = Index(w.base, w.adj, w.entry, storage="bf16", keep_f32=True)
    yield ix, w
    ix.close()


@pytest.mark.parametrize("mode", ["sync", "async"])
def test_concurrent_persistent_searches_match_serial_ones(env, mode):
    ix, w = env
    q = torch.from_numpy(w.queries).cuda()
    parts = [q[0:400], q[400:800], q[800:1200]]
    kw = dict(rerank=True, persistent=True, mode=mode, R_ratio=0.8)
    # 400 queries per call: a grid of 400 CTAs leaves room on the GPU for the other streams' grids
    serial = []
    for p in parts:
        serial.append(ix.search(p, 10, 128, 8, **kw))
        torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in parts]
    for rep in range(3):
        outs = [(torch.full((p.shape[0], 10), -9, dtype=torch.int64, device="cuda"),
                 torch.zeros((p.shape[0], 10), device="cuda")) for p in parts]
        torch.cuda.synchronize()
        for p, s, o in zip(parts, streams, outs):
            ix.search(p, 10, 128, 8, out=o, stream=s, **kw)
        torch.cuda.synchronize()
        for (ids, d), (rid, rd) in zip(outs, serial):
            assert (ids >= 0).all(), "a query was skipped"
            if mode == "sync":
                assert torch.equal(ids, rid) and torch.equal(d, rd)
            else:  # the walkers' interleaving varies from run to run; every query must be answered in full
                assert (d < float("inf")).all()


def test_default_and_side_streams_share_nothing(env):
    """The legacy default stream and a side stream also get separate counters."""
    ix, w = env
    q = torch.from_numpy(w.queries).cuda()
    a_ref = ix.search(q[:600], 10, 96, 8, persistent=True)
    b_ref = ix.search(q[600:], 10, 96, 8, persistent=True)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    a = (torch.empty_like(a_ref[0]), torch.empty_like(a_ref[1]))
    b = (torch.empty_like(b_ref[0]), torch.empty_like(b_ref[1]))
    ix.search(q[:600], 10, 96, 8, persistent=True, out=a, stream=torch.cuda.default_stream())
    ix.search(q[600:], 10, 96, 8, persistent=True, out=b, stream=s)
    torch.cuda.synchronize()
    assert torch.equal(a[0], a_ref[0]) and torch.equal(b[0], b_ref[0])
