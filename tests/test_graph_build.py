"""The large-set graph builder (device tensors, paper_2201_13007_gb300.graph)
step by step against the builder of the synthetic workloads
(paper_2201_13007_gb300.synth), on CPU tensors: both must give the same
candidate lists, pruned lists, reverse fill and reachable set."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_13007_gb300 import graph, synth


@pytest.fixture(scope="module")
def small_set():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2500, 32)).astype(np.float32)
    x = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    ids, dd = synth.knn_lists(x, 16, exact64=True)
    return x, ids, dd


def test_builder_steps_match_the_workload_builder(small_set):
    x, ids, dd = small_set
    X = torch.from_numpy(x)
    cand, cd = graph.union_candidates(torch.from_numpy(ids), torch.from_numpy(dd), 40)
    c2, cd2 = synth.union_candidates(ids, dd, 40)
    np.testing.assert_array_equal(cand.numpy(), c2)
    np.testing.assert_array_equal(cd.numpy(), cd2)
    pr = graph.occlusion_prune(X, cand, cd, 12, batch=700)
    pr2 = synth.occlusion_prune(x, c2, cd2, 12)
    np.testing.assert_array_equal(pr.numpy(), pr2)
    rf = graph.reverse_fill(X, pr, 16, chunk=3001)
    rf2 = synth.reverse_fill(x, pr2, 16)
    np.testing.assert_array_equal(rf.numpy(), rf2)


def test_reachable_matches_scipy_bfs(small_set):
    x, ids, dd = small_set
    adj = synth.reverse_fill(x, ids[:, :4], 6)
    adj[:, 2:] = -1                      # sparse enough to leave parts unreachable
    for entry in (0, 17, 2499):
        got = graph.reachable(torch.from_numpy(adj), entry)
        np.testing.assert_array_equal(got, synth.reachable_from(adj, entry))


def test_medoid_matches_the_workload_entry_point(small_set):
    x, _, _ = small_set
    assert graph.medoid(torch.from_numpy(x)) == synth.entry_point(x)


def test_repair_with_the_device_bfs_equals_the_repair_with_scipy(small_set):
    """The large-set builder repairs reachability through synth's repair loop
    with its own BFS: the same links as with scipy's BFS, and afterwards
    every vertex is reachable."""
    x, ids, _ = small_set
    adj = synth.reverse_fill(x, ids[:, :3], 4)
    adj[::7, :] = -1                      # cut many vertices off
    entry = synth.entry_point(x)
    a1, n1 = synth.repair_reachability(adj, entry, None, x, device="cpu")
    a2, n2 = synth.repair_reachability(adj, entry, None, x, device="cpu",
                                       reach=lambda A, e: graph.reachable(torch.from_numpy(A), e))
    assert n1 == n2 > 0
    np.testing.assert_array_equal(a1, a2)
    assert synth.reachable_from(a2, entry).all()
