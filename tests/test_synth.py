"""The seeded input generators: deterministic, well-formed graphs."""
import numpy as np

from paper_2201_13007_gb300 import synth


def test_tiny_workload_shape_and_reachability():
    w = synth.make_workload("tiny", 2000, 10, cache=False)
    assert w.base.shape == (2000, 32) and w.adj.shape == (2000, 24) and w.queries.shape == (10, 32)
    assert ((w.adj >= -1) & (w.adj < w.n)).all()
    assert (w.adj != np.arange(w.n)[:, None]).all()  # no self loops
    assert synth.reachable_from(w.adj, w.entry).all()
    for row in w.adj:
        r = row[row >= 0]
        assert len(set(r.tolist())) == len(r)


def test_generators_are_deterministic():
    a = synth.mixture_sift(300, 5, seed=200)
    b = synth.mixture_sift(300, 5, seed=200)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert a[0].min() >= 0 and a[0].max() <= 255 and (a[0] == np.rint(a[0])).all()
    d = synth.mixture_deep(200, 3)[0]
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, rtol=1e-5)
    g = synth.mixture_gist(50, 2, d=96)[0]
    assert (g > 0).all()


def test_pruned_graph_small():
    base, q = synth.mixture_sift(1500, 4, seed=200)
    adj, knn = synth.build_pruned_graph(base, R=16, k=32)
    e = synth.entry_point(base)
    adj, _ = synth.repair_reachability(adj, e, knn, base)
    assert adj.shape == (1500, 16)
    assert synth.reachable_from(adj, e).all()


def test_graph_quality_on_a_hand_built_graph():
    """A 4-cycle 0 -> 1 -> 2 -> 3 -> 0 plus the chords 0 -> 2 and 2 -> 0,
    with an isolated vertex 4 (R = 2, -1 padded)."""
    adj = np.array([[1, 2], [2, -1], [3, 0], [0, -1], [-1, -1]], np.int32)
    knn = np.array([[1], [2], [3], [0], [3]], np.int32)
    q = synth.graph_quality(adj, 0, knn, sample=5)
    assert q["out_degree"]["max"] == 2 and q["out_degree"]["min"] == 0
    assert q["out_degree"]["full_rows"] == 2 / 5
    assert q["in_degree"]["max"] == 2 and q["in_degree"]["zero"] == 1 / 5
    assert q["reachable_from_entry"] == 4 / 5
    # edges 0-1, 0-2, 1-2, 2-3, 2-0, 3-0: reciprocal are 0->2 and 2->0
    assert q["reciprocal_edges"] == 2 / 6
    # exact 1-NN among out-neighbours: vertices 0, 1, 2, 3 yes, 4 no
    assert q["exact_1nn_in_out_edges"] == 4 / 5
