"""GPU parity of the synchronous top-M search kernel against the FP64 oracle,
called through the C ABI (libann.so via ctypes)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2201_13007_gb300 import synth  # noqa: E402
from parity_util import compare_exact, compare_float, fp32_tie_window  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ann():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_13007_gb300 as pkg
    from paper_2201_13007_gb300.index import Index, stats_dict
    return pkg, Index, stats_dict


@pytest.fixture(scope="module")
def tiny():
    return synth.make_workload("tiny", 10000, 100)


@pytest.fixture(scope="module")
def sift_small():
    return synth.make_workload("sift", 20000, 64)


def _run(Index, w, storage="f32", keep_f32=False, k=10, L=64, M=4, queries=None, **kw):
    ix = Index(w.base, w.adj, w.entry, storage=storage, metric=w.metric, keep_f32=keep_f32)
    q = torch.from_numpy(queries if queries is not None else w.queries).cuda()
    ids, dists, st = ix.search(q, k, L, M, with_stats=True, **kw)
    torch.cuda.synchronize()
    out = ids.cpu().numpy(), dists.cpu().numpy(), st.cpu().numpy()
    ix.close()
    return out


@pytest.mark.parametrize("L", [32, 64, 128])
@pytest.mark.parametrize("M", [1, 4])
def test_tiny_float_parity(ann, oracle_mod, tiny, L, M):
    """Config: 10,000 x 32 FP32 mixture, exact 16-NN + reverse edges (cap 24),
    100 queries, k = 10, one CTA per query."""
    _, Index, stats_dict = ann
    ids, dists, st = _run(Index, tiny, L=L, M=M, hash_bits=15, visited_mode=1)
    o_ids, o_keys, o_st = oracle_mod.search(tiny.base, tiny.adj, tiny.entry, tiny.queries, algo="topm",
                                            L=L, K=10, M0=1, M_max=M, t=1, nthreads=8,
                                            tie_tol=fp32_tie_window(tiny.base, tiny.queries, "l2")[0])
    rep = compare_float(ids, dists, o_ids, o_keys, o_st["tie_events"], tiny.base, tiny.queries, "l2",
                        label=f"tiny L={L} M={M}")
    s = stats_dict(st)
    clean = (o_st["tie_events"] == 0)
    assert (s["hash_resets"] == 0).all()
    # with no forgotten vertices the distance count is exactly |V| of the oracle
    np.testing.assert_array_equal(s["evals"][clean], o_st["evals"][clean])
    np.testing.assert_array_equal(s["steps"][clean], o_st["steps"][clean])
    # every row either matches the oracle (up to swaps of near-equal keys) or is listed as exempt
    assert rep["match_frac"] >= 0.95, rep


@pytest.mark.parametrize("gather", [1, 2])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("L,M", [(16, 1), (64, 2), (100, 8), (200, 16), (64, 32)])
def test_integer_data_bit_exact(ann, oracle_mod, sift_small, storage, L, M, gather):
    """0..255 integer vectors, d = 128: FP32 sums are exact, so ids and keys
    must equal the oracle's bit for bit (BF16 holds 0..255 exactly), with
    each warp gathering its own fresh rows or all warps one list."""
    _, Index, stats_dict = ann
    w = sift_small
    ids, dists, st = _run(Index, w, storage=storage, L=L, M=M, hash_bits=15, visited_mode=1, gather=gather)
    o_ids, o_keys, o_st = oracle_mod.search(w.base, w.adj, w.entry, w.queries, algo="topm", L=L, K=10,
                                            M0=1, M_max=M, t=1, nthreads=8)
    compare_exact(ids, dists, o_ids, o_keys)
    s = stats_dict(st)
    np.testing.assert_array_equal(s["evals"], o_st["evals"])
    np.testing.assert_array_equal(s["steps"], o_st["steps"])
    np.testing.assert_array_equal(s["expansions"], o_st["expansions"])


@pytest.mark.parametrize("hash_bits", [8, 9, 11])
def test_forgetful_visited_table_keeps_ids(ann, oracle_mod, sift_small, hash_bits):
    """A small visited table is reset many times per query; ids and keys stay
    exact (the merge drops re-found queued ids), only evals grow."""
    _, Index, stats_dict = ann
    w = sift_small
    ids, dists, st = _run(Index, w, L=128, M=8, hash_bits=hash_bits, visited_mode=1)
    o_ids, o_keys, o_st = oracle_mod.search(w.base, w.adj, w.entry, w.queries, algo="topm", L=128, K=10,
                                            M0=1, M_max=8, t=1, nthreads=8)
    compare_exact(ids, dists, o_ids, o_keys)
    s = stats_dict(st)
    assert (s["hash_resets"] > 0).any()
    assert (s["evals"] >= o_st["evals"]).all()


@pytest.mark.parametrize("M0,t", [(1, 2), (2, 1), (4, 3)])
def test_schedule_variants(ann, oracle_mod, sift_small, M0, t):
    _, Index, _ = ann
    w = sift_small
    ids, dists, _ = _run(Index, w, L=96, M=16, M0=M0, t=t, hash_bits=15)
    o_ids, o_keys, _ = oracle_mod.search(w.base, w.adj, w.entry, w.queries, algo="topm", L=96, K=10,
                                         M0=M0, M_max=16, t=t, nthreads=8)
    compare_exact(ids, dists, o_ids, o_keys)


@pytest.mark.parametrize("threads", [64, 128, 256, 512])
def test_block_sizes_agree(ann, oracle_mod, sift_small, threads):
    _, Index, _ = ann
    w = sift_small
    ids, dists, _ = _run(Index, w, L=64, M=8, threads=threads)
    o_ids, o_keys, _ = oracle_mod.search(w.base, w.adj, w.entry, w.queries, algo="topm", L=64, K=10,
                                         M0=1, M_max=8, t=1, nthreads=8)
    compare_exact(ids, dists, o_ids, o_keys)


def test_ip_metric_parity(ann, oracle_mod):
    _, Index, _ = ann
    w = synth.make_workload("deep", 20000, 64, components=32)
    ids, dists, st = _run(Index, w, L=64, M=4, hash_bits=15)
    o_ids, o_keys, o_st = oracle_mod.search(w.base, w.adj, w.entry, w.queries, algo="topm", metric="ip",
                                            L=64, K=10, M0=1, M_max=4, t=1, nthreads=8,
                                            tie_tol=0.0, tie_abs=fp32_tie_window(w.base, w.queries, "ip")[1])
    compare_float(ids, dists, o_ids, o_keys, o_st["tie_events"], w.base, w.queries, "ip")


def test_edge_cases_small_graphs(ann, oracle_mod):
    """L = 1, k = L, L > n (queue never fills), -1 padded rows, unreachable
    vertices, duplicate vectors (exact key ties broken by id), ragged d."""
    _, Index, _ = ann
    for seed, (n, d, R, pad, dup) in enumerate([(50, 3, 4, 0.3, 0.2), (300, 37, 7, 0.1, 0.1),
                                                 (9, 5, 2, 0.5, 0.0), (1, 4, 1, 0.0, 0.0)]):
        base, adj, q = synth.random_graph(max(n, 2), d, R, seed=seed, nq=16, pad_frac=pad, dup_frac=dup)
        base, adj = base[:n], np.where(adj[:n] < n, adj[:n], -1).astype(np.int32)
        # integer-valued copies make the comparison exact
        base = np.rint(base * 8).astype(np.float32)
        q = np.rint(q * 8).astype(np.float32)
        w = synth.Workload("edge", base, q, adj, 0, "l2")
        for k, L, M in [(1, 1, 1), (3, 3, 2), (5, 64, 4), (2, 8, 64)]:
            ids, dists, _ = _run(Index, w, k=k, L=L, M=M, queries=q)
            o_ids, o_keys, _ = oracle_mod.search(base, adj, 0, q, algo="topm", L=L, K=k, M0=1, M_max=M, t=1)
            compare_exact(ids, dists, o_ids, o_keys)


def test_empty_batch_and_argument_errors(ann, tiny):
    pkg, Index, _ = ann
    ix = Index(tiny.base, tiny.adj, tiny.entry)
    q = torch.zeros((0, tiny.d), device="cuda")
    ids, dists = ix.search(q, 10, 32, 4)
    assert ids.shape == (0, 10)
    qq = torch.zeros((2, tiny.d), device="cuda")
    with pytest.raises(pkg.AnnError):
        ix.search(qq, 11, 10, 1)  # k > L
    with pytest.raises(pkg.AnnError):
        ix.search(qq, 1, 4096, 1)  # L too large
    with pytest.raises(pkg.AnnError):
        ix.search(qq, 1, 8, 65)  # M too large
    ix.search(qq, 1, 8, 1, rerank=True)  # an FP32 base is its own re-rank copy
    ix.close()
    ixb = Index(tiny.base, tiny.adj, tiny.entry, storage="bf16")
    with pytest.raises(pkg.AnnError):
        ixb.search(qq, 1, 8, 1, rerank=True)  # no FP32 copy kept
    ixb.close()


def test_bad_adjacency_rejected(ann):
    pkg, Index, _ = ann
    base = np.zeros((4, 8), np.float32)
    adj = np.array([[1], [2], [7], [0]], np.int32)
    with pytest.raises(pkg.AnnError):
        Index(base, adj, 0)
    with pytest.raises(pkg.AnnError):
        Index(torch.from_numpy(base).cuda(), torch.from_numpy(adj).cuda(), 0)


def test_persistent_per_query_and_host_paths_agree(ann, sift_small):
    _, Index, _ = ann
    w = sift_small
    ix = Index(w.base, w.adj, w.entry)
    q = torch.from_numpy(w.queries).cuda()
    ids0, d0 = ix.search(q, 10, 80, 8)
    ids1, d1 = ix.search(q, 10, 80, 8, persistent=True)
    assert torch.equal(ids0, ids1) and torch.equal(d0, d1)
    hi, hd = ix.search_host(torch.from_numpy(w.queries).pin_memory(), 10, 80, 8)
    assert torch.equal(hi, ids0.cpu()) and torch.equal(hd, d0.cpu())
    # per-query k / L / M: each row equals its own uniform call
    nq = q.shape[0]
    g = np.random.default_rng(0)
    ks = g.choice([1, 5, 10], nq).astype(np.int32)
    Ls = np.maximum(ks, g.choice([16, 40, 80], nq)).astype(np.int32)
    Ms = g.choice([1, 2, 8], nq).astype(np.int32)
    ids2, d2 = ix.search(q, 10, 80, 8, k_per_query=torch.from_numpy(ks).cuda(),
                         L_per_query=torch.from_numpy(Ls).cuda(), M_per_query=torch.from_numpy(Ms).cuda(),
                         persistent=True)
    ids2, d2 = ids2.cpu(), d2.cpu()
    for i in range(nq):
        a, b = ix.search(q[i:i + 1], int(ks[i]), int(Ls[i]), int(Ms[i]))
        assert torch.equal(ids2[i, :ks[i]], a[0].cpu()) and torch.equal(d2[i, :ks[i]], b[0].cpu())
        assert (ids2[i, ks[i]:] == -1).all()
    ix.close()


def test_deterministic_reruns(ann, tiny):
    _, Index, _ = ann
    ix = Index(tiny.base, tiny.adj, tiny.entry)
    q = torch.from_numpy(tiny.queries).cuda()
    ref = ix.search(q, 10, 128, 4, hash_bits=9)
    for _ in range(20):
        got = ix.search(q, 10, 128, 4, hash_bits=9)
        assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])
    ix.close()


@pytest.mark.parametrize("storage", ["bf16", "f16", "e4m3"])
def test_reduced_precision_with_rerank(ann, oracle_mod, storage):
    """Reduced-precision storage: the search must follow the oracle run on
    the stored (rounded) values; the re-rank must equal the oracle's exact
    re-rank of that final queue with FP32 rows."""
    _, Index, _ = ann
    w = synth.make_workload("gist", 8000, 48, d=240)
    L, M = 64, 4
    stored = oracle_mod.stored_values(w.base, storage)
    ix = Index(w.base, w.adj, w.entry, storage=storage, keep_f32=True)
    q = torch.from_numpy(w.queries).cuda()
    ids_nr, d_nr = ix.search(q, L, L, M, hash_bits=15)          # whole final queue, stored keys
    ids_rr, d_rr = ix.search(q, 10, L, M, hash_bits=15, rerank=True)
    torch.cuda.synchronize()
    o_ids, o_keys, o_st = oracle_mod.search(stored, w.adj, w.entry, w.queries, algo="topm", L=L, K=L,
                                            M0=1, M_max=M, t=1, nthreads=8,
                                            tie_tol=fp32_tie_window(stored, w.queries, "l2")[0])
    compare_float(ids_nr.cpu().numpy(), d_nr.cpu().numpy(), o_ids, o_keys, o_st["tie_events"], stored,
                  w.queries, "l2")
    clean = o_st["tie_events"] == 0
    r_ids, r_keys = oracle_mod.rerank(w.base, w.queries, o_ids, 10)
    compare_float(ids_rr.cpu().numpy()[clean], d_rr.cpu().numpy()[clean], r_ids[clean], r_keys[clean],
                  np.zeros(clean.sum()), w.base, w.queries[clean], "l2")
    # and on every row, the re-rank of the GPU's own final queue
    r_ids, r_keys = oracle_mod.rerank(w.base, w.queries, ids_nr.cpu().numpy(), 10)
    compare_float(ids_rr.cpu().numpy(), d_rr.cpu().numpy(), r_ids, r_keys, np.zeros(r_ids.shape[0]), w.base,
                  w.queries, "l2", max_exempt_frac=0.0)
    ix.close()


@pytest.mark.parametrize("storage", ["e4m3", "f16"])
def test_high_dimension_d960_with_rerank(ann, oracle_mod, storage):
    """The high-dimension workload's shape (d = 960, log-normal mixture) in
    FP8-E4M3 with per-vector scales and in FP16, with the launch the library
    chooses: the search follows the oracle run on the stored values within
    the FP32 error bound, and the FP32 re-rank equals the oracle's re-rank
    of its final queue."""
    _, Index, _ = ann
    w = synth.make_workload("gist", 20000, 64)
    assert w.d == 960
    L, M = 128, 8
    stored = oracle_mod.stored_values(w.base, storage)
    ix = Index(w.base, w.adj, w.entry, storage=storage, keep_f32=True)
    q = torch.from_numpy(w.queries).cuda()
    ids_nr, d_nr = ix.search(q, L, L, M)              # the whole final queue, stored keys
    ids_rr, d_rr = ix.search(q, 10, L, M, rerank=True)
    torch.cuda.synchronize()
    o_ids, o_keys, o_st = oracle_mod.search(stored, w.adj, w.entry, w.queries, algo="topm", L=L, K=L,
                                            M0=1, M_max=M, t=1, nthreads=8,
                                            tie_tol=fp32_tie_window(stored, w.queries, "l2")[0])
    compare_float(ids_nr.cpu().numpy(), d_nr.cpu().numpy(), o_ids, o_keys, o_st["tie_events"], stored,
                  w.queries, "l2", label=f"d=960 {storage} stored keys")
    # the re-rank step itself, on every row: the oracle re-ranks the GPU's own final queue (the same
    # deterministic search without re-rank) with the FP32 rows
    r_ids, r_keys = oracle_mod.rerank(w.base, w.queries, ids_nr.cpu().numpy(), 10)
    compare_float(ids_rr.cpu().numpy(), d_rr.cpu().numpy(), r_ids, r_keys, np.zeros(r_ids.shape[0]), w.base,
                  w.queries, "l2", max_exempt_frac=0.0, label=f"d=960 {storage} re-rank")
    ix.close()


@pytest.mark.parametrize("visited_mode,slot_bytes", [(2, 1), (3, 4), (4, 4)])
@pytest.mark.parametrize("hash_bits", [8, 10, 12])
def test_direct_mapped_visited_cache_keeps_ids(ann, oracle_mod, sift_small, hash_bits, visited_mode, slot_bytes):
    """The direct-mapped visited cache forgets a vertex whenever another one
    hashes to its slot, the set-associative one when a fourth vertex enters a
    full set; ids and keys must still be exact (reading 14). Mode 2 keeps a
    one-byte tag per slot here (20,000 ids need 15 bits), mode 3 a full id,
    mode 4 three tags per set word."""
    _, Index, stats_dict = ann
    w = sift_small
    ix = Index(w.base, w.adj, w.entry)
    assert ix.describe(64, 10, 128, 8, hash_bits=hash_bits, visited_mode=visited_mode)["visited_slot_bytes"] == slot_bytes
    if visited_mode == 4:
        assert ix.describe(64, 10, 128, 8, hash_bits=hash_bits, visited_mode=4)["visited_ways"] == 3
    ix.close()
    ids, dists, st = _run(Index, w, L=128, M=8, hash_bits=hash_bits, visited_mode=visited_mode)
    o_ids, o_keys, o_st = oracle_mod.search(w.base, w.adj, w.entry, w.queries, algo="topm", L=128, K=10,
                                            M0=1, M_max=8, t=1, nthreads=8)
    compare_exact(ids, dists, o_ids, o_keys)
    s = stats_dict(st)
    assert (s["evals"] >= o_st["evals"]).all()


_TEAM_ORACLE = {}


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("team_lanes", [-1, 1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("l2_prefetch", [1, 2])
def test_team_sizes_exact(ann, oracle_mod, sift_small, storage, team_lanes, l2_prefetch):
    """Any number of lanes per row in the distance gather (with or without
    the L2 prefetch of fresh rows) gives exactly the oracle's ids, keys and
    distance counts on integer data; the re-rank's FP32 rows take the same
    team size rule."""
    _, Index, stats_dict = ann
    w = sift_small
    for L, M in ((64, 4), (200, 16), (128, 32)):
        ids, dists, st = _run(Index, w, storage=storage, keep_f32=storage != "f32", L=L, M=M, hash_bits=15,
                              visited_mode=1, team_lanes=team_lanes, l2_prefetch=l2_prefetch,
                              rerank=storage != "f32")
        if (L, M) not in _TEAM_ORACLE:
            _TEAM_ORACLE[(L, M)] = oracle_mod.search(w.base, w.adj, w.entry, w.queries, algo="topm", L=L, K=10,
                                                     M0=1, M_max=M, t=1, nthreads=8)
        o_ids, o_keys, o_st = _TEAM_ORACLE[(L, M)]
        compare_exact(ids, dists, o_ids, o_keys)
        np.testing.assert_array_equal(stats_dict(st)["evals"], o_st["evals"])


@pytest.mark.parametrize("storage", ["f32", "f16", "e4m3"])
@pytest.mark.parametrize("team_lanes", [1, 4, 32])
def test_team_sizes_float_ragged_rows(ann, oracle_mod, storage, team_lanes):
    """Float data with d = 200: rows whose chunk count is not a multiple of
    the team size times the chunks in flight (ragged last round per lane).
    Keys follow the oracle on the stored values within the FP32 error bound;
    the FP32 re-rank of the final queue equals the oracle's re-rank."""
    _, Index, _ = ann
    w = synth.make_workload("gist", 6000, 48, d=200)
    L, M = 64, 8
    stored = oracle_mod.stored_values(w.base, storage)
    ix = Index(w.base, w.adj, w.entry, storage=storage, keep_f32=storage != "f32")
    q = torch.from_numpy(w.queries).cuda()
    ids, d = ix.search(q, L, L, M, hash_bits=15, team_lanes=team_lanes)
    torch.cuda.synchronize()
    o_ids, o_keys, o_st = oracle_mod.search(stored, w.adj, w.entry, w.queries, algo="topm", L=L, K=L,
                                            M0=1, M_max=M, t=1, nthreads=8,
                                            tie_tol=fp32_tie_window(stored, w.queries, "l2")[0])
    compare_float(ids.cpu().numpy(), d.cpu().numpy(), o_ids, o_keys, o_st["tie_events"], stored, w.queries, "l2")
    if storage != "f32":
        ids_rr, d_rr = ix.search(q, 10, L, M, hash_bits=15, rerank=True, team_lanes=team_lanes)
        torch.cuda.synchronize()
        clean = o_st["tie_events"] == 0
        r_ids, r_keys = oracle_mod.rerank(w.base, w.queries, o_ids, 10)
        compare_float(ids_rr.cpu().numpy()[clean], d_rr.cpu().numpy()[clean], r_ids[clean], r_keys[clean],
                      np.zeros(clean.sum()), w.base, w.queries[clean], "l2")
    ix.close()


def test_gather_option_errors(ann, tiny):
    pkg, Index, _ = ann
    ix = Index(tiny.base, tiny.adj, tiny.entry)
    q = torch.from_numpy(tiny.queries).cuda()
    for bad in (dict(team_lanes=3), dict(team_lanes=64), dict(team_lanes=-2), dict(l2_prefetch=3),
                dict(l2_prefetch=-1)):
        with pytest.raises(pkg.AnnError):
            ix.search(q, 10, 64, 4, **bad)
    ix.close()


@pytest.mark.parametrize("hash_bits,slot_bytes", [(8, 2), (9, 2), (10, 1)])
def test_two_byte_visited_tags_exact(ann, oracle_mod, hash_bits, slot_bytes):
    """70,000 vertices need 17 id bits, so 2^8 / 2^9 / 2^10 slots leave tags
    of 9 / 8 / 7 bits: two bytes per slot, two bytes, one byte. Results stay
    exact on integer data."""
    _, Index, stats_dict = ann
    w = synth.make_workload("sift", 70000, 48)
    ix = Index(w.base, w.adj, w.entry)
    assert ix.describe(48, 10, 96, 8, hash_bits=hash_bits, visited_mode=2)["visited_slot_bytes"] == slot_bytes
    ix.close()
    ids, dists, st = _run(Index, w, L=96, M=8, hash_bits=hash_bits, visited_mode=2)
    o_ids, o_keys, o_st = oracle_mod.search(w.base, w.adj, w.entry, w.queries, algo="topm", L=96, K=10,
                                            M0=1, M_max=8, t=1, nthreads=8)
    compare_exact(ids, dists, o_ids, o_keys)
    assert (stats_dict(st)["evals"] >= o_st["evals"]).all()
