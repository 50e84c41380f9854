"""The paper's qualitative claims about its search variants, checked on the
oracle with a small seeded workload (6,000 points of the sift-like mixture,
300 queries, L = 64). These are trends, not exact values: the margins are
wide, and each check names the passage whose claim it restates.
"""
import numpy as np
import pytest

from paper_2201_13007_gb300 import synth

L = 64


@pytest.fixture(scope="module")
def runs(oracle_mod):
    w = synth.make_workload("sift", 6000, 300)

    def run(**kw):
        ids, keys, st = oracle_mod.search(w.base, w.adj, w.entry, w.queries, K=10, L=L, nthreads=8, **kw)
        return ids, keys, st

    out = {"bfis": run(algo="bfis")}
    for M in (4, 16):
        out[f"fixed{M}"] = run(algo="topm", M0=M, M_max=M, t=1)
    out["staged16"] = run(algo="topm", M0=1, M_max=16, t=1)
    for M in (2, 8):
        out[f"nosync{M}"] = run(algo="speedann", M0=1, M_max=M, R_ratio=float("inf"))
    return out


def _mean(r, f):
    return float(r[2][f].mean())


def test_top_m_takes_fewer_steps_than_bfis(runs):
    """Sec. 4.1: expanding the top M unchecked vertices per step shortens the
    dependent chain of steps (the convergence critical path)."""
    s_b, s4, s16 = (_mean(runs[k], "steps") for k in ("bfis", "fixed4", "fixed16"))
    assert s4 < 0.5 * s_b and s16 < s4, (s_b, s4, s16)


def test_distance_evaluations_grow_with_m(runs):
    """Sec. 4.2: a wider expansion computes more distances (it also expands
    vertices that sequential search would have skipped)."""
    e_b, e4, e16 = (_mean(runs[k], "evals") for k in ("bfis", "fixed4", "fixed16"))
    assert e_b <= e4 <= e16 and e16 > 1.2 * e_b, (e_b, e4, e16)


def test_staged_search_keeps_evals_near_bfis_and_steps_near_top_m(runs):
    """Sec. 4.2: starting at M = 1 and doubling keeps the distance count close
    to the sequential search's while the step count stays close to the wide
    search's."""
    e_b, e16, e_s = (_mean(runs[k], "evals") for k in ("bfis", "fixed16", "staged16"))
    s16, s_s = _mean(runs["fixed16"], "steps"), _mean(runs["staged16"], "steps")
    assert s_s <= 1.5 * s16, (s_s, s16)
    assert e_s - e_b < 0.5 * (e16 - e_b), (e_b, e_s, e16)


@pytest.mark.parametrize("M", [2, 8])
def test_no_sync_from_one_entry_is_bfis(runs, M):
    """Algorithm 3 with R = inf never merges. Under the reading of the deal
    (only unchecked entries are dealt, and the first queue holds only P),
    walker 0 alone receives P, so the whole search is Algorithm 1: same ids,
    keys and distance count. (The paper's NoSync comparison, Table 2, cannot
    be reproduced in this form.)"""
    b, n = runs["bfis"], runs[f"nosync{M}"]
    np.testing.assert_array_equal(n[0], b[0])
    np.testing.assert_array_equal(n[1], b[1])
    np.testing.assert_array_equal(n[2]["evals"], b[2]["evals"])
