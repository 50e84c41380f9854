"""Comparison rules between the CUDA path and the FP64 oracle.

Float workloads: ids must equal the oracle's, except that a mismatched id is
accepted when its FP64 key is within ``rel`` (1e-5) of the oracle's key at the
same rank (a swap among near-equal distances); GPU keys (FP32) must be within
``rel`` of the FP64 key of the id they report. Queries on which the oracle
logged a near-tie at a selection, truncation or output boundary may take a
different trajectory under FP32 rounding; they are reported separately and
judged by recall against the oracle's answer, and at least 90% of all rows
must match. The near-tie window passed to the oracle is the FP32 error bound
of the key (fp32_tie_window). For inner product the key tolerance is taken
relative to |q| |x| rather than |key|, since the dot product cancels.

Integer-valued workloads (0..255, d <= 128, FP32 or BF16 storage): every
partial sum is an integer below 2^24, so FP32 accumulation is exact in any
order and the comparison is bit-exact: ids and keys identical.
"""
import numpy as np


def fp64_keys(base, q, ids, metric):
    out = np.full(ids.shape, np.inf)
    for i in range(ids.shape[0]):
        m = ids[i] >= 0
        x = base[ids[i][m]].astype(np.float64)
        qq = q[i].astype(np.float64)
        if metric == "l2":
            out[i, m] = ((x - qq) ** 2).sum(1)
        else:
            out[i, m] = -(x @ qq)
    return out


def _close(a, b, rel, floor):
    both_inf = np.isinf(a) & np.isinf(b)
    return both_inf | (np.abs(a - b) <= rel * np.maximum(np.maximum(np.abs(a), np.abs(b)), floor))


def fp32_tie_window(base, q, metric):
    """(relative, absolute) window in which FP32 rounding can swap two keys.
    A squared-L2 key is a sum of d non-negative terms, each the rounded square
    of a rounded difference: relative error <= (d + 2) u, u = 2^-24. An
    inner-product key has absolute error <= d u sum|q_i x_i| <= d u |q| |x|.
    Two keys can only swap order when their gap is below twice the bound."""
    d = base.shape[1]
    u = 2.0 ** -24
    if metric == "l2":
        return 2.0 * (d + 2) * u, 0.0
    bound = float(np.linalg.norm(q, axis=1).max() * np.linalg.norm(base, axis=1).max())
    return 0.0, 2.0 * (d + 2) * u * bound


def compare_float(gpu_ids, gpu_keys, orc_ids, orc_keys, tie_events, base, q, metric, rel=1e-5,
                  min_tie_recall=0.9, min_match_frac=0.9):
    """Returns a report dict; asserts the rules in the module docstring."""
    gpu_ids = np.asarray(gpu_ids)
    gpu_keys = np.asarray(gpu_keys, np.float64)
    k64 = fp64_keys(base, q, gpu_ids, metric)
    # key scale: |key| for L2; |q| |x| for inner product (cancellation)
    if metric == "l2":
        floor = 1e-6
    else:
        floor = float(np.linalg.norm(q, axis=1).max() * np.linalg.norm(base, axis=1).max())
    ok_keys = _close(gpu_keys, k64, rel, floor)
    assert ok_keys.all(), f"GPU keys off by more than {rel} relative at {np.argwhere(~ok_keys)[:5]}"
    clean = np.asarray(tie_events) == 0
    same = gpu_ids == orc_ids
    swap_ok = _close(k64, orc_keys, rel, floor)
    good_rows = (same | swap_ok).all(1)
    bad_rows = np.flatnonzero(clean & ~good_rows)
    assert bad_rows.size == 0, (
        f"{bad_rows.size} tie-free queries differ from the oracle, e.g. row {bad_rows[0]}: "
        f"gpu {gpu_ids[bad_rows[0]].tolist()} oracle {orc_ids[bad_rows[0]].tolist()}")
    tie_rows = np.flatnonzero(~clean)
    rec = 1.0
    if tie_rows.size:
        rec = float(np.mean([len(set(gpu_ids[r].tolist()) & set(orc_ids[r].tolist())) / orc_ids.shape[1]
                             for r in tie_rows]))
        assert rec >= min_tie_recall, f"recall vs oracle on near-tie queries {rec}"
    frac = float(good_rows.mean())
    assert frac >= min_match_frac, f"only {frac:.3f} of the queries match the oracle"
    return {"tie_free": int(clean.sum()), "tie_rows": int(tie_rows.size), "match_frac": frac,
            "tie_recall": rec}


def compare_exact(gpu_ids, gpu_keys, orc_ids, orc_keys):
    np.testing.assert_array_equal(np.asarray(gpu_ids), np.asarray(orc_ids))
    g = np.asarray(gpu_keys, np.float64)
    o = np.asarray(orc_keys, np.float64)
    np.testing.assert_array_equal(g, o)
