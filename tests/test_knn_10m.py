"""Spot check of the graph builder's k-NN lists at serving scale: the
brute-force kernel's 64 nearest neighbours of a sample of rows of the 10M x
96 BF16 point set, against the FP64 oracle over all 10M rows (Def. 1).

The rows are BF16-rounded unit vectors; a key is formed in FP32 as
|q|^2 + |x|^2 - 2<q, x>, so ids may swap only where the oracle's keys lie
within that form's FP32 error bound of each other. The sample is a
contiguous block of rows at a seeded offset (the rows are drawn i.i.d., so a
block is a random sample) of ANN_SPOT_SAMPLE rows (default 10,000).
"""
import os

import numpy as np
import pytest

import oracle

N = int(os.environ.get("ANN_SPOT_N", "10000000"))
SAMPLE = int(os.environ.get("ANN_SPOT_SAMPLE", "10000"))
K = 64


@pytest.mark.gpu
def test_knn_lists_of_the_10m_point_set_match_the_oracle():
    import torch
    from paper_2201_13007_gb300 import _abi, synth
    base, _ = synth.deep_bf16(N, 20_000)
    n, d = base.shape
    off = int(np.random.Generator(np.random.PCG64(23)).integers(0, n - SAMPLE))
    X = torch.from_numpy(base).cuda().to(torch.bfloat16).view(torch.int16)
    ids = torch.empty((SAMPLE, K), dtype=torch.int32, device="cuda")
    dist = torch.empty((SAMPLE, K), dtype=torch.float32, device="cuda")
    _abi.ann_knn_bf16(X.data_ptr(), n, d, X[off:off + SAMPLE].data_ptr(), SAMPLE, off, 0, K, ids.data_ptr(),
                      dist.data_ptr(), None)
    gi = ids.cpu().numpy().astype(np.int64)
    gd = dist.cpu().numpy()
    del X
    torch.cuda.empty_cache()

    q = base[off:off + SAMPLE]
    # K + 2 keys: after the query's own row, the 65th neighbour's key bounds the last rank's gap
    oi, ok = oracle.exact_knn_blocked(base, q, K + 2)
    norms = np.linalg.norm(base[:100_000].astype(np.float64), axis=1).max()
    tol = 2.0 * (d + 2) * 2.0 ** -24 * (2 * norms) ** 2
    identical = 0
    for r in range(SAMPLE):
        keep = oi[r] != off + r
        o_ids, o_keys, k_next = oi[r][keep][:K], ok[r][keep][:K], ok[r][keep][K]
        x = base[gi[r]].astype(np.float64)
        exact = ((x - q[r].astype(np.float64)) ** 2).sum(1)
        assert off + r not in gi[r]
        assert np.unique(gi[r]).size == K
        assert np.all(np.abs(gd[r] - exact) <= tol / 2), r
        assert np.all(np.abs(exact - o_keys) <= tol), r
        gap_lo = np.r_[np.inf, np.diff(o_keys)]
        gap_hi = np.r_[np.diff(o_keys), k_next - o_keys[-1]]
        clear = (gap_lo > tol) & (gap_hi > tol)
        assert np.array_equal(gi[r][clear], o_ids[clear]), r
        identical += int(np.array_equal(gi[r], o_ids))
    print(f"spot check: {SAMPLE} rows at offset {off} of {n}; {identical} identical to the oracle in order, "
          f"the rest differ only by swaps inside the FP32 window {tol:.2e}")
    assert identical >= 0.9 * SAMPLE
