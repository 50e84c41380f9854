"""Brute-force k-NN kernel (graph construction, Def. 1 of Sec. 2.1) against
the FP64 oracle.

Integer-valued rows (0..255, d <= 128) make every product and partial sum
an integer below 2^24, so the kernel's FP32 keys are exact and the result
must equal the oracle's bit for bit, ties broken by id. BF16-rounded unit
vectors are compared under the FP32 error bound of a key formed as
|q|^2 + |x|^2 - 2<q, x>: ids may swap only inside that window.
"""
import numpy as np
import pytest

import oracle

K_MAX = 64


def _bf16(x):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, np.float32)).to(torch.bfloat16)
    return t.to(torch.float32).numpy(), t.view(torch.int16)


def _gpu_knn(base_bits, q_bits, self_offset, metric, k):
    import torch
    from paper_2201_13007_gb300 import _abi
    b = base_bits.cuda().contiguous()
    q = q_bits.cuda().contiguous()
    n, d = b.shape
    nq = q.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device="cuda")
    dist = torch.empty((nq, k), dtype=torch.float32, device="cuda")
    _abi.ann_knn_bf16(b.data_ptr(), n, d, q.data_ptr(), nq, self_offset, 0 if metric == "l2" else 1, k,
                      ids.data_ptr(), dist.data_ptr(), None)
    torch.cuda.synchronize()
    return ids.cpu().numpy().astype(np.int64), dist.cpu().numpy()


def _oracle_knn(base, q, self_offset, metric, k, extra=0):
    """Oracle answer with each query's own row removed when the queries are
    rows of the base set; `extra` more keys past the k-th (+inf if none)."""
    n = base.shape[0]
    kk = min(k + extra + 1, n) if self_offset >= 0 else min(k + extra, n)
    ids, keys = oracle.exact_knn(base, q, kk, metric=metric, nthreads=8)
    out_i = np.full((q.shape[0], k + extra), -1, np.int64)
    out_k = np.full((q.shape[0], k + extra), np.inf)
    for r in range(q.shape[0]):
        m = ids[r] >= 0
        if self_offset >= 0:
            m &= ids[r] != self_offset + r
        ii, kv = ids[r][m][:k + extra], keys[r][m][:k + extra]
        out_i[r, :ii.size] = ii
        out_k[r, :kv.size] = kv
    return out_i, out_k


def _integer_rows(n, d, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    centres = g.integers(0, 256, (16, d))
    lab = g.integers(0, 16, n)
    x = np.clip(centres[lab] + g.normal(0, 30, (n, d)).round(), 0, 255)
    x[5::97] = x[4::97][: x[5::97].shape[0]]  # exact duplicates: ties resolved by id
    return x.astype(np.float32)


def _unit_rows(n, d, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    centres = g.standard_normal((32, d))
    x = centres[g.integers(0, 32, n)] + 0.5 * g.standard_normal((n, d))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x.astype(np.float32)


CASES = [
    # (d, metric, n, queries, k): queries = ("self", lo, hi) rows of the base, or ("new", count)
    (96, "l2", 5000, ("self", 1000, 1300), 64),
    (128, "l2", 4097, ("new", 129), 64),
    (64, "ip", 3000, ("new", 257), 10),
    (32, "l2", 2000, ("self", 0, 2000), 33),
    (96, "ip", 2500, ("self", 2300, 2500), 64),
    (96, "l2", 40, ("self", 0, 40), 64),   # fewer rows than k: (-1, +inf) padding
    (128, "l2", 127, ("new", 1), 5),
]


def _setup(case, rows):
    d, metric, n, qs, k = case
    base, bits = _bf16(rows(n, d, 10 + d + n))
    if qs[0] == "self":
        lo, hi = qs[1], qs[2]
        return base, bits, base[lo:hi], bits[lo:hi], lo, metric, k
    q, qbits = _bf16(rows(qs[1], d, 20 + d))
    return base, bits, q, qbits, -1, metric, k


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=[f"d{c[0]}-{c[1]}-n{c[2]}-{c[3][0]}-k{c[4]}" for c in CASES])
def test_knn_integer_rows_bit_exact(case):
    base, bits, q, qbits, self_offset, metric, k = _setup(case, _integer_rows)
    gi, gd = _gpu_knn(bits, qbits, self_offset, metric, k)
    oi, ok = _oracle_knn(base, q, self_offset, metric, k)
    assert np.array_equal(gi, oi)
    fin = np.isfinite(ok)
    assert np.array_equal(np.isfinite(gd), fin)
    assert np.array_equal(gd[fin].astype(np.float64), ok[fin])


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES[:5], ids=[f"d{c[0]}-{c[1]}-n{c[2]}-{c[3][0]}-k{c[4]}" for c in CASES[:5]])
def test_knn_unit_rows_within_fp32_bound(case):
    base, bits, q, qbits, self_offset, metric, k = _setup(case, _unit_rows)
    d = base.shape[1]
    gi, gd = _gpu_knn(bits, qbits, self_offset, metric, k)
    oi, ok_all = _oracle_knn(base, q, self_offset, metric, k, extra=1)
    oi, ok, k_next = oi[:, :k], ok_all[:, :k], ok_all[:, k]
    # FP32 error of |q|^2 + |x|^2 - 2<q, x> (or -<q, x>) for unit-norm rows:
    # at most (d + 2) u (|q| + |x|)^2 = 4 (d + 2) u; swaps need twice that.
    tol = 2.0 * 4.0 * (d + 2) * 2.0 ** -24
    n = base.shape[0]
    for r in range(q.shape[0]):
        ids = gi[r]
        assert np.all((ids >= 0) & (ids < n))
        assert np.unique(ids).size == k
        if self_offset >= 0:
            assert self_offset + r not in ids
        x = base[ids].astype(np.float64)
        qq = q[r].astype(np.float64)
        exact = ((x - qq) ** 2).sum(1) if metric == "l2" else -(x @ qq)
        assert np.all(np.abs(gd[r] - exact) <= tol / 2), r
        assert np.all(np.abs(exact - ok[r]) <= tol), r
        # a rank whose oracle key stands clear of both neighbours must hold the same id
        kr = ok[r]
        gap_lo = np.r_[np.inf, np.diff(kr)]
        gap_hi = np.r_[np.diff(kr), k_next[r] - kr[-1]]  # the last rank against the (k+1)-th key
        clear = (gap_lo > tol) & (gap_hi > tol)
        assert np.array_equal(ids[clear], oi[r][clear]), r


@pytest.mark.gpu
def test_knn_argument_errors():
    import torch
    from paper_2201_13007_gb300 import _abi
    b = torch.zeros((256, 96), dtype=torch.int16, device="cuda")
    ids = torch.empty((4, 8), dtype=torch.int32, device="cuda")
    dist = torch.empty((4, 8), dtype=torch.float32, device="cuda")
    bad = [
        dict(d=80), dict(k=0), dict(k=65), dict(metric=2), dict(self_offset=253), dict(n=0),
    ]
    for kw in bad:
        a = dict(n=256, d=96, nq=4, self_offset=-1, metric=0, k=8)
        a.update(kw)
        with pytest.raises(_abi.AnnError):
            _abi.ann_knn_bf16(b.data_ptr(), a["n"], a["d"], b.data_ptr(), a["nq"], a["self_offset"], a["metric"],
                              a["k"], ids.data_ptr(), dist.data_ptr(), None)
    with pytest.raises(_abi.AnnError):  # misaligned base
        _abi.ann_knn_bf16(b.data_ptr() + 2, 255, 96, b.data_ptr(), 4, -1, 0, 8, ids.data_ptr(), dist.data_ptr(),
                          None)
