"""Pins of the oracle's storage formats against torch's own CPU conversions
(round to nearest, ties to even) and the definitions of the formats."""
import numpy as np
import pytest
import torch


def _samples():
    r = np.random.default_rng(0)
    x = np.concatenate([
        r.standard_normal(20000) * 10.0 ** r.integers(-8, 8, 20000),
        np.arange(0, 256, dtype=np.float64),             # integers 0..255
        [0.0, -0.0, 1.0, -1.0, 65504.0, 65519.0, 6.1e-5, 5.96e-8, 1e-40],
    ]).astype(np.float32)
    # exact ties: midpoints between neighbouring bf16 values
    mids = (np.arange(1, 200, dtype=np.float32) * 2 + 1) * np.float32(2.0 ** -8)
    return np.concatenate([x, mids, -mids])


def test_bf16_matches_torch(oracle_mod):
    x = _samples()
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle_mod.round_bf16(x), want)


def test_fp16_matches_torch(oracle_mod):
    x = _samples()
    x = x[np.abs(x) < 1e5]
    want = torch.from_numpy(x).to(torch.float16).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle_mod.round_fp16(x), want)


def test_e4m3_matches_torch_in_range(oracle_mod):
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    r = np.random.default_rng(1)
    x = np.concatenate([r.uniform(-448, 448, 20000), r.standard_normal(5000) * 1e-2,
                        [0.0, 448.0, -448.0, 2.0 ** -9, 2.0 ** -10, 3 * 2.0 ** -10]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle_mod.round_e4m3(x), want)


def test_e4m3_saturates(oracle_mod):
    out = oracle_mod.round_e4m3(np.array([500.0, -1e9, 464.0], np.float32))
    assert out.tolist() == [448.0, -448.0, 448.0]


def test_integers_0_255_exact_in_bf16_and_fp16(oracle_mod):
    x = np.arange(256, dtype=np.float32)
    np.testing.assert_array_equal(oracle_mod.round_bf16(x), x)
    np.testing.assert_array_equal(oracle_mod.round_fp16(x), x)


def test_fp8_scaled_rows(oracle_mod):
    r = np.random.default_rng(3)
    x = np.abs(r.standard_normal((50, 33))).astype(np.float32)
    x[4] = 0.0
    deq, sc = oracle_mod.fp8_scaled(x)
    mx = np.abs(x).max(1)
    np.testing.assert_array_equal(sc[mx > 0], (mx[mx > 0] / np.float32(448.0)).astype(np.float32))
    assert sc[4] == 1.0 and (deq[4] == 0).all()
    # the largest element of each row is coded as 448 and comes back as scale*448
    i = np.argmax(np.abs(x), 1)
    got = deq[np.arange(50), i]
    np.testing.assert_allclose(got, x[np.arange(50), i], rtol=2 ** -20)
    # every dequantised value is scale * (an E4M3 value)
    codes = deq / sc[:, None]
    np.testing.assert_allclose(oracle_mod.round_e4m3(codes), codes, rtol=1e-6)
    # E4M3 has 3 mantissa bits: relative error <= 2^-4 for normal codes
    big = np.abs(x) > sc[:, None] * 2 ** -6
    assert (np.abs(deq - x)[big] <= np.abs(x)[big] * 2 ** -4 + 1e-30).all()
