"""Host-side logic of bench.py on the CPU: the method's byte count, the
operating-point choice, the clock summary and the ncu traffic record."""
import json
import types

import numpy as np
import pytest

import bench


def test_algorithmic_bytes_follows_the_byte_formula():
    # columns: steps, expansions, evals, ...
    st = np.zeros((3, 8), np.int64)
    st[:, 1] = [10, 20, 30]
    st[:, 2] = [100, 200, 300]
    R, row, d, k, rr = 32, 256, 128, 10, 576
    want = sum(e * R * 4 + v * row + rr * d * 4 + d * 4 + k * 12 for e, v in zip([10, 20, 30], [100, 200, 300]))
    assert bench.algorithmic_bytes(st, R, row, d, k, rr) == pytest.approx(want)


def test_recall_counts_set_overlap_per_row():
    ids = np.array([[1, 2, 3], [4, 5, 6]])
    gt = np.array([[3, 2, 9], [7, 8, 9]])
    assert bench.recall_at_k(ids, gt) == pytest.approx(2 / 6)


class _FakeTorch:
    class cuda:
        @staticmethod
        def synchronize():
            pass


def test_cheapest_points_takes_the_fastest_point_that_reaches_each_target(monkeypatch):
    gt = np.arange(40).reshape(4, 10)
    recall_of = {(16, 4): 0.5, (32, 4): 0.92, (64, 4): 0.995, (16, 8): 0.91, (32, 8): 0.99, (64, 8): 0.999}
    cost_of = {(16, 4): 1.0, (32, 4): 2.0, (64, 4): 4.0, (16, 8): 1.5, (32, 8): 3.0, (64, 8): 6.0}
    clock = {"t": 0.0}

    def search(q, L, M):
        clock["t"] += cost_of[(L, M)]
        hits = int(round(recall_of[(L, M)] * 10))
        return types.SimpleNamespace(cpu=lambda: types.SimpleNamespace(
            numpy=lambda: np.where(np.arange(10)[None, :] < hits, gt, -1)))

    monkeypatch.setattr(bench.time, "perf_counter", lambda: clock["t"])
    pts = bench.cheapest_points(_FakeTorch, search, None, gt, (16, 32, 64), (4, 8), (0.9, 0.99), k=10)
    # the fake quantises recall to tenths: for 0.9, (16, 8) at cost 1.5 beats (32, 4) at 2.0; for 0.99
    # (10 of 10 hits), (32, 8) at cost 3.0 beats (64, 4) at 4.0
    assert pts[0.9][:2] == (16, 8)
    assert pts[0.99][:2] == (32, 8)


def test_cheapest_points_falls_back_to_the_best_recall_when_a_target_is_out_of_reach(monkeypatch):
    gt = np.arange(10).reshape(1, 10)
    monkeypatch.setattr(bench.time, "perf_counter", lambda: 0.0)

    def search(q, L, M):
        hits = {16: 5, 32: 7}[L]
        return types.SimpleNamespace(cpu=lambda: types.SimpleNamespace(
            numpy=lambda: np.where(np.arange(10)[None, :] < hits, gt, -1)))

    pts = bench.cheapest_points(_FakeTorch, search, None, gt, (16, 32), (4,), (0.9,), k=10)
    assert pts[0.9] == (32, 4, 0.7)


def test_clock_summary_parses_samples_and_active_reasons():
    c = bench.ClockSampler(0)
    c.lines = [
        "0, 2070, 2070, 900.1, 0x0000, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1380.0, 0x0004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    s = c.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.ClockSampler(0).summary()["samples"] == 0


def test_traffic_record_is_used_only_for_the_same_launch_and_sources(tmp_path, monkeypatch):
    rec = tmp_path / "traffic.json"
    label = "sync_search_kernel<256, BF16>, grid 608, 43776 B shared, 2^12 visited slots of 4 B"
    rec.write_text(json.dumps({"config": label, "sources": bench.kernel_sources_digest(),
                               "dram_bytes_per_launch": 1.5e10}))
    monkeypatch.setattr(bench, "TRAFFIC_SIDECAR", str(rec))
    assert bench.profiled_traffic(label) == 1.5e10
    assert bench.profiled_traffic(label.replace("608", "456")) is None
    rec.write_text(json.dumps({"config": label, "sources": "0" * 16, "dram_bytes_per_launch": 1.5e10}))
    assert bench.profiled_traffic(label) is None
    monkeypatch.setattr(bench, "TRAFFIC_SIDECAR", str(tmp_path / "missing.json"))
    assert bench.profiled_traffic(label) is None


def test_the_committed_traffic_record_matches_the_current_kernel_sources():
    rec = json.load(open(bench.TRAFFIC_SIDECAR))
    assert rec["sources"] == bench.kernel_sources_digest()
    assert rec["dram_bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
