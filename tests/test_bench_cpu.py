"""The arithmetic behind bench.py's roofline figures, on hand numbers (CPU;
the timed runs themselves need a GPU)."""
import pytest

pytest.importorskip("torch")

import bench  # noqa: E402


def test_march_roofline_arithmetic(monkeypatch):
    # 1e6 queries of 25 algorithmic bytes and 1e5 hits of 76 in 2 ms:
    # 32.6e6 B / 2e-3 s = 16.3 GB/s; against a 7600 GB/s peak, 0.00214
    monkeypatch.setattr(bench, "hbm_peak", lambda: (7600.0, "test"))
    r = bench.roofline_march([1.5, 2.5], 1_000_000, 100_000)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["ms_per_launch"] == pytest.approx(2.0)
    assert r["achieved"] == pytest.approx(
        (1e6 * bench.MARCH_BYTES_PER_QUERY + 1e5 * bench.MARCH_BYTES_PER_HIT) / 2e-3 / 1e9)
    assert r["achieved"] == pytest.approx(16.3)
    assert r["frac"] == pytest.approx(16.3 / 7600.0)
    assert r["launches_timed"] == 2
    if r["traffic"] is not None:
        assert r["traffic"] == pytest.approx(bench.MARCH_NCU_TRAFFIC["bytes_per_query"] * 1e6)
    assert bench.roofline_march([], 10) is None


def test_po_roofline_arithmetic():
    # 1e9 terms of 64 flops per launch in 2 ms: 32 TFLOP/s; against the FP32
    # peak at 2070 MHz (80.55 TFLOP/s), 0.397
    r = bench.roofline_po([1.0, 3.0], 1e9, "po_rot_kernel", 2070.0)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and r["kernel"] == "po_rot_kernel"
    assert r["ms_per_launch"] == pytest.approx(2.0)
    assert r["achieved"] == pytest.approx(1e9 * bench.PO_FLOPS_PER_TERM / 2e-3 / 1e12)
    assert r["achieved"] == pytest.approx(32.0)
    assert r["frac"] == pytest.approx(32.0 / (152 * 128 * 2 * 2.07e9 / 1e12))
    assert r["launches_timed"] == 2
    assert bench.roofline_po([], 1e9) is None
    assert bench.roofline_po([1.0], 0) is None


def test_alu_peak_from_the_sampled_clock():
    v, how = bench.alu_peak(2070.0)
    assert v == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)       # 80.55 TFLOP/s
    assert "2070" in how
    v2, how2 = bench.alu_peak(1455.0)
    assert v2 == pytest.approx(v * 1455.0 / 2070.0)
    assert bench.alu_peak(None)[0] == pytest.approx(v)             # maximum clock when unsampled


def test_oracle_query_count_matches_the_device_counters_rule():
    # 6 screen rays, mb = 3: M = 0 (primary miss), 1 (bounce-2 query misses),
    # 2 (bounce-3 query misses, shadow ray), 3 (stops at mb, shadow ray)
    M = [0, 1, 2, 3, 3, 1]
    # primary 6; bounce 2: rays with M >= 1 (5); bounce 3: rays with M >= 2
    # (3); shadow rays: M >= 2 (3)
    assert bench._angle_queries(M, 3, 6) == 6 + 5 + 3 + 3
    assert bench._angle_queries([1, 0], 1, 2) == 2
