"""Host logic of bench.py (no GPU): the algorithmic byte model and roofline arithmetic of the
bench line, the comment-blind source hash that ties a committed ncu summary to the kernels it was
taken on, the summary's parser, and the clock-record summary that decides whether a run is kept."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_model():
    # 28 B per bead-update (24-byte position + 4-byte link read), 24 B per moved bead written,
    # 28 B per partner evaluated outside the support
    assert bench.alg_bytes(1, 0, 0) == 28.0
    assert bench.alg_bytes(0, 1, 0) == 24.0
    assert bench.alg_bytes(0, 0, 1) == 28.0
    assert bench.alg_bytes(10, 3, 7) == 28.0 * 10 + 24.0 * 3 + 28.0 * 7


def test_roofline_block_arithmetic():
    # 48 launches moving 10 MB each in 96 ms: 480 MB / 0.096 s = 5 GB/s
    r = bench.roofline_block("k", 48 * 10e6, 96.0, 48, 6770.1, "measured", traffic=3.2e7)
    assert r["achieved"] == pytest.approx(5.0)
    assert r["frac"] == pytest.approx(5.0 / 6770.1)
    assert r["alg_bytes_per_launch"] == pytest.approx(10e6)
    assert r["avg_launch_us"] == pytest.approx(2000.0)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] == 3.2e7
    assert bench.roofline_block("k", 1.0, 0.0, 0, 1.0, "fallback")["achieved"] == 0.0


def test_source_hash_ignores_comments_and_blank_lines_only():
    a = "int x = 1;\n__global__ void k() {}\n"
    b = "// a note\nint x = 1;   // why\n\n__global__ void k() {}\n"
    c = "int x = 2;\n__global__ void k() {}\n"
    assert bench.code_sha([a]) == bench.code_sha([b])
    assert bench.code_sha([a]) != bench.code_sha([c])
    assert bench.code_sha([a, c]) != bench.code_sha([c, a])


def test_profile_traffic_only_for_the_source_it_was_taken_on(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "wavelet_concurrent_suspension.md").write_text(
        "# summary\n\n- kernel_source_sha256: `abc123`\n- dram_bytes_per_launch: 32275000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_traffic("abc123") == 32275000.0
    assert bench.profile_traffic("def456") is None
    (prof / "wavelet_concurrent_suspension.md").unlink()
    assert bench.profile_traffic("abc123") is None


def test_clock_summary_reports_median_and_active_reasons():
    c = bench.ClockSampler(0)
    c.rows = [["2070", "2070", "900.1", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["2055", "2070", "1390.0", "Not Active", "Not Active", "Not Active", "Active"],
              ["2070", "2070", "1400.0", "Not Active", "Active", "Not Active", "Active"],
              ["[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]", "[N/A]"]]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.ClockSampler(0).summary()["reasons"] == ["unavailable"]
