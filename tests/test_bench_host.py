"""Host-side pieces of the benchmark that need no GPU: the clock summary
that decides whether a timed run is kept, the peak table, the source hash
that gates the reported DRAM traffic and the recorded traffic itself."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_summary_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1995, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    c = bench.summarize_clocks(lines)
    assert c["samples"] == 3
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_slowdown():
    c = bench.summarize_clocks(["0, 1500, 2070, 1000, 0x20, Not Active, Active, Active, Not Active"])
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert bench.summarize_clocks([])["sm_mhz"] is None


def test_peaks_and_traffic_gate():
    pk = bench.peaks()
    assert pk["hbm_gbs"] > 1000 and pk["bf16_tflops"] > 100
    sha = bench.kernel_sha()
    assert len(sha) == 64 and int(sha, 16) >= 0
    M = N = bench.M
    for k, b in bench.TRAFFIC["bytes_per_launch"].items():
        alg = 4.0 * M * N + 2.0 * N * int(k) + 4.0 * M * int(k)
        assert 0.99 * alg <= b <= 1.1 * alg          # within 10 % of the algorithmic bytes


def test_clock_sampler_without_nvidia_smi(monkeypatch):
    monkeypatch.setenv("PATH", "/nonexistent")
    cs = bench.ClockSampler(0)
    cs.start()
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]
