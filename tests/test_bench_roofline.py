"""bench.py's roofline arithmetic on the CPU, from a fixed set of kernel timings:
achieved bandwidth = algorithmic bytes / kernel time, the fraction of the peak,
the DRAM traffic scaled from a capture only while the kernel sources are the
captured ones, the latency-bound form of the L2-resident kernel, the FP64 ALU
form, and the per-outer-step averages."""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _job(ms0, bytes0, pixels0, launches0=4, ms1=1.0, flops1=0.0):
    return SimpleNamespace(timing={"launches": [launches0, 2], "ms": [ms0, ms1],
                                   "pixels": [pixels0, 100], "bytes": [bytes0, 0.0],
                                   "flops": [0.0, flops1], "phase_ms": {}})


def test_streaming_kernel_bandwidth_fraction_and_traffic(monkeypatch):
    wl = SimpleNamespace(radius=12, n=1000)
    peaks = {"hbm_gbs": 5000.0}
    monkeypatch.setattr(bench, "measured_peaks", lambda: (peaks, "measured"))
    # 8 GB in 2 ms over 4 launches of 50 steps each: 4000 GB/s, 0.8 of 5000
    job = _job(ms0=2.0, bytes0=8e9, pixels0=200 * 1000)
    e = bench.roofline_entry(job, 4.0, 2, wl, "mixed", (1.0, "x"), tuned_variant=2)
    assert e["kernel"] == "k_mr_tma<float,12>"
    assert e["stencil"] == "A as two autocorrelation passes"
    assert e["bound"] == "hbm" and e["unit"] == "GB/s"
    assert e["achieved"] == pytest.approx(4000.0)
    assert e["frac"] == pytest.approx(0.8)
    assert e["kernel_time_share_of_step"] == pytest.approx(0.5)
    assert e["algorithmic_bytes_per_launch"] == pytest.approx(2e9)
    assert e["us_per_minres_step"] == pytest.approx(2000.0 / 200)
    # the recorded capture applies only to the sources it was taken on
    cap = bench.TRAFFIC["k_mr_tma<float,12>"]
    if cap["src"] == bench.kernel_src_sha():
        assert e["traffic"] == pytest.approx(cap["dram_per_alg"] * 2e9)
    monkeypatch.setitem(bench.TRAFFIC, "k_mr_tma<float,12>", dict(cap, src="0" * 16))
    e = bench.roofline_entry(job, 4.0, 2, wl, "mixed", (1.0, "x"), tuned_variant=1)
    assert e["traffic"] is None and "changed" in e["traffic_source"]
    assert e["stencil"] == "A as four blur passes"


def test_resident_kernel_is_reported_per_step_not_against_hbm(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: ({"hbm_gbs": 5000.0}, "measured"))
    wl = SimpleNamespace(radius=8, n=100)
    e = bench.roofline_entry(_job(ms0=1.3, bytes0=1e9, pixels0=100 * 100), 2.0, 1, wl, "mixed", (1.0, "x"))
    assert e["kernel"] == "k_mr_resident<float,8>"
    assert e["bound"] == "latency" and e["frac"] is None
    assert e["us_per_minres_step"] == pytest.approx(13.0)
    assert "stencil" not in e


def test_fp64_residual_kernel_is_reported_against_the_fp64_rate(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: ({"hbm_gbs": 5000.0}, "measured"))
    wl = SimpleNamespace(radius=8, n=100)
    # the FP64 matvec dominates: 2e9 flop in 2 ms = 1 TFLOP/s against a 1.25 TFLOP/s peak
    job = _job(ms0=0.5, bytes0=1e6, pixels0=100, ms1=2.0, flops1=2e9)
    e = bench.roofline_entry(job, 4.0, 0, wl, "fp64", (1250.0, "measured"))
    assert e["bound"] == "alu" and e["unit"] == "TFLOP/s"
    assert e["achieved"] == pytest.approx(1.0)
    assert e["frac"] == pytest.approx(0.8)
    assert e["algorithmic_flops_per_launch"] == pytest.approx(1e9)


def test_per_k_averages_the_steps_of_each_outer_index():
    res = [{"k": 0}, {"k": 1}, {"k": 0}, {"k": 1}]
    assert bench.per_k([10.0, 4.0, 12.0, 6.0], res) == {"0": 11.0, "1": 5.0}
