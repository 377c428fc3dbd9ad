"""The bench's accounting, on the CPU: the algorithmic flops and HBM bytes per frame that its
roofline divides by, the ncu-summary reader behind `roofline.traffic`, and the clock-sample
summary that decides whether a run's clocks were clean."""

import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("zotfs_bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_flops_per_frame_at_the_benchmark_shape(bench):
    """64x32 16-QAM, P = 6, 10 iterations: the CG's MN [iters (16P + 24) + 8P + 4] =
    2,564,096 flops, plus two 32-point Doppler transforms (5 MN log2 N each) and the
    demapper's 8 sqrt(Q) flops per symbol."""
    cg = 2048 * (10 * (16 * 6 + 24) + 8 * 6 + 4)
    assert cg == 2564096
    assert bench.flops_per_frame(6) == cg + 2 * 5 * 2048 * 5 + 2048 * 8 * 4
    # each extra path costs one forward and one adjoint gather (8 flops each) per element and
    # iteration, plus the b = H^H y gather
    assert bench.flops_per_frame(7) - bench.flops_per_frame(6) == 2048 * (10 * 16 + 8)


def test_hbm_bytes_per_frame(bench):
    """Pilot and data TD frames in (complex64), float32 LLRs (4 per 16-QAM symbol), packed hard
    bits and the status word out; without LLRs only the bits and the status."""
    assert bench.hbm_bytes_per_frame() == 2 * 2048 * 8 + 2048 * 4 * 4 + 2048 * 4 // 8 + 4 == 66564
    assert bench.hbm_bytes_per_frame(llr=False) == 2 * 2048 * 8 + 2048 * 4 // 8 + 4 == 33796


def test_profiled_traffic_needs_a_matching_kernel_hash(bench, monkeypatch):
    real = bench.profiled_traffic()
    assert real is None or real > 0
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")
    assert bench.profiled_traffic() is None


def test_clock_summary(bench):
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 2040, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbled line"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.lines.append("0, 1500, 2070, 1400.0, 0x8, Active, Not Active, Active, Not Active")
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    c.lines = []
    assert c.summary()["reasons"] == ["no samples"]
