"""Frame numerology and packet sizing (`paper_2604_02266_gb300/numerology.py`) against the
values Sec. VI-A prints (`tests/golden/numerology_sec6a.txt`) and the relations of
Eq. bandwidth_frametime and Eq. delay_Doppler_res."""

import importlib.util
import os

import pytest

from tests.golden import read_fixture

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _numerology():
    # plain arithmetic: loaded by path so the test needs neither the CUDA library nor a GPU
    spec = importlib.util.spec_from_file_location(
        "zotfs_numerology", os.path.join(ROOT, "paper_2604_02266_gb300", "numerology.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _f(fx, key):
    return float(fx[key][0][0])


def test_printed_numerology():
    nm = _numerology()
    fx = read_fixture("numerology_sec6a.txt")
    N, df = int(_f(fx, "N")), _f(fx, "delta_f_hz")
    p = nm.frame_numerology(64, N, df)
    assert p["doppler_res_hz"] == pytest.approx(_f(fx, "doppler_res_hz"), abs=0.005)
    assert p["frame_s"] * 1e3 == pytest.approx(_f(fx, "frame_ms"), abs=0.0005)
    assert nm.coherence_time(_f(fx, "nu_max_hz")) * 1e3 == pytest.approx(_f(fx, "coherence_ms"), abs=0.005)
    assert nm.packet_deadline(N, df) * 1e3 == pytest.approx(_f(fx, "two_frame_deadline_ms"), abs=0.005)


def test_resolution_relations():
    """Delay resolution x bandwidth = 1, Doppler resolution x frame duration = 1, and
    B T = M N (the grid's time-bandwidth product)."""
    nm = _numerology()
    for M, N, df in ((64, 32, 30e3), (16384, 32, 30e3), (128, 16, 15e3), (1, 1, 1.0)):
        p = nm.frame_numerology(M, N, df)
        assert p["delay_res_s"] * p["bandwidth_hz"] == pytest.approx(1.0)
        assert p["doppler_res_hz"] * p["frame_s"] == pytest.approx(1.0)
        assert p["bandwidth_hz"] * p["frame_s"] == pytest.approx(M * N)
        # M only sets the bandwidth: the frame duration is that of any other M
        assert p["frame_s"] == nm.frame_numerology(2 * M, N, df)["frame_s"]
    for bad in ((0, 32, 30e3), (64, 0, 30e3), (64, 32, 0.0)):
        with pytest.raises(ValueError):
            nm.frame_numerology(*bad)


def test_data_frames_per_pilot():
    """At the paper's nu_max = 100 Hz (T_c = 4.23 ms, T = 1.067 ms) a channel-static packet
    holds the pilot and 2 data frames; D grows as 1/nu_max, never drops below one data frame
    per pilot, and the packet of D data frames always fits in T_c when D > 1."""
    nm = _numerology()
    assert nm.data_frames_per_pilot(100.0, 32, 30e3) == 2
    assert nm.data_frames_per_pilot(44.0, 32, 30e3) == 8  # (1 + 8) T = 9.6 ms <= 0.423 / 44 Hz
    assert nm.data_frames_per_pilot(45.0, 32, 30e3) == 7
    assert nm.data_frames_per_pilot(1000.0, 32, 30e3) == 1  # T_c = 0.42 ms < T: the worst case
    prev = None
    for nu in (10.0, 20.0, 50.0, 100.0, 200.0, 400.0):
        D = nm.data_frames_per_pilot(nu, 32, 30e3)
        T = nm.frame_numerology(1, 32, 30e3)["frame_s"]
        if D > 1:
            assert (1 + D) * T <= nm.coherence_time(nu) < (2 + D) * T
        assert prev is None or D <= prev
        prev = D
    # a span that equals T_c exactly counts as fitting: T_c = 4 T at nu_max = 0.423 / (4 T)
    T = 32 / 30e3
    assert nm.data_frames_per_pilot(0.423 / (4 * T), 32, 30e3) == 3
    assert nm.packet_deadline(32, 30e3, 3) == pytest.approx(4 * T)
    with pytest.raises(ValueError):
        nm.packet_deadline(32, 30e3, 0)
    with pytest.raises(ValueError):
        nm.coherence_time(0.0)
