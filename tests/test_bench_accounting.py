"""The bench's accounting, on the CPU: the algorithmic flops and HBM bytes per frame that its
roofline divides by, the ncu-summary reader behind `roofline.traffic`, the clock-sample
summary that decides whether a run's clocks were clean, and the BER sweep's bookkeeping (bit
error counting, its LMMSE leg, the claims it checks)."""

import importlib.util
import os

import numpy as np

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


def test_bit_error_counting_reads_lsb_first_packing(bench):
    g = np.random.default_rng(4)
    tx = g.integers(0, 2, size=(3, 64)).astype(np.uint8)
    packed = np.packbits(tx, axis=1, bitorder="little")  # the library's order: bit b -> byte b/8, position b%8
    assert (bench.bit_errors(packed, tx, 3) == 0).all()
    flipped = tx.copy()
    flipped[1, [0, 9, 63]] ^= 1
    assert bench.bit_errors(np.packbits(flipped, axis=1, bitorder="little"), tx, 3).tolist() == [0, 3, 0]


def test_lmmse_leg_matches_cg_to_convergence_and_recovers_noiseless_frames(bench):
    """The sweep's LMMSE leg (dense Eq. Hdd + Cholesky on a given list) decides like the
    oracle's CG run to convergence, and returns the transmitted bits of a noiseless
    integer-offset frame."""
    import synth
    from oracle import equalizer as eq, qam, receiver
    M, N, Q = 16, 16, 16
    b = synth.fractional_batch(2, seed=21, M=M, N=N, Q=Q, snr_db=(60,), integer=True)
    b2 = synth.veh_a_batch(2, 22, M=M, N=N, Q=Q, snr_db=(10,))
    for bb, noiseless in ((b, True), (b2, False)):
        for f in range(2):
            r = receiver.receive(bb["y_pilot_td"][f], bb["y_data_td"][f], M, N, 1, 1, Q, float(bb["noise_var"][f]),
                                 float(bb["theta"][f]), 10, bb["a_pilot"], p_max=64)
            pl = r["paths"][0][0]
            bits = bench._lmmse_bits(bb["y_data_td"][f, 0], pl.dk, pl.dl, pl.h, M, N, Q, float(bb["noise_var"][f]))
            x, _ = eq.cg_to_convergence([[pl]], r["y_dd"], float(bb["noise_var"][f]))
            assert np.array_equal(bits, qam.hard_demod(x, Q)[1].reshape(-1))
            if noiseless:
                assert np.array_equal(bits, bb["bits"][f].reshape(-1))


def test_ber_claims_bookkeeping(bench):
    row = lambda c, l, m, nb=100000, c20=None: {"ber_cga": c, "ber_cga20": c if c20 is None else c20, "ber_lmmse": l,
                                                 "ber_mrc": m, "bits": nb, "M": 32, "N": 32, "qam": 4, "snr_db": 10}
    ok = bench.ber_claims([row(0.01, 0.01, 0.05), row(0.002, 0.0015, 0.01), row(0.0, 0.0, 0.0)])
    assert ok["cga_within_factor_of_lmmse"] and ok["cga20_within_factor_of_lmmse"] and ok["cga_at_or_below_mrc"]
    assert ok["cga_points_compared"] == 2 and abs(ok["worst_ratio_cga_lmmse"] - 0.002 / 0.0015) < 1e-12
    bad = bench.ber_claims([row(0.05, 0.01, 0.06, c20=0.015)])
    assert bad["cga_within_factor_of_lmmse"] is False and bad["cga20_within_factor_of_lmmse"] is True
    # points resting on fewer than min_errors bit errors decide nothing
    few = bench.ber_claims([row(0.00015, 0.00001, 0.0001)])
    assert few["cga_points_compared"] == 0 and few["cga_within_factor_of_lmmse"] is None
    # SS-CGA above SS-MRC only counts beyond the binomial noise of the difference
    assert bench.ber_claims([row(0.0340, 0.034, 0.0322, nb=65536)])["cga_at_or_below_mrc"]
    assert not bench.ber_claims([row(0.0400, 0.04, 0.0322, nb=65536)])["cga_at_or_below_mrc"]
