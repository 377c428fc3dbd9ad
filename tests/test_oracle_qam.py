"""Pins for the oracle's QAM demapper: unit energy, Gray adjacency, brute-force argmin
(Eq. demod) versus LLR signs, the QPSK closed form, and the independent TX mapping."""

import numpy as np
import pytest

import synth
from oracle import qam


@pytest.mark.parametrize("Q", [4, 16, 64])
def test_unit_energy_and_gray_adjacency(Q):
    pts = qam.constellation(Q)
    assert np.isclose(np.mean(np.abs(pts) ** 2), 1.0, rtol=1e-12)
    bits = qam.label_bits(Q)
    d = np.abs(pts[:, None] - pts[None, :])
    dmin = d[d > 1e-12].min()
    for a in range(Q):
        for b in range(Q):
            if abs(d[a, b] - dmin) < 1e-9:
                assert (bits[a] != bits[b]).sum() == 1  # nearest neighbours differ in one bit


@pytest.mark.parametrize("Q", [4, 16, 64])
def test_llr_sign_equals_argmin(Q):
    g = np.random.default_rng(Q)
    x = (g.standard_normal(4000) + 1j * g.standard_normal(4000)) * 0.8
    lab, hb = qam.hard_demod(x, Q)
    llr = qam.maxlog_llr(x, 0.1, Q)
    assert (qam.hard_bits_from_llr(llr) == hb).all()


def test_qpsk_closed_form():
    """4-QAM: levels +-d with Gray label 1 at +d, so LLR_I = -4 d Re(x)/lambda, LLR_Q = -4 d Im(x)/lambda."""
    g = np.random.default_rng(1)
    x = g.standard_normal(100) + 1j * g.standard_normal(100)
    lam = 0.37
    d = 1 / np.sqrt(2)
    llr = qam.maxlog_llr(x, lam, 4)
    np.testing.assert_allclose(llr[:, 0], -4 * d * x.real / lam, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(llr[:, 1], -4 * d * x.imag / lam, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("Q", [4, 16, 64])
def test_tx_mapping_roundtrip(Q):
    """synth's TX mapping and the oracle's demapper agree on every label."""
    bps = int(np.log2(Q))
    g = np.random.default_rng(2)
    bits = g.integers(0, 2, size=300 * bps)
    sym = synth.qam_map(bits, Q)
    _, hb = qam.hard_demod(sym, Q)
    assert (hb.reshape(-1) == bits).all()


def test_tie_gives_zero():
    assert qam.hard_bits_from_llr(np.array([0.0, -0.0, 1e-30, -1e-30])).tolist() == [0, 0, 0, 1]


def test_pack_bits_lsb_first():
    assert qam.pack_bits([1, 0, 0, 0, 0, 0, 0, 0, 0, 1]).tolist() == [1, 2]
