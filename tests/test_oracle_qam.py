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


def test_16qam_closed_form():
    """16-QAM, per axis u (Re x for the I bits, Im x for the Q bits), levels -3d, -d, d, 3d with
    Gray labels 00, 01, 11, 10 and d = 1/sqrt(10): the max-log LLRs are the piecewise-linear
    forms derived by hand from the nearest level of each label class --
    sign bit: -4 d u / lambda for |u| <= 2d, else -8 d (u - d sgn u) / lambda;
    second bit: 4 d (|u| - 2d) / lambda."""
    g = np.random.default_rng(16)
    x = (g.standard_normal(2000) + 1j * g.standard_normal(2000)) * 0.9
    lam = 0.23
    d = 1 / np.sqrt(10)

    def axis(u):
        msb = np.where(np.abs(u) <= 2 * d, -4 * d * u, -8 * d * (u - d * np.sign(u))) / lam
        lsb = 4 * d * (np.abs(u) - 2 * d) / lam
        return msb, lsb
    llr = qam.maxlog_llr(x, lam, 16)
    for col, ref in zip(range(4), (*axis(x.real), *axis(x.imag))):
        np.testing.assert_allclose(llr[:, col], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("Q", [16, 64])
def test_llr_axis_separability_and_reflection_symmetry(Q):
    """Square Gray QAM labelled I-axis first: the I bits' LLRs depend on Re x only and the Q
    bits' on Im x only; mirroring an axis negates its sign bit's LLR and leaves the other bits'
    unchanged (the reflected Gray code's symmetry)."""
    h = int(np.log2(Q)) // 2
    g = np.random.default_rng(Q + 1)
    x = (g.standard_normal(500) + 1j * g.standard_normal(500)) * 0.9
    other = (g.standard_normal(500) + 1j * g.standard_normal(500)) * 0.9
    lam = 0.4
    a = qam.maxlog_llr(x, lam, Q)
    np.testing.assert_allclose(qam.maxlog_llr(x.real + 1j * other.imag, lam, Q)[:, :h], a[:, :h], atol=1e-12)
    np.testing.assert_allclose(qam.maxlog_llr(other.real + 1j * x.imag, lam, Q)[:, h:], a[:, h:], atol=1e-12)
    m = qam.maxlog_llr(-x.real + 1j * x.imag, lam, Q)
    np.testing.assert_allclose(m[:, 0], -a[:, 0], atol=1e-12)
    np.testing.assert_allclose(m[:, 1:], a[:, 1:], atol=1e-12)


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
