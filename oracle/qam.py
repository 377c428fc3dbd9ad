"""Square Gray QAM, hard demodulation and max-log LLRs, FP64.

Test infrastructure only (see :mod:`oracle`).

The paper uses hard demodulation (Eq. demod: argmin_s |x - s|^2, then demap to bits) and
does not fix the bit labelling.  Readings used here:

* square Q-QAM (Q in {4, 16, 64}) as two sqrt(Q)-PAM axes with levels
  (2i - (sqrt(Q) - 1)) d, d chosen so that the mean symbol energy E_s = 1;
* each axis labelled with the binary-reflected Gray code g = i ^ (i >> 1);
* a symbol's bits are the I-axis label (MSB first) followed by the Q-axis label;
* the max-log LLR of bit j (not in the paper) is
  (min_{s: b_j(s) = 1} |x - s|^2 - min_{s: b_j(s) = 0} |x - s|^2) / lambda,
  so LLR > 0 favours bit 0; the hard bit is (LLR < 0) and an exact tie gives bit 0.
"""

import numpy as np


def bits_per_symbol(Q):
    b = int(round(np.log2(Q)))
    if Q not in (4, 16, 64):
        raise ValueError("square QAM with Q in {4, 16, 64}")
    return b


def pam_levels(Q):
    """Level index i -> amplitude (2i - (m-1)) d for m = sqrt(Q), with E_s = 1."""
    m = int(round(np.sqrt(Q)))
    d = np.sqrt(3.0 / (2.0 * (Q - 1)))
    return (2 * np.arange(m) - (m - 1)) * d


def _gray(i):
    return i ^ (i >> 1)


def constellation(Q):
    """Points s[label] for label in [0, Q): label = (Gray(i_I) << h) | Gray(i_Q), h = log2(Q)/2."""
    b = bits_per_symbol(Q)
    h = b // 2
    m = 1 << h
    lev = pam_levels(Q)
    pts = np.zeros(Q, np.complex128)
    for iI in range(m):
        for iQ in range(m):
            label = (_gray(iI) << h) | _gray(iQ)
            pts[label] = lev[iI] + 1j * lev[iQ]
    return pts


def label_bits(Q):
    """(Q, bps) array: bit j of each label, MSB first."""
    b = bits_per_symbol(Q)
    lab = np.arange(Q)[:, None]
    return (lab >> (b - 1 - np.arange(b))[None, :]) & 1


def hard_demod(x, Q):
    """Eq. demod: nearest constellation point, returned as (labels, bits[len(x), bps])."""
    x = np.asarray(x, np.complex128).reshape(-1)
    pts = constellation(Q)
    d2 = np.abs(x[:, None] - pts[None, :]) ** 2
    lab = np.argmin(d2, axis=1)
    return lab, label_bits(Q)[lab]


def maxlog_llr(x, lam, Q):
    """Max-log LLRs by brute force over all Q points: shape (len(x), bps)."""
    x = np.asarray(x, np.complex128).reshape(-1)
    pts = constellation(Q)
    bits = label_bits(Q)
    d2 = np.abs(x[:, None] - pts[None, :]) ** 2  # (n, Q)
    b = bits.shape[1]
    out = np.empty((len(x), b))
    for j in range(b):
        one = bits[:, j] == 1
        out[:, j] = (d2[:, one].min(axis=1) - d2[:, ~one].min(axis=1)) / lam
    return out


def hard_bits_from_llr(llr):
    """Hard bit = (LLR < 0); an exact tie gives 0."""
    return (np.asarray(llr) < 0).astype(np.uint8)


def pack_bits(bits):
    """Pack a flat 0/1 bit stream LSB-first into bytes (bit b -> byte b // 8, position b % 8)."""
    bits = np.asarray(bits, np.uint8).reshape(-1)
    return np.packbits(bits, bitorder="little")


__all__ = ["bits_per_symbol", "pam_levels", "constellation", "label_bits", "hard_demod",
           "maxlog_llr", "hard_bits_from_llr", "pack_bits"]
