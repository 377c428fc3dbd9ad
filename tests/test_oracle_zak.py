"""Pins for the oracle's Zak transform pair (Eq. iZak, Eq. zak) against closed forms and an
independent implementation (the transmitter in ``synth``)."""

import numpy as np
import pytest

import synth
from oracle import zak

SHAPES = [(8, 2), (4, 4), (16, 16), (64, 32), (32, 64)]


@pytest.mark.parametrize("M,N", SHAPES)
def test_roundtrip_both_ways(M, N):
    g = np.random.default_rng(M * 1000 + N)
    X = g.standard_normal((M, N)) + 1j * g.standard_normal((M, N))
    assert np.abs(zak.dzt(zak.idzt(X), M, N) - X).max() < 1e-12
    x = g.standard_normal(M * N) + 1j * g.standard_normal(M * N)
    assert np.abs(zak.idzt(zak.dzt(x, M, N)) - x).max() < 1e-12


@pytest.mark.parametrize("M,N", SHAPES)
def test_unitary(M, N):
    """DZT is unitary (Parseval): ||Y||_F = ||y||."""
    g = np.random.default_rng(7)
    y = g.standard_normal(M * N) + 1j * g.standard_normal(M * N)
    assert np.isclose(np.linalg.norm(zak.dzt(y, M, N)), np.linalg.norm(y), rtol=1e-13)


@pytest.mark.parametrize("M,N", [(8, 2), (16, 16), (64, 32)])
def test_impulse_closed_form(M, N):
    """A TD impulse at i0 = k0 + n0 M maps to Y[k, l] = N^-1/2 e^{-j2pi n0 l/N} delta[k - k0]."""
    for i0 in (0, 1, M - 1, M + 3, M * N - 1):
        k0, n0 = i0 % M, i0 // M
        y = np.zeros(M * N, complex)
        y[i0] = 1.0
        Y = zak.dzt(y, M, N)
        exp = np.zeros((M, N), complex)
        exp[k0, :] = np.exp(-2j * np.pi * n0 * np.arange(N) / N) / np.sqrt(N)
        assert np.abs(Y - exp).max() < 1e-14


@pytest.mark.parametrize("M,N", [(8, 2), (16, 16), (64, 32)])
def test_quasi_periodicity(M, N):
    """Extending Eq. zak's sum to k + M with the MN-periodic y gives
    Y[k + M, l] = e^{j2pi l/N} Y[k, l]; and Y[k, l + N] = Y[k, l] (footnote of Eq. y_channel_DD)."""
    g = np.random.default_rng(3)
    y = g.standard_normal(M * N) + 1j * g.standard_normal(M * N)
    Y = zak.dzt(y, M, N)
    i = np.arange(N)
    for k in (0, M // 2, M - 1):
        for l in range(N):
            direct = (y[np.mod(k + M + i * M, M * N)] * np.exp(-2j * np.pi * i * l / N)).sum() / np.sqrt(N)
            assert abs(direct - np.exp(2j * np.pi * l / N) * Y[k, l]) < 1e-12
            direct_l = (y[k + i * M] * np.exp(-2j * np.pi * i * (l + N) / N)).sum() / np.sqrt(N)
            assert abs(direct_l - Y[k, l]) < 1e-12
    # the oracle's quasi_periodic() helper agrees with the definition above
    k = np.arange(-M, 2 * M)
    for l in range(N):
        ext = zak.quasi_periodic(Y, k, l)
        for kk, v in zip(k, ext):
            direct = (y[np.mod(kk + i * M, M * N)] * np.exp(-2j * np.pi * i * l / N)).sum() / np.sqrt(N)
            assert abs(direct - v) < 1e-12


@pytest.mark.parametrize("M,N", SHAPES)
def test_idzt_matches_independent_transmitter(M, N):
    """synth.idzt (an inverse DFT along Doppler) and oracle.zak.idzt (Eq. iZak's sum) agree."""
    g = np.random.default_rng(11)
    X = g.standard_normal((M, N)) + 1j * g.standard_normal((M, N))
    assert np.abs(synth.idzt(X) - zak.idzt(X)).max() < 1e-12


def test_vec_order():
    M, N = 4, 3
    X = np.arange(M * N).reshape(M, N)
    v = zak.vec(X)
    for k in range(M):
        for l in range(N):
            assert v[l * M + k] == X[k, l]
    assert (zak.unvec(v, M, N) == X).all()
