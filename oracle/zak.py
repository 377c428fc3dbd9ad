"""Discrete Zak transform pair, FP64 (Sec. III-B "Zak Transform", Eq. iZak and Eq. zak).

Test infrastructure only (see :mod:`oracle`).

Conventions used across the oracle:

* a DD grid is an ``(M, N)`` complex array ``X[k, l]`` with delay bin ``k`` and Doppler
  bin ``l``;
* its vectorised form uses ``q = l*M + k`` (Sec. IV-B, "We index the q-th row ... as
  q = l M + k"), i.e. ``vec(X) = X.reshape(-1, order="F")``;
* a time-domain (TD) frame is a length-``MN`` vector indexed ``i = k + n*M``.
"""

import numpy as np


def _roots(num, den):
    """exp(j*2*pi*num/den) with the integer numerator reduced mod den first (exact argument)."""
    num = np.mod(np.asarray(num, dtype=np.int64), den)
    return np.exp(2j * np.pi * num.astype(np.float64) / den)


def idzt(X):
    """Inverse DZT, Eq. iZak: x[i] = N^-1/2 sum_l X[<i>_M, l] exp(j 2 pi floor(i/M) l / N)."""
    X = np.asarray(X, dtype=np.complex128)
    M, N = X.shape
    i = np.arange(M * N)
    k = i % M
    n = i // M
    l = np.arange(N)
    E = _roots(np.outer(n, l), N)  # (MN, N)
    return (X[k, :] * E).sum(axis=1) / np.sqrt(N)


def dzt(y, M, N):
    """DZT, Eq. zak: Y[k, l] = N^-1/2 sum_{i<N} y[k + i M] exp(-j 2 pi i l / N).

    Written as the definition: gather the samples y[k + iM] into an (M, N) array
    (column i), then contract with the N x N DFT kernel.
    """
    y = np.asarray(y, dtype=np.complex128)
    assert y.shape == (M * N,)
    k = np.arange(M)[:, None]
    i = np.arange(N)[None, :]
    Ytd = y[k + i * M]  # Ytd[k, i] = y[k + iM]
    F = _roots(-np.outer(np.arange(N), np.arange(N)), N)  # F[i, l] = exp(-j2pi il/N)
    return Ytd @ F / np.sqrt(N)


def vec(X):
    """Column-major vectorisation q = l*M + k."""
    return np.asarray(X).reshape(-1, order="F")


def unvec(v, M, N):
    """Inverse of :func:`vec`."""
    return np.asarray(v).reshape((M, N), order="F")


def quasi_periodic(X, k, l):
    """Quasi-periodic extension of a DD grid (Sec. III-B, footnote on the received frame):
    X[k + nM, l + mN] = X[k, l] exp(j 2 pi n l / N) for k in [0,M), l in [0,N), any n, m."""
    X = np.asarray(X)
    M, N = X.shape
    k = np.asarray(k)
    l = np.asarray(l)
    n = np.floor_divide(k, M)
    kk = k - n * M
    ll = np.mod(l, N)
    return X[kk, ll] * _roots(n * ll, N)
