"""Delay-Doppler channel: read-off, thresholding, dense and structured-sparse H_dd, FP64.

Test infrastructure only (see :mod:`oracle`).

Passages followed:

* Eq. heff (Sec. III-B "Channel Estimation") and its Hadamard form Eq. heff_exp /
  Eq. heff_hadamard (Sec. IV-A): point-pilot read-off of the effective channel;
* Eq. heff_thres (Sec. IV-B "Dominant path determination"): keep |h_eff| > theta;
* Eq. Hdd (Sec. III-B): dense DD channel matrix from h_eff;
* Eq. forward_mapping / Eq. map_chMatDD_col, Eq. herm_mapping and the phase
  phi = 2pi/(MN) [(l_p - L0) A + n l_{p,q} M] (Sec. IV-B "Analytical indices mapping",
  "Phase correction and coefficient synthesis");
* Eq. y_discrete_td (Sec. III-B), read with the Doppler nu_p in the exponent, for an
  integer-offset time-domain channel used only to pin the above;
* the twisted convolution and quasi-periodic extension of Eq. y_channel_DD.

A path list follows the paper's notation: path p sits at (k_p, l_p) on the pilot grid
(uncentred, k_p in [0,M), l_p in [0,N)) with gain h_p; the pilot is at (K0, L0).  The
physical delay/Doppler offsets are k_p - K0 and l_p - L0.
"""

from dataclasses import dataclass, field

import numpy as np

from .zak import _roots, vec, unvec, quasi_periodic


@dataclass
class PathList:
    """Dominant paths {(h_p, k_p, l_p)} of one (rx, tx) antenna pair (Sec. IV-B)."""

    M: int
    N: int
    K0: int
    L0: int
    h: np.ndarray = field(default_factory=lambda: np.zeros(0, np.complex128))
    kp: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    lp: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    truncated: bool = False

    @property
    def P(self):
        return len(self.h)

    @property
    def dk(self):
        """Centred delay offset k_p - K0 of each path."""
        return self.kp - self.K0

    @property
    def dl(self):
        """Centred Doppler offset l_p - L0 of each path."""
        return self.lp - self.L0

    @staticmethod
    def from_offsets(M, N, K0, L0, h, dk, dl):
        dk = np.asarray(dk, np.int64)
        dl = np.asarray(dl, np.int64)
        return PathList(M, N, K0, L0, np.asarray(h, np.complex128),
                        np.mod(K0 + dk, M), np.mod(L0 + dl, N))


# --------------------------------------------------------------------------------------
# Channel estimation (Eq. heff, Eq. heff_exp, Eq. heff_hadamard)
# --------------------------------------------------------------------------------------

def twist_matrix(M, N, K0, L0):
    """E_twist[k, l] = exp(-j 2 pi K0 (l - L0) / (MN))   (Eq. heff_exp)."""
    l = np.arange(N)[None, :]
    return np.broadcast_to(_roots(-K0 * (l - L0), M * N), (M, N)).copy()


def heff_readoff(Yp, K0, L0, a_pilot=1.0):
    """Effective-channel grid on the pilot grid: h_eff = (Y_p o E_twist) / a_pilot
    (Eq. heff_hadamard; with K0 = M/2 it is Eq. heff's exp(-j pi l / N) factor).

    Returned uncentred: entry [k, l] is the tap at delay offset k - K0 and Doppler
    offset l - L0.  The pilot amplitude a_pilot is divided out (the paper's pilot is a
    unit impulse, for which this is the identity).
    """
    Yp = np.asarray(Yp, np.complex128)
    M, N = Yp.shape
    return Yp * twist_matrix(M, N, K0, L0) / a_pilot


def readoff_region(M, N, K0, L0, dk_range=None):
    """Boolean (M, N) mask of the read-off region on the pilot grid.

    ``dk_range=None`` is the paper's separate pilot frame: all delay offsets
    [-M/2, M/2) and Doppler offsets [-N/2, N/2) (Eq. heff's index ranges).  For an
    embedded pilot, ``dk_range=(lo, hi)`` restricts the delay offsets to [lo, hi].
    """
    k = np.arange(M)[:, None]
    dk = np.mod(k - K0 + M // 2, M) - M // 2  # centred offset of row k
    mask = np.ones((M, N), bool)
    if dk_range is not None:
        lo, hi = dk_range
        mask &= (dk >= lo) & (dk <= hi)
    return mask


def threshold_paths(heff, K0, L0, theta, p_max=None, region=None):
    """Dominant paths, Eq. heff_thres: Omega = {(k, l) : |h_eff[k, l]| > theta}; h_p = h_eff[k_p, l_p].

    Order (the paper leaves it open): ascending q = l*M + k on the pilot grid.  When
    more than ``p_max`` taps pass, the ``p_max`` largest magnitudes are kept (ties to the
    lower q), still listed in ascending q, and ``truncated`` is set.
    """
    heff = np.asarray(heff, np.complex128)
    M, N = heff.shape
    if region is None:
        region = np.ones((M, N), bool)
    mag = np.abs(heff)
    sel = (mag > theta) & region
    q_sel = np.flatnonzero(vec(sel))  # ascending q
    truncated = False
    if p_max is not None and len(q_sel) > p_max:
        mags = vec(mag)[q_sel]
        order = np.lexsort((q_sel, -mags))  # largest magnitude first, then lower q
        q_sel = np.sort(q_sel[order[:p_max]])
        truncated = True
    kp = q_sel % M
    lp = q_sel // M
    return PathList(M, N, K0, L0, vec(heff)[q_sel].copy(), kp, lp, truncated)


def heff_from_paths(paths):
    """Sparse effective-channel grid (Eq. heff_model) holding exactly the listed taps."""
    H = np.zeros((paths.M, paths.N), np.complex128)
    for h, k, l in zip(paths.h, paths.kp, paths.lp):
        H[k, l] += h
    return H


# --------------------------------------------------------------------------------------
# Dense channel matrix (Eq. Hdd)
# --------------------------------------------------------------------------------------

def dense_H(heff, K0, L0, nm_range=2):
    """Dense H_dd from h_eff by Eq. Hdd, summing literally over the windows n, m.

    H[(k',l'), (k,l)] = sum_{n,m} exp(j2pi (l'-l-mN)(k+nM)/(MN)) h_c[k'-k-nM, l'-l-mN] exp(j2pi n l / N)

    where h_c is the centred effective channel, zero outside delay offsets [-M/2, M/2)
    and Doppler offsets [-N/2, N/2) (Eq. heff's index ranges); ``heff`` is given on the
    uncentred pilot grid, i.e. h_c[dk, dl] = heff[K0 + dk, L0 + dl].  Rows and columns use
    the vectorisation q = l*M + k (the paper writes k*N + l; any consistent order gives the
    same operator).  Only for tiny grids: the result is MN x MN.
    """
    heff = np.asarray(heff, np.complex128)
    M, N = heff.shape
    kq = np.arange(M)
    lq = np.arange(N)
    # 4-D index grids [k', l', k, l]
    k1 = kq[:, None, None, None]
    l1 = lq[None, :, None, None]
    k0 = kq[None, None, :, None]
    l0 = lq[None, None, None, :]
    H4 = np.zeros((M, N, M, N), np.complex128)
    for n in range(-nm_range, nm_range + 1):
        for m in range(-nm_range, nm_range + 1):
            dk = k1 - k0 - n * M
            dl = l1 - l0 - m * N
            valid = (dk >= -(M // 2)) & (dk < M - M // 2) & (dl >= -(N // 2)) & (dl < N - N // 2)
            tap = np.where(valid, heff[np.mod(K0 + dk, M), np.mod(L0 + dl, N)], 0.0)
            phase = _roots(dl * (k0 + n * M), M * N) * _roots(n * l0, N)
            H4 = H4 + tap * phase
    # rows (k', l') -> q' = l' M + k'; columns (k, l) -> q = l M + k
    return H4.transpose(1, 0, 3, 2).reshape(M * N, M * N)


# --------------------------------------------------------------------------------------
# Structured-sparse representation (Sec. IV-B)
# --------------------------------------------------------------------------------------

def ss_forward_map(paths, q):
    """Column index of path p's entry in row q, Eq. map_chMatDD_col:
    c_p(q) = <l_q + d_l>_N M + <k_q + d_k>_M with d_k = K0 - k_p, d_l = L0 - l_p.
    Returns an array of shape (P, len(q))."""
    M, N = paths.M, paths.N
    q = np.asarray(q)
    k_q = q % M
    l_q = q // M
    d_k = (paths.K0 - paths.kp)[:, None]
    d_l = (paths.L0 - paths.lp)[:, None]
    return np.mod(l_q + d_l, N) * M + np.mod(k_q + d_k, M)


def ss_inverse_map(paths, r):
    """Row index whose forward map is r, Eq. herm_mapping:
    q_p(r) = <l_r - d_l>_N M + <k_r - d_k>_M.  Shape (P, len(r))."""
    M, N = paths.M, paths.N
    r = np.asarray(r)
    k_r = r % M
    l_r = r // M
    d_k = (paths.K0 - paths.kp)[:, None]
    d_l = (paths.L0 - paths.lp)[:, None]
    return np.mod(l_r - d_l, N) * M + np.mod(k_r - d_k, M)


def ss_coefficients(paths, q, p=None):
    """D_{p,q} = h_p exp(j phi), phi = 2pi/(MN) [(l_p - L0) A + n l_{p,q} M]
    with A = K0 + k_q - k_p, n = floor(A / M), l_{p,q} = <L0 + l_q - l_p>_N
    (Sec. IV-B "Phase correction and coefficient synthesis").  Shape (P, len(q)), or
    (len(q),) for a single path index ``p``."""
    M, N = paths.M, paths.N
    q = np.asarray(q)
    k_q = q % M
    l_q = q // M
    if p is not None:
        one = PathList(M, N, paths.K0, paths.L0, paths.h[p:p + 1], paths.kp[p:p + 1], paths.lp[p:p + 1])
        return ss_coefficients(one, q)[0]
    kp = paths.kp[:, None]
    lp = paths.lp[:, None]
    A = paths.K0 + k_q - kp
    n = np.floor_divide(A, M)
    l_pq = np.mod(paths.L0 + l_q - lp, N)
    phi_num = (lp - paths.L0) * A + n * l_pq * M
    return paths.h[:, None] * _roots(phi_num, M * N)


def ss_to_dense(paths):
    """Dense matrix holding exactly the structured-sparse entries {D_{p,q}, c_p(q)} (Eq. ds_repr)."""
    MN = paths.M * paths.N
    q = np.arange(MN)
    H = np.zeros((MN, MN), np.complex128)
    cols = ss_forward_map(paths, q)
    D = ss_coefficients(paths, q)
    for p in range(paths.P):
        H[q, cols[p]] += D[p]
    return H


# --------------------------------------------------------------------------------------
# Physical channel models used to pin the above (Eq. y_discrete_td, Eq. y_channel_DD)
# --------------------------------------------------------------------------------------

def td_channel_integer(x, h, dk, dl, M, N):
    """Integer-offset TD channel, Eq. y_discrete_td with the Doppler nu_p in the exponent:
    y[i] = sum_p h_p x[<i - k_p>_{MN}] exp(j 2 pi l_p (i - k_p) / (MN))
    where k_p, l_p are the path's delay and Doppler offsets in bins (x is MN-periodic, as
    the IDZT output is).  Noise-free."""
    x = np.asarray(x, np.complex128)
    MN = M * N
    i = np.arange(MN)
    y = np.zeros(MN, np.complex128)
    for hp, k, l in zip(h, dk, dl):
        y += hp * x[np.mod(i - k, MN)] * _roots(l * (i - k), MN)
    return y


def twisted_convolution(h, dk, dl, X):
    """Y[k, l] = sum_p h_p X_qp[k - k_p, l - l_p] exp(j 2pi (k - k_p) l_p / (MN)):
    the discrete twisted convolution (footnote of Eq. y_channel_DD) of a sparse h_eff with
    the quasi-periodic extension X_qp of X."""
    X = np.asarray(X, np.complex128)
    M, N = X.shape
    k = np.arange(M)[:, None]
    l = np.arange(N)[None, :]
    Y = np.zeros((M, N), np.complex128)
    for hp, a, b in zip(h, dk, dl):
        Y += hp * quasi_periodic(X, k - a, l - b) * _roots((k - a) * b, M * N)
    return Y


__all__ = [
    "PathList", "twist_matrix", "heff_readoff", "readoff_region", "threshold_paths",
    "heff_from_paths", "dense_H", "ss_forward_map", "ss_inverse_map", "ss_coefficients",
    "ss_to_dense", "td_channel_integer", "twisted_convolution", "vec", "unvec",
]
