"""SS-MRC: maximal-ratio-combining decision-feedback equaliser on the path list, FP64.

Test infrastructure only (see :mod:`oracle`).

Passage followed: Sec. III-B "Equalization", paragraph "Maximum ratio combining (MRC)", and
the evaluation setup of Sec. V (SS-MRC = MRC with the channel in its structured-sparse form,
10 iterations).  The paper describes the equaliser in words only: it works on symbol vectors
(the symbols of one delay bin across all Doppler bins); each transmitted vector reaches several
received vectors through the channel's delay branches; per vector, the branch components are
extracted with the interference of the current estimates cancelled, combined coherently to
maximise the SNR, mapped to the nearest constellation point, and the estimates are refined
iteratively by decision feedback.  Cost O(iters P M N).

Reading (the cited algorithm itself is not restated in the paper):

* Domain.  The combining runs in the delay-time (DT) domain, where the Doppler axis of the DD
  grid is taken back to time by the inverse of the Zak transform's DFT:
  X_dt[k, n] = N^-1/2 sum_l X_dd[k, l] exp(j2pi n l / N), so X_dd[k, l] =
  N^-1/2 sum_n X_dt[k, n] exp(-j2pi n l / N) (Eq. zak's DFT along n).  There the structured-
  sparse operator of Sec. IV-B (Eq. sparse_mvm with the wrap count and phase of
  Eq. map_chMatDD_col) becomes, with A = k' - dk_p:
      (H v)_dt[k', n] = sum_p h_p exp(j2pi dl_p (A + n M) / (MN)) v_dt[<A>_M, <n + floor(A/M)>_N]
  (derivation: expand v_ext[A, l - dl_p] of the SS form through the DFT; the quasi-periodic
  phase exp(j2pi floor(A/M) l / N) becomes the time shift floor(A/M)).
* Branches.  Paths with equal delay offset d form one branch: symbol vector k reaches received
  vector <k + d>_M, element n landing on time index <n + f>_N with f = floor((k + d)/M), through
  the diagonal gain G_{k,d}[n] = sum_{p: dk_p = d} h_p exp(j2pi dl_p (<k+d>_M - d + (n+f) M)/(MN)).
  A branch is a diagonal gain times a cyclic time shift, so K^H K is diagonal:
  D_k[n] = sum_d |G_{k,d}[n]|^2.
* Iteration (Gauss-Seidel over the delay bins, k = 0 .. M-1 in order, starting from x_hat = 0
  and the residual dy = y_dt):
      c[n]  = x_hat_dt[k, n] + sum_d conj(G_{k,d}[n]) dy[<k+d>_M, <n+f_d>_N] / D_k[n]
              (= D^-1 sum_d K^H (dy + K x_hat_k): interference of the current estimates of all
              other vectors cancelled, branches combined with their conjugate gains);
      c_dd  = DFT of c along n; x_hat_dd[k, :] = nearest constellation point of each entry
              (Eq. demod's argmin);
      dy[<k+d>, <n+f_d>] -= G_{k,d}[n] (x_hat_dt_new[k, n] - x_hat_dt_old[k, n]) for every d.
  Where D_k[n] = 0 (no branch reaches the element) c keeps x_hat.  No noise term enters the
  combining (maximal ratio, not MMSE).
* Output.  The soft estimate c_dd of the last iteration (one value per DD bin) is the
  equaliser's output x_hat; its nearest points are the fed-back decisions, and the max-log
  demapper of :mod:`oracle.qam` gives LLRs and hard bits from it as for the CGA.
* SISO only (the paper's setting).
"""

import numpy as np

from .qam import constellation


def dd_to_dt(X_dd):
    """(M, N) DD grid -> delay-time grid: unitary inverse DFT along the Doppler axis."""
    X_dd = np.asarray(X_dd, np.complex128)
    return np.fft.ifft(X_dd, axis=1) * np.sqrt(X_dd.shape[1])


def dt_to_dd(X_dt):
    """Delay-time grid -> DD grid: unitary DFT along the time axis (Eq. zak's DFT)."""
    X_dt = np.asarray(X_dt, np.complex128)
    return np.fft.fft(X_dt, axis=1) / np.sqrt(X_dt.shape[1])


def branches(paths):
    """The delay branches of a path list: {d: (h, dl)} with the paths of delay offset d."""
    out = {}
    for h, d, l in zip(paths.h, paths.dk, paths.dl):
        hs, ls = out.setdefault(int(d), ([], []))
        hs.append(complex(h))
        ls.append(int(l))
    return {d: (np.array(hs), np.array(ls)) for d, (hs, ls) in sorted(out.items())}


def branch_gain(paths_d, k, d, M, N):
    """G_{k,d}[n] for n in [0, N), and the target row <k+d>_M and time shift f = floor((k+d)/M)."""
    hs, ls = paths_d
    kt = (k + d) % M
    f = (k + d) // M
    n = np.arange(N)
    G = np.zeros(N, np.complex128)
    for h, l in zip(hs, ls):
        t = np.mod(l * (kt - d + (n + f) * M), M * N)
        G += h * np.exp(2j * np.pi * t / (M * N))
    return G, kt, f


def dt_apply(paths, V_dt):
    """(H v) in the delay-time domain assembled branch by branch (Sec. IV-B's operator moved to
    DT, see the module reading): returns the (M, N) DT grid of H v."""
    M, N = paths.M, paths.N
    V_dt = np.asarray(V_dt, np.complex128)
    out = np.zeros((M, N), np.complex128)
    br = branches(paths)
    n = np.arange(N)
    for k in range(M):
        for d, pd in br.items():
            G, kt, f = branch_gain(pd, k, d, M, N)
            out[kt, np.mod(n + f, N)] += G * V_dt[k]
    return out


def combine_row(gk, D, x_row, dy):
    """MRC of one symbol vector: x_row + D^-1 sum_d conj(G_d) dy[target_d] (DT domain);
    entries no branch reaches keep x_row."""
    g = np.zeros(len(x_row), np.complex128)
    for G, kt, nt in gk:
        g += np.conj(G) * dy[kt, nt]
    c = np.asarray(x_row, np.complex128).copy()
    ok = D > 0
    c[ok] += g[ok] / D[ok]
    return c


def feed_back(gk, delta, dy):
    """Decision feedback: remove a symbol vector's change from the residual of every branch
    it reaches (dy updated in place)."""
    for G, kt, nt in gk:
        dy[kt, nt] -= G * delta


def mrc(paths, y_dd_vec, iters, Q, return_decisions=False):
    """SS-MRC on one SISO frame.  y_dd_vec: DD grid vectorised q = l M + k.  Returns the soft
    estimate x_hat (vectorised like y) of the last iteration (and the decided points)."""
    M, N = paths.M, paths.N
    y_dd = np.asarray(y_dd_vec, np.complex128).reshape(N, M).T
    dy = dd_to_dt(y_dd)
    br = branches(paths)
    pts = constellation(Q)
    n = np.arange(N)
    gains = []  # per delay bin: [(G, target row, target time indices)] and D_k
    for k in range(M):
        gk = []
        D = np.zeros(N)
        for d, pd in br.items():
            G, kt, f = branch_gain(pd, k, d, M, N)
            gk.append((G, kt, np.mod(n + f, N)))
            D += np.abs(G) ** 2
        gains.append((gk, D))
    x_dt = np.zeros((M, N), np.complex128)
    x_dec = np.zeros((M, N), np.complex128)
    soft = np.zeros((M, N), np.complex128)
    for _ in range(iters):
        for k in range(M):
            gk, D = gains[k]
            c = combine_row(gk, D, x_dt[k], dy)
            c_dd = dt_to_dd(c[None, :])[0]
            s = pts[np.argmin(np.abs(c_dd[:, None] - pts[None, :]) ** 2, axis=1)]
            new_dt = dd_to_dt(s[None, :])[0]
            feed_back(gk, new_dt - x_dt[k], dy)
            x_dt[k] = new_dt
            x_dec[k] = s
            soft[k] = c_dd
    x_hat = soft.T.reshape(-1)
    if return_decisions:
        return x_hat, x_dec.T.reshape(-1)
    return x_hat


__all__ = ["dd_to_dt", "dt_to_dd", "branches", "branch_gain", "dt_apply", "combine_row", "feed_back", "mrc"]
