"""Receiver stages composed per frame, FP64 (Fig. 1 pipeline, Sec. III-B; Sec. V setup).

Test infrastructure only (see :mod:`oracle`).

Per frame: DZT of the pilot frame(s) (Eq. zak) -> h_eff read-off (Eq. heff_hadamard) ->
thresholding (Eq. heff_thres) -> DZT of the data frame -> CGA (Algorithm 1) -> max-log
demapping.  The paper sends a separate point-pilot frame before each data frame; an
embedded pilot (pilot and guard band inside the data frame) is also supported, in which
case the read-off covers delay offsets [0, k_guard] and the pilot's response H(a e_pilot)
is subtracted from the data before equalisation.

MIMO (not in the paper): tx antenna t sends its own pilot frame; rx antenna r's copy of
it gives the (r, t) path list.  Pilot TD frames are laid out [t][r], data frames [r].
"""

import numpy as np

from . import zak, ddchannel, equalizer, qam


def estimate(y_pilot_td, M, N, K0, L0, a_pilot, theta, p_max=None, dk_range=None):
    """Path list of one antenna pair from its received pilot frame (TD)."""
    Yp = zak.dzt(y_pilot_td, M, N)
    heff = ddchannel.heff_readoff(Yp, K0, L0, a_pilot)
    region = ddchannel.readoff_region(M, N, K0, L0, dk_range)
    return ddchannel.threshold_paths(heff, K0, L0, theta, p_max, region)


def subtract_pilot(y_dd_vec, paths, a_pilot):
    """y - H (a_pilot e_(K0,L0)): remove an embedded pilot's response (Eq. sparse_mvm applied
    to the pilot grid)."""
    M, N = paths.M, paths.N
    e = np.zeros(M * N, np.complex128)
    e[paths.L0 * M + paths.K0] = a_pilot
    return y_dd_vec - equalizer.ss_forward(paths, e)


def receive(y_pilot_td, y_data_td, M, N, n_rx, n_tx, Q, noise_var, theta, iters,
            a_pilot, K0=None, L0=None, p_max=None, embedded_guard=None, cg_eps=0.0):
    """Full receiver for one frame.

    y_pilot_td: separate-pilot mode: (n_tx, n_rx, MN) complex; embedded mode: ignored.
    y_data_td:  (n_rx, MN) complex.
    Returns dict with path lists [r][t], y_dd (n_rx*MN), x_hat (n_tx*MN), llr (n_tx*MN, bps),
    bits (n_tx*MN, bps).
    """
    K0 = M // 2 if K0 is None else K0
    L0 = N // 2 if L0 is None else L0
    y_data_td = np.asarray(y_data_td, np.complex128).reshape(n_rx, M * N)
    y_dd = np.stack([zak.vec(zak.dzt(y_data_td[r], M, N)) for r in range(n_rx)])
    if embedded_guard is None:
        yp = np.asarray(y_pilot_td, np.complex128).reshape(n_tx, n_rx, M * N)
        paths = [[estimate(yp[t, r], M, N, K0, L0, a_pilot, theta, p_max) for t in range(n_tx)]
                 for r in range(n_rx)]
    else:
        assert n_rx == 1 and n_tx == 1, "embedded pilot: SISO"
        heff = ddchannel.heff_readoff(zak.unvec(y_dd[0], M, N), K0, L0, a_pilot)
        region = ddchannel.readoff_region(M, N, K0, L0, (0, embedded_guard))
        pl = ddchannel.threshold_paths(heff, K0, L0, theta, p_max, region)
        paths = [[pl]]
        y_dd = subtract_pilot(y_dd[0], pl, a_pilot)[None, :]
    y_vec = y_dd.reshape(-1)
    x_hat = equalizer.cga(paths, y_vec, noise_var, iters, eps=cg_eps)
    llr = qam.maxlog_llr(x_hat, noise_var, Q)
    return {
        "paths": paths,
        "y_dd": y_vec,
        "x_hat": x_hat,
        "llr": llr,
        "bits": qam.hard_bits_from_llr(llr),
    }


__all__ = ["estimate", "subtract_pilot", "receive"]
