"""Seeded synthetic Zak-OTFS frames: transmitter and channel only.

This module generates the inputs that both the CUDA library and the FP64 oracle
consume.  It holds no receiver arithmetic (no DZT, read-off, thresholding, channel
matrix, equaliser or demapper): only random draws (NumPy PCG64), the transmitter
(Gray square QAM mapping and the inverse Zak transform of Eq. iZak) and the channel
(Eq. y_discrete_td, read with the Doppler nu_p in the exponent, plus AWGN at
sigma^2 = rho_s / gamma, Sec. V "Channel model").  It is written independently of the
oracle; the oracle's tests check the two against each other (a noiseless frame must
come back bit-exact).

Workload recipes (shapes and distributions of the paper's experiments, Sec. V-VI):

* ``integer_embedded_frame``  -- 16x16 4-QAM frame with an embedded pilot at (8, 8) and a
  guard band of delay offsets [-2, 2] around it, 3 integer paths (delay 0..2, Doppler
  -2..2 bins, distinct), CN(0, 1/3) gains, 20 dB.
* ``fractional_batch``         -- separate pilot frame + data frame per user, sinc-pulse
  fractional channel: ``n_paths`` paths, delays U[0, 4] bins, Dopplers U[-3, 3] bins,
  exponential power-delay profile exp(-tau / 1 bin) normalised to unit total power,
  CN(0, power) gains, SNR drawn per frame from a list of dB values; n_rx x n_tx MIMO with
  independent channels per antenna pair and time-orthogonal pilot frames.

The pilot frame carries the same energy as a data frame (a_pilot = sqrt(MN)), so the
same noise variance applies to both and the read-off noise has standard deviation
sigma / a_pilot; the threshold "3 sigma" is theta = 3 sigma / a_pilot.
"""

import numpy as np

__all__ = ["rng", "qam_map", "idzt", "channel_integer", "channel_fractional", "awgn",
           "integer_embedded_frame", "fractional_batch", "packet_batch", "veh_a_batch", "uneven_batch",
           "VEH_A_DELAYS_US", "VEH_A_POWERS_DB"]

# The Veh-A power-delay profile of Sec. V "Channel model" (Table vehAProf): excess delays in
# microseconds and relative powers in dB of its six paths.
VEH_A_DELAYS_US = (0.00, 0.31, 0.71, 1.09, 1.73, 2.51)
VEH_A_POWERS_DB = (0.0, -1.0, -9.0, -10.0, -15.0, -20.0)


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------- transmitter

def _qam_table(Q):
    """Gray square QAM points indexed by label (I-axis Gray label in the high bits)."""
    m = int(round(np.sqrt(Q)))
    h = int(round(np.log2(m)))
    d = np.sqrt(3.0 / (2.0 * (Q - 1)))
    pts = np.zeros(Q, np.complex128)
    for a in range(m):          # PAM level index, I axis
        for b in range(m):      # PAM level index, Q axis
            ga = a ^ (a >> 1)
            gb = b ^ (b >> 1)
            pts[(ga << h) | gb] = complex((2 * a - m + 1) * d, (2 * b - m + 1) * d)
    return pts


def qam_map(bits, Q):
    """bits (..., n_sym * bps) 0/1, MSB of each label first -> symbols (..., n_sym)."""
    bps = int(round(np.log2(Q)))
    bits = np.asarray(bits, np.int64)
    shp = bits.shape[:-1] + (bits.shape[-1] // bps, bps)
    b = bits.reshape(shp)
    labels = (b << np.arange(bps - 1, -1, -1)).sum(axis=-1)
    return _qam_table(Q)[labels]


def idzt(X):
    """Inverse DZT (Eq. iZak) of an (M, N) grid: x[k + nM] = N^-1/2 sum_l X[k, l] e^{j2pi n l/N}.
    Evaluated as an inverse DFT along the Doppler axis."""
    X = np.asarray(X, np.complex128)
    M, N = X.shape
    xt = np.fft.ifft(X, axis=1) * np.sqrt(N)   # xt[k, n]
    return xt.T.reshape(-1)                    # sample index i = k + nM


# -------------------------------------------------------------------------------- channel

def _cis(num, den):
    return np.exp(2j * np.pi * np.mod(num, den) / den)


def channel_integer(x, gains, delays, dopplers):
    """y[i] = sum_p h_p x[i - k_p] exp(j 2pi l_p (i - k_p)/(MN)) on the MN-periodic x."""
    x = np.asarray(x, np.complex128)
    L = x.size
    i = np.arange(L)
    y = np.zeros(L, np.complex128)
    for g, k, l in zip(gains, delays, dopplers):
        y += g * np.roll(x, int(k)) * _cis(int(l) * (i - int(k)), L)
    return y


def channel_fractional(x, gains, delays, dopplers):
    """Fractional delays (band-limited periodic interpolation, i.e. a sinc pulse in delay)
    and fractional Dopplers (phase ramp over the frame, i.e. a sinc pulse in Doppler):
    y[i] = sum_p h_p x(i - tau_p) exp(j 2pi nu_p (i - tau_p)/(MN))."""
    x = np.asarray(x, np.complex128)
    L = x.size
    i = np.arange(L)
    f = np.fft.fftfreq(L) * L
    Xf = np.fft.fft(x)
    y = np.zeros(L, np.complex128)
    for g, tau, nu in zip(gains, delays, dopplers):
        xs = np.fft.ifft(Xf * np.exp(-2j * np.pi * f * tau / L))
        y += g * xs * np.exp(2j * np.pi * nu * (i - tau) / L)
    return y


def awgn(shape, sigma2, g):
    return np.sqrt(sigma2 / 2.0) * (g.standard_normal(shape) + 1j * g.standard_normal(shape))


# ------------------------------------------------------------------------------ workloads

def integer_embedded_frame(seed, M=16, N=16, Q=4, snr_db=20.0, n_paths=3, guard=2,
                           a_pilot=None, noiseless=False):
    """One SISO frame with an embedded pilot at (M/2, N/2) and integer-offset paths."""
    g = rng(seed)
    K0, L0 = M // 2, N // 2
    a_pilot = np.sqrt(M * N) * 0.5 if a_pilot is None else a_pilot
    bps = int(round(np.log2(Q)))
    # distinct (delay, Doppler) pairs with delay 0..guard, Doppler -2..2
    cand = [(k, l) for k in range(guard + 1) for l in range(-2, 3)]
    pick = g.choice(len(cand), size=n_paths, replace=False)
    delays = np.array([cand[c][0] for c in pick])
    dopplers = np.array([cand[c][1] for c in pick])
    gains = np.sqrt(1.0 / (2 * n_paths)) * (g.standard_normal(n_paths) + 1j * g.standard_normal(n_paths))
    k = np.arange(M)[:, None]
    dk = np.mod(k - K0 + M // 2, M) - M // 2
    data_mask = np.broadcast_to(np.abs(dk) > guard, (M, N)).copy()
    bits = g.integers(0, 2, size=(int(data_mask.sum()) * bps,))
    # data symbols fill the non-guard bins in ascending q = l*M + k
    Xv = np.zeros(M * N, np.complex128)
    Xv[np.flatnonzero(data_mask.reshape(-1, order="F"))] = qam_map(bits, Q)
    X = Xv.reshape((M, N), order="F")
    X[K0, L0] = a_pilot
    sigma2 = 10.0 ** (-snr_db / 10.0)
    x = idzt(X)
    y = channel_integer(x, gains, delays, dopplers)
    if not noiseless:
        y = y + awgn(y.shape, sigma2, g)
    return {
        "M": M, "N": N, "Q": Q, "K0": K0, "L0": L0, "a_pilot": float(a_pilot), "guard": guard,
        "y_data_td": y, "noise_var": sigma2, "theta": 3.0 * np.sqrt(sigma2) / a_pilot,
        "bits": bits.astype(np.uint8), "data_mask": data_mask, "X": X,
        "gains": gains, "delays": delays, "dopplers": dopplers,
    }


def fractional_batch(n_frames, seed, M=64, N=32, Q=16, n_rx=1, n_tx=1, n_paths=6,
                     snr_db=tuple(range(31)), delay_max=4.0, doppler_max=3.0,
                     dtype=np.complex64, theta_sigmas=3.0, integer=False):
    """Batch of frames, each with n_tx separate pilot frames and one data frame.

    Returns arrays shaped for the C ABI:
      y_pilot_td [n_frames, n_tx, n_rx, MN], y_data_td [n_frames, n_rx, MN] (``dtype``),
      noise_var [n_frames], theta [n_frames] (float32), bits [n_frames, n_tx, MN*bps] (u8).
    Frame f uses the generator seeded with seed + f.
    """
    MN = M * N
    bps = int(round(np.log2(Q)))
    K0, L0 = M // 2, N // 2
    a_pilot = np.sqrt(MN)
    yp = np.zeros((n_frames, n_tx, n_rx, MN), np.complex128)
    yd = np.zeros((n_frames, n_rx, MN), np.complex128)
    noise_var = np.zeros(n_frames)
    bits = np.zeros((n_frames, n_tx, MN * bps), np.uint8)
    snrs = np.zeros(n_frames)
    chan = []
    Xp = np.zeros((M, N), np.complex128)
    Xp[K0, L0] = a_pilot
    xp = idzt(Xp)
    for f in range(n_frames):
        g = rng(seed + f)
        snr = float(g.choice(np.asarray(snr_db, float)))
        sigma2 = 10.0 ** (-snr / 10.0)
        b = g.integers(0, 2, size=(n_tx, MN * bps)).astype(np.uint8)
        xs = [idzt(qam_map(b[t], Q).reshape((M, N), order="F")) for t in range(n_tx)]
        pairs = {}
        for r in range(n_rx):
            for t in range(n_tx):
                if integer:
                    tau = g.integers(0, int(delay_max) + 1, size=n_paths).astype(float)
                    nu = g.integers(-int(doppler_max), int(doppler_max) + 1, size=n_paths).astype(float)
                else:
                    tau = g.uniform(0.0, delay_max, size=n_paths)
                    nu = g.uniform(-doppler_max, doppler_max, size=n_paths)
                pw = np.exp(-tau)
                pw = pw / pw.sum()
                h = np.sqrt(pw / 2.0) * (g.standard_normal(n_paths) + 1j * g.standard_normal(n_paths))
                pairs[(r, t)] = (h, tau, nu)
        for t in range(n_tx):
            for r in range(n_rx):
                h, tau, nu = pairs[(r, t)]
                ch = channel_integer if integer else channel_fractional
                yp[f, t, r] = ch(xp, h, tau.astype(int) if integer else tau,
                                 nu.astype(int) if integer else nu) + awgn(MN, sigma2, g)
        for r in range(n_rx):
            acc = np.zeros(MN, np.complex128)
            for t in range(n_tx):
                h, tau, nu = pairs[(r, t)]
                ch = channel_integer if integer else channel_fractional
                acc += ch(xs[t], h, tau.astype(int) if integer else tau,
                          nu.astype(int) if integer else nu)
            yd[f, r] = acc + awgn(MN, sigma2, g)
        noise_var[f] = sigma2
        bits[f] = b
        snrs[f] = snr
        chan.append(pairs)
    return {
        "M": M, "N": N, "Q": Q, "n_rx": n_rx, "n_tx": n_tx, "K0": K0, "L0": L0,
        "a_pilot": float(a_pilot),
        "y_pilot_td": yp.astype(dtype), "y_data_td": yd.astype(dtype),
        "noise_var": noise_var.astype(np.float32),
        "theta": (theta_sigmas * np.sqrt(noise_var) / a_pilot).astype(np.float32),
        "bits": bits, "snr_db": snrs, "channels": chan,
    }


def packet_batch(n_packets, data_per_pilot, seed, M=64, N=32, Q=16, n_rx=1, n_tx=1, n_paths=6,
                 snr_db=tuple(range(31)), delay_max=4.0, doppler_max=3.0, dtype=np.complex64,
                 theta_sigmas=3.0):
    """Packets of one pilot frame (per tx antenna) and ``data_per_pilot`` data frames through
    the same fractional channel (block-static within the coherence time), each data frame with
    its own bits and noise at the packet's SNR.  Channel recipe as ``fractional_batch``.

    Returns y_pilot_td [P, n_tx, n_rx, MN], y_data_td [P D, n_rx, MN], noise_var [P D],
    theta [P], bits [P D, n_tx, MN*bps], path_ids [P D] (int32: the packet of each data frame).
    Packet p uses the generator seeded with seed + p.
    """
    MN = M * N
    bps = int(round(np.log2(Q)))
    K0, L0 = M // 2, N // 2
    a_pilot = np.sqrt(MN)
    D = data_per_pilot
    yp = np.zeros((n_packets, n_tx, n_rx, MN), np.complex128)
    yd = np.zeros((n_packets * D, n_rx, MN), np.complex128)
    noise_var = np.zeros(n_packets * D)
    theta = np.zeros(n_packets)
    bits = np.zeros((n_packets * D, n_tx, MN * bps), np.uint8)
    Xp = np.zeros((M, N), np.complex128)
    Xp[K0, L0] = a_pilot
    xp = idzt(Xp)
    for pk in range(n_packets):
        g = rng(seed + pk)
        snr = float(g.choice(np.asarray(snr_db, float)))
        sigma2 = 10.0 ** (-snr / 10.0)
        pairs = {}
        for r in range(n_rx):
            for t in range(n_tx):
                tau = g.uniform(0.0, delay_max, size=n_paths)
                nu = g.uniform(-doppler_max, doppler_max, size=n_paths)
                pw = np.exp(-tau)
                pw = pw / pw.sum()
                h = np.sqrt(pw / 2.0) * (g.standard_normal(n_paths) + 1j * g.standard_normal(n_paths))
                pairs[(r, t)] = (h, tau, nu)
        for t in range(n_tx):
            for r in range(n_rx):
                h, tau, nu = pairs[(r, t)]
                yp[pk, t, r] = channel_fractional(xp, h, tau, nu) + awgn(MN, sigma2, g)
        theta[pk] = theta_sigmas * np.sqrt(sigma2) / a_pilot
        for d in range(D):
            f = pk * D + d
            b = g.integers(0, 2, size=(n_tx, MN * bps)).astype(np.uint8)
            xs = [idzt(qam_map(b[t], Q).reshape((M, N), order="F")) for t in range(n_tx)]
            for r in range(n_rx):
                acc = np.zeros(MN, np.complex128)
                for t in range(n_tx):
                    h, tau, nu = pairs[(r, t)]
                    acc += channel_fractional(xs[t], h, tau, nu)
                yd[f, r] = acc + awgn(MN, sigma2, g)
            noise_var[f] = sigma2
            bits[f] = b
    return {
        "M": M, "N": N, "Q": Q, "n_rx": n_rx, "n_tx": n_tx, "K0": K0, "L0": L0,
        "a_pilot": float(a_pilot),
        "y_pilot_td": yp.astype(dtype), "y_data_td": yd.astype(dtype),
        "noise_var": noise_var.astype(np.float32), "theta": theta.astype(np.float32),
        "bits": bits, "path_ids": (np.arange(n_packets * D) // D).astype(np.int32),
    }


def veh_a_batch(n_frames, seed, M=128, N=32, Q=16, snr_db=(20,), nu_max_hz=100.0, delta_f_hz=30e3,
                dtype=np.complex64, theta_sigmas=3.0):
    """SISO frames (separate pilot frame + data frame) through the Veh-A channel of Sec. V:
    the six paths of Table vehAProf (delays in bins: tau_us 1e-6 M delta_f; powers normalised to
    unit total, CN(0, power) gains), Doppler nu_p = nu_max cos(2 pi U_p), U_p ~ U(0, 1), in bins
    of delta_f / N; both fractional.  SNR per frame from ``snr_db``.  Same return layout as
    ``fractional_batch``.  Frame f uses the generator seeded with seed + f."""
    MN = M * N
    bps = int(round(np.log2(Q)))
    K0, L0 = M // 2, N // 2
    a_pilot = np.sqrt(MN)
    tau = np.asarray(VEH_A_DELAYS_US) * 1e-6 * M * delta_f_hz
    pw = 10.0 ** (np.asarray(VEH_A_POWERS_DB) / 10.0)
    pw = pw / pw.sum()
    yp = np.zeros((n_frames, 1, 1, MN), np.complex128)
    yd = np.zeros((n_frames, 1, MN), np.complex128)
    noise_var = np.zeros(n_frames)
    bits = np.zeros((n_frames, 1, MN * bps), np.uint8)
    Xp = np.zeros((M, N), np.complex128)
    Xp[K0, L0] = a_pilot
    xp = idzt(Xp)
    for f in range(n_frames):
        g = rng(seed + f)
        snr = float(g.choice(np.asarray(snr_db, float)))
        sigma2 = 10.0 ** (-snr / 10.0)
        b = g.integers(0, 2, size=(1, MN * bps)).astype(np.uint8)
        x = idzt(qam_map(b[0], Q).reshape((M, N), order="F"))
        h = np.sqrt(pw / 2.0) * (g.standard_normal(6) + 1j * g.standard_normal(6))
        nu = nu_max_hz * np.cos(2.0 * np.pi * g.uniform(0.0, 1.0, size=6)) / (delta_f_hz / N)
        yp[f, 0, 0] = channel_fractional(xp, h, tau, nu) + awgn(MN, sigma2, g)
        yd[f, 0] = channel_fractional(x, h, tau, nu) + awgn(MN, sigma2, g)
        noise_var[f] = sigma2
        bits[f] = b
    return {
        "M": M, "N": N, "Q": Q, "n_rx": 1, "n_tx": 1, "K0": K0, "L0": L0, "a_pilot": float(a_pilot),
        "y_pilot_td": yp.astype(dtype), "y_data_td": yd.astype(dtype),
        "noise_var": noise_var.astype(np.float32),
        "theta": (theta_sigmas * np.sqrt(noise_var) / a_pilot).astype(np.float32), "bits": bits,
    }


def uneven_batch(n_frames, seed, Ms=(32, 64, 128), Ns=(16, 32, 64), mimo=((1, 1), (2, 2)),
                 Qs=(16,), n_paths=6, snr_db=tuple(range(31)), dtype=np.complex64):
    """Frames of mixed shapes: M, N, antenna configuration and QAM order drawn uniformly per
    frame (generator seed + f).  Returns a list of per-frame dicts in the
    ``fractional_batch`` layout with a leading batch dimension of 1."""
    out = []
    for f in range(n_frames):
        g = rng(seed + f)
        M = int(g.choice(Ms))
        N = int(g.choice(Ns))
        n_rx, n_tx = mimo[int(g.integers(0, len(mimo)))]
        Q = int(g.choice(Qs))
        fr = fractional_batch(1, seed=int(g.integers(0, 2 ** 31)), M=M, N=N, Q=Q, n_rx=n_rx,
                              n_tx=n_tx, n_paths=n_paths, snr_db=snr_db, dtype=dtype)
        out.append(fr)
    return out
