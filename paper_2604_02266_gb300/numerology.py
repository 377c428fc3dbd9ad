"""Zak-OTFS frame numerology and packet sizing.

The grid (M delay bins, N Doppler bins) and the frequency spacing delta_f fix the frame's
time and bandwidth (Eq. bandwidth_frametime: B = M delta_f, T = N / delta_f) and its
resolutions (Eq. delay_Doppler_res: delay 1 / B, Doppler 1 / T).  Sec. VI-A takes the
channel coherence time as T_c ~ 0.423 / nu_max and puts one pilot frame and the data frames
that share its channel in a packet, which must be processed before the next packet has been
received: with one data frame per pilot (the paper's worst case) the deadline is 2 T.

Reading (not stated in the paper): a packet of one pilot frame and D data frames lasts
(1 + D) T and is channel-static if that span fits in T_c, so D = floor(T_c / T) - 1, at least 1
(one pilot per data frame when the channel changes faster); the packet's processing deadline is
its own duration (1 + D) T.
"""

import math

__all__ = ["frame_numerology", "coherence_time", "data_frames_per_pilot", "packet_deadline"]

COHERENCE_FACTOR = 0.423  # T_c ~ 0.423 / nu_max (Sec. VI-A)


def frame_numerology(M, N, delta_f_hz):
    """Bandwidth B, frame duration T, delay resolution 1/B and Doppler resolution 1/T of an
    M x N grid at frequency spacing delta_f (Eq. bandwidth_frametime, Eq. delay_Doppler_res),
    in Hz and seconds."""
    if M < 1 or N < 1 or not delta_f_hz > 0:
        raise ValueError("M, N >= 1 and delta_f > 0 required")
    B = M * delta_f_hz
    T = N / delta_f_hz
    return {"bandwidth_hz": B, "frame_s": T, "delay_res_s": 1.0 / B, "doppler_res_hz": 1.0 / T}


def coherence_time(nu_max_hz):
    """Channel coherence time T_c ~ 0.423 / nu_max in seconds (Sec. VI-A)."""
    if not nu_max_hz > 0:
        raise ValueError("nu_max must be > 0")
    return COHERENCE_FACTOR / nu_max_hz


def data_frames_per_pilot(nu_max_hz, N, delta_f_hz):
    """Data frames D that one pilot frame serves: the largest D with (1 + D) T <= T_c, at
    least 1."""
    T = frame_numerology(1, N, delta_f_hz)["frame_s"]
    # the small slack keeps a span that equals T_c up to rounding inside it
    return max(1, int(math.floor(coherence_time(nu_max_hz) / T * (1 + 1e-12))) - 1)


def packet_deadline(N, delta_f_hz, data_frames=1):
    """Processing deadline of a packet of one pilot frame and ``data_frames`` data frames: its
    duration (1 + D) T in seconds (2 T for the paper's one data frame per pilot)."""
    if data_frames < 1:
        raise ValueError("a packet carries at least one data frame")
    return (1 + data_frames) * frame_numerology(1, N, delta_f_hz)["frame_s"]
