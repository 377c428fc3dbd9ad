"""The packet generator's data frames share their pilot's channel: the oracle receiver, given
a packet's pilot frame and each of its data frames, returns the transmitted bits up to the
read-off's fractional-channel floor, while the other packet's pilot gives chance-level bits."""

import numpy as np

import synth
from oracle import receiver


def test_packet_data_frames_share_the_pilot_channel():
    M, N, Q, P, D = 32, 16, 4, 2, 3
    b = synth.packet_batch(P, D, 31, M=M, N=N, Q=Q, snr_db=(45,))
    assert (b["path_ids"] == np.repeat(np.arange(P), D)).all()

    def ber(p, f):
        ref = receiver.receive(b["y_pilot_td"][p], b["y_data_td"][f], M, N, 1, 1, Q, float(b["noise_var"][f]),
                               float(b["theta"][p]), 30, b["a_pilot"], p_max=256)
        return float((ref["bits"].reshape(-1) != b["bits"][f].reshape(-1)).mean())

    for f in range(P * D):
        p = int(b["path_ids"][f])
        assert ber(p, f) < 0.02, f
        assert ber(1 - p, f) > 0.2, f
