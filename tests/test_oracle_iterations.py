"""Pins for the BER-driven iteration budget (Eq. ber_convergence): properties that follow from
the definition -- a geometric BER decay has a constant relative change 1 - q, a rebound always
converges, an all-zero BER converges at once through the zeta guard -- and the library's host
implementation against the oracle's on random curves."""

import numpy as np

from oracle import iterations as it


def test_geometric_decay():
    """BER_xi = b q^(xi - 1): r_xi = 1 - q for every xi, so the curve converges at xi = 2 when
    1 - q < eta and never (the last iteration) otherwise."""
    for q, conv in ((0.995, 2), (0.5, 12)):
        ber = [0.2 * q ** i for i in range(12)]
        assert it.convergence_iteration(ber) == conv


def test_rebound_converges_at_the_rise():
    ber = [0.3, 0.2, 0.1, 0.05, 0.06, 0.02]
    assert it.convergence_iteration(ber) == 5  # r_5 < 0
    # r_2 = 2/3, r_3 = 0.2: a negligible-gain threshold of 0.3 stops at 3
    assert it.convergence_iteration([0.3, 0.1, 0.08, 0.07], eta=0.3) == 3


def test_relative_change_is_taken_against_the_previous_ber():
    """Halving the BER is a relative change of 1/2 (against the previous BER), so with
    eta = 0.6 the curve has converged at the second iteration."""
    assert it.convergence_iteration([0.2, 0.1, 0.0999], eta=0.6) == 2


def test_zero_ber_and_zeta_guard():
    assert it.convergence_iteration([0.0, 0.0, 0.0]) == 2
    # a fall to zero from a tiny BER is a full relative gain (r = 1), not a division by zero
    assert it.convergence_iteration([1e-14, 0.0, 0.0]) == 3


def test_budget_is_the_largest_convergence_iteration():
    curves = [[0.3, 0.299], [0.4, 0.2, 0.1, 0.1], [0.5, 0.25, 0.2497]]
    assert it.budget(curves) == 4


def test_library_matches_oracle_on_random_curves():
    from paper_2604_02266_gb300 import iterations as lib
    g = np.random.default_rng(3)
    curves = []
    for _ in range(200):
        n = int(g.integers(1, 31))
        kind = g.integers(0, 3)
        if kind == 0:
            c = np.sort(g.uniform(0, 0.5, n))[::-1]
        elif kind == 1:
            c = g.uniform(0, 0.5, n)
        else:
            c = np.where(g.uniform(size=n) < 0.5, 0.0, g.uniform(0, 1e-3, n))
        curves.append(list(c))
        assert lib.convergence_iteration(c) == it.convergence_iteration(list(c))
    assert lib.iteration_budget(curves) == it.budget(curves)


def test_veh_a_frames_decode_at_high_snr():
    """The Veh-A generator (Table vehAProf delays and powers, Doppler nu_max cos(2 pi U)) makes
    frames the oracle receiver decodes to a low BER at 40 dB."""
    import synth
    from oracle import receiver
    M, N, Q = 32, 16, 4
    b = synth.veh_a_batch(2, 17, M=M, N=N, Q=Q, snr_db=(40,))
    for f in range(2):
        out = receiver.receive(b["y_pilot_td"][f], b["y_data_td"][f], M, N, 1, 1, Q, float(b["noise_var"][f]),
                               float(b["theta"][f]), 30, b["a_pilot"], p_max=256)
        ber = float((out["bits"].reshape(-1) != b["bits"][f].reshape(-1)).mean())
        assert ber < 0.02, (f, ber)
