"""Pins of the SS-MRC oracle (oracle/mrc.py) against things other than itself.

* The delay-time branch operator equals the dense DD matrix of Eq. Hdd (built literally from
  h_eff, independent of the structured-sparse formulas), wrap-around offsets included.
* One path: H is h times a unitary, so one MRC pass from x_hat = 0 is the exact inverse,
  checked against a dense solve.
* Every MRC row step is a least-squares solve for that delay bin's symbols with the other
  bins' current estimates fixed.  A reference written only with the dense Eq. Hdd matrix and
  numpy's lstsq (block Gauss-Seidel over the delay bins in order, nearest-point decisions fed
  back) must give the same soft outputs and decisions: this fixes the combining weights, the
  branch geometry and the update order.
* Noiseless integer-offset 4-QAM frames through the independent transmitter decode to the
  transmitted bits.
"""

import numpy as np
import pytest

import synth
from oracle import ddchannel as dc, mrc, qam, receiver, zak


def _paths(g, M, N, P, edge=True):
    cand = [(a, b) for a in range(-(M // 2), M // 2) for b in range(-(N // 2), N // 2)]
    pick = list(g.choice(len(cand), size=P, replace=False))
    if edge:  # wrap-around offsets at the edges of the centred range
        pick[0] = cand.index((-(M // 2), -(N // 2)))
        pick[1] = cand.index((M // 2 - 1, N // 2 - 1))
    h = (g.standard_normal(P) + 1j * g.standard_normal(P)) / np.sqrt(2 * P)
    return dc.PathList.from_offsets(M, N, M // 2, N // 2, h, [cand[c][0] for c in pick], [cand[c][1] for c in pick])


@pytest.mark.parametrize("M,N,P", [(16, 8, 7), (8, 16, 5), (32, 16, 12)])
def test_dt_operator_equals_dense_hdd(M, N, P):
    g = np.random.default_rng(M + N + P)
    pl = _paths(g, M, N, P)
    H = dc.dense_H(dc.heff_from_paths(pl), M // 2, N // 2)
    V = g.standard_normal((M, N)) + 1j * g.standard_normal((M, N))
    got = mrc.dt_to_dd(mrc.dt_apply(pl, mrc.dd_to_dt(V)))
    np.testing.assert_allclose(got, zak.unvec(H @ zak.vec(V), M, N), atol=1e-12)


def test_dd_dt_transforms_are_inverse_unitary():
    g = np.random.default_rng(3)
    X = g.standard_normal((8, 16)) + 1j * g.standard_normal((8, 16))
    np.testing.assert_allclose(mrc.dt_to_dd(mrc.dd_to_dt(X)), X, atol=1e-13)
    np.testing.assert_allclose(np.linalg.norm(mrc.dd_to_dt(X)), np.linalg.norm(X), rtol=1e-13)


@pytest.mark.parametrize("dk,dl", [(3, -2), (-8, -4), (7, 3), (0, 0)])
def test_single_path_one_pass_is_the_exact_inverse(dk, dl):
    M, N = 16, 8
    g = np.random.default_rng(11)
    pl = dc.PathList.from_offsets(M, N, M // 2, N // 2, np.array([0.7 - 0.4j]), [dk], [dl])
    H = dc.dense_H(dc.heff_from_paths(pl), M // 2, N // 2)
    y = g.standard_normal(M * N) + 1j * g.standard_normal(M * N)
    np.testing.assert_allclose(mrc.mrc(pl, y, 1, 16), np.linalg.solve(H, y), atol=1e-12)


def _dense_gauss_seidel_ls(H, y, M, N, iters, Q):
    """Reference from the dense matrix only: per delay bin k in order, the least-squares
    symbols of that bin given the other bins' current decisions, then the nearest points."""
    pts = qam.constellation(Q)
    x = np.zeros(M * N, np.complex128)
    soft = np.zeros(M * N, np.complex128)
    for _ in range(iters):
        for k in range(M):
            cols = np.arange(N) * M + k  # q = l M + k
            r = y - H @ x + H[:, cols] @ x[cols]
            c = np.linalg.lstsq(H[:, cols], r, rcond=None)[0]
            soft[cols] = c
            x[cols] = pts[np.argmin(np.abs(c[:, None] - pts[None, :]) ** 2, axis=1)]
    return soft, x


@pytest.mark.parametrize("M,N,P,Q,iters", [(16, 8, 6, 4, 3), (8, 8, 9, 16, 2), (16, 16, 5, 16, 3)])
def test_mrc_equals_dense_block_gauss_seidel_least_squares(M, N, P, Q, iters):
    g = np.random.default_rng(100 + M * P + Q)
    pl = _paths(g, M, N, P, edge=False)
    H = dc.dense_H(dc.heff_from_paths(pl), M // 2, N // 2)
    x_tx = qam.constellation(Q)[g.integers(0, Q, M * N)]
    y = H @ x_tx + 0.05 * (g.standard_normal(M * N) + 1j * g.standard_normal(M * N))
    soft, dec = mrc.mrc(pl, y, iters, Q, return_decisions=True)
    soft_ref, dec_ref = _dense_gauss_seidel_ls(H, y, M, N, iters, Q)
    np.testing.assert_allclose(soft, soft_ref, atol=1e-9)
    np.testing.assert_array_equal(dec, dec_ref)


def test_noiseless_integer_4qam_frames_decode_to_the_transmitted_bits():
    M, N, Q = 32, 16, 4
    b = synth.fractional_batch(6, seed=9, M=M, N=N, Q=Q, snr_db=(60,), integer=True)
    for f in range(6):
        r = receiver.receive(b["y_pilot_td"][f], b["y_data_td"][f], M, N, 1, 1, Q, float(b["noise_var"][f]),
                             float(b["theta"][f]), 10, b["a_pilot"], p_max=64)
        x = mrc.mrc(r["paths"][0][0], r["y_dd"], 4, Q)
        bits = qam.hard_bits_from_llr(qam.maxlog_llr(x, 1.0, Q)).reshape(-1)
        assert np.array_equal(bits, b["bits"][f].reshape(-1)), f
