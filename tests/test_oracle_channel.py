"""Pins for the oracle's DD channel: the paper's worked example, its counting identities,
Eq. Hdd against the physical TD channel, the structured-sparse maps against Eq. Hdd, the
pilot read-off against the true taps, and thresholding against brute force."""

import numpy as np
import pytest

import synth
from oracle import zak, ddchannel as dc
from tests.golden import read_fixture


def _physical_matrix(h, dk, dl, M, N):
    """Columns DZT(TD channel(IDZT(e_q))): the operator the DD model must reproduce."""
    MN = M * N
    H = np.zeros((MN, MN), complex)
    for q in range(MN):
        e = np.zeros(MN, complex)
        e[q] = 1.0
        x = zak.idzt(zak.unvec(e, M, N))
        H[:, q] = zak.vec(zak.dzt(dc.td_channel_integer(x, h, dk, dl, M, N), M, N))
    return H


def _random_paths(g, M, N, P, wide=True):
    """Distinct integer offsets; ``wide`` spans the whole centred range so wraps occur."""
    cand = [(a, b) for a in range(-(M // 2), M - M // 2) for b in range(-(N // 2), N - N // 2)]
    if not wide:
        cand = [(a, b) for a, b in cand if abs(a) <= 3 and abs(b) <= 3]
    pick = g.choice(len(cand), size=P, replace=False)
    dk = np.array([cand[c][0] for c in pick])
    dl = np.array([cand[c][1] for c in pick])
    h = g.standard_normal(P) + 1j * g.standard_normal(P)
    return h, dk, dl


def test_worked_example_column_map():
    fx = read_fixture("worked_example_8x2.txt")
    M, N, K0, L0 = (int(fx[k][0][0]) for k in ("M", "N", "K0", "L0"))
    kp = np.array([int(p[0]) for p in fx["path"]])
    lp = np.array([int(p[1]) for p in fx["path"]])
    row = fx["row"][0]
    q = int(row[0])
    cols = [int(c) for c in row[2:]]
    pl = dc.PathList(M, N, K0, L0, np.ones(len(kp), complex), kp, lp)
    assert list(dc.ss_forward_map(pl, [q])[:, 0]) == cols
    # the dense Eq. Hdd matrix built from the two unit taps has its row-q support there
    Hd = dc.dense_H(dc.heff_from_paths(pl), K0, L0)
    assert sorted(np.flatnonzero(np.abs(Hd[q]) > 1e-12)) == sorted(cols)
    # inverse map sends those columns back to row q
    for p, c in enumerate(cols):
        assert dc.ss_inverse_map(pl, [c])[p, 0] == q
    # 256 -> 32 multiplications: (MN)^2 dense entries vs P*MN structured-sparse entries,
    # and Eq. Hdd really has exactly P*MN nonzeros
    assert (M * N) ** 2 == int(fx["mults_dense"][0][0])
    assert len(kp) * M * N == int(fx["mults_ss"][0][0])
    assert int((np.abs(Hd) > 1e-12).sum()) == int(fx["mults_ss"][0][0])


def test_worked_example_physical_reading():
    """Path (0, 0) against pilot (4, 1): offsets (-4, -1) bins -> 0.017 ms and 15 kHz."""
    fx = read_fixture("worked_example_8x2.txt")
    M, N = int(fx["M"][0][0]), int(fx["N"][0][0])
    df = float(fx["delta_f_hz"][0][0])
    dk, dl = 0 - int(fx["K0"][0][0]), 0 - int(fx["L0"][0][0])
    delay_ms = abs(dk) / (M * df) * 1e3
    doppler_khz = abs(dl) * df / N / 1e3
    assert round(delay_ms, 3) == float(fx["path1_delay_ms"][0][0])
    assert doppler_khz == float(fx["path1_doppler_khz"][0][0])


def test_counting_identities():
    fx = read_fixture("counting_identities.txt")
    M, N, P = int(fx["M"][0][0]), int(fx["N"][0][0]), int(fx["P"][0][0])
    assert P * M * N == int(fx["ss_values"][0][0])
    assert round((M * N) ** 2 / (P * M * N), 1) == float(fx["ratio"][0][0])
    assert round((M * N) ** 2 / 1e6, 1) == float(fx["dense_values_millions"][0][0])
    bM, bN, B = (int(fx[k][0][0]) for k in ("big_M", "big_N", "bytes_per_entry"))
    assert round(B * bM ** 2 * bN ** 2 / 1e9, 1) == float(fx["dense_GB"][0][0])


def test_counting_nnz_scales_with_paths():
    """Eq. Hdd built from P distinct taps has exactly P nonzeros per row (P*MN total)."""
    g = np.random.default_rng(5)
    M, N = 8, 4
    for P in (1, 3, 6):
        h, dk, dl = _random_paths(g, M, N, P)
        pl = dc.PathList.from_offsets(M, N, M // 2, N // 2, h, dk, dl)
        Hd = dc.dense_H(dc.heff_from_paths(pl), M // 2, N // 2)
        assert ((np.abs(Hd) > 1e-12).sum(axis=1) == P).all()


@pytest.mark.parametrize("M,N,P,seed", [(8, 2, 2, 0), (8, 4, 4, 1), (16, 16, 5, 2), (16, 8, 8, 3), (4, 8, 3, 4)])
def test_dense_hdd_equals_physical_channel(M, N, P, seed):
    """Eq. Hdd from the true taps equals DZT o (Eq. y_discrete_td) o IDZT for integer offsets,
    including offsets at the edge of the centred range (quasi-periodic wraps)."""
    g = np.random.default_rng(seed)
    h, dk, dl = _random_paths(g, M, N, P)
    pl = dc.PathList.from_offsets(M, N, M // 2, N // 2, h, dk, dl)
    Hd = dc.dense_H(dc.heff_from_paths(pl), M // 2, N // 2)
    assert np.abs(Hd - _physical_matrix(h, dk, dl, M, N)).max() < 1e-12


@pytest.mark.parametrize("M,N,P,seed", [(8, 2, 2, 10), (16, 16, 6, 11), (32, 8, 7, 12), (8, 16, 9, 13)])
def test_ss_representation_equals_dense(M, N, P, seed):
    """{D_{p,q}, c_p(q)} (Eq. ds_repr with the analytic map and phase) reproduces Eq. Hdd."""
    g = np.random.default_rng(seed)
    h, dk, dl = _random_paths(g, M, N, P)
    pl = dc.PathList.from_offsets(M, N, M // 2, N // 2, h, dk, dl)
    Hd = dc.dense_H(dc.heff_from_paths(pl), M // 2, N // 2)
    assert np.abs(dc.ss_to_dense(pl) - Hd).max() < 1e-12
    # the inverse map inverts the forward map for every path (Eq. herm_mapping)
    q = np.arange(M * N)
    fwd = dc.ss_forward_map(pl, q)
    for p in range(P):
        assert (dc.ss_inverse_map(pl, fwd[p])[p] == q).all()


@pytest.mark.parametrize("M,N,seed", [(8, 4, 0), (16, 16, 1), (8, 8, 2)])
def test_twisted_convolution(M, N, seed):
    """DZT(TD channel(IDZT(X))) = h_eff *_sigma X_qp (Eq. y_channel_DD), noise-free."""
    g = np.random.default_rng(seed)
    h, dk, dl = _random_paths(g, M, N, 4)
    X = g.standard_normal((M, N)) + 1j * g.standard_normal((M, N))
    Y = zak.dzt(dc.td_channel_integer(zak.idzt(X), h, dk, dl, M, N), M, N)
    assert np.abs(Y - dc.twisted_convolution(h, dk, dl, X)).max() < 1e-12


@pytest.mark.parametrize("M,N,seed", [(8, 2, 0), (16, 16, 1), (64, 32, 2)])
def test_pilot_readoff_recovers_taps(M, N, seed):
    """A noiseless point pilot through an integer channel: Eq. heff returns h_p at (K0+dk, L0+dl)
    and zero elsewhere (offsets inside the centred range, no pilot-response wrap)."""
    g = np.random.default_rng(seed)
    h, dk, dl = _random_paths(g, M, N, min(4, M * N // 4), wide=False)
    K0, L0 = M // 2, N // 2
    a = np.sqrt(M * N)
    Xp = np.zeros((M, N), complex)
    Xp[K0, L0] = a
    yp = dc.td_channel_integer(zak.idzt(Xp), h, dk, dl, M, N)
    heff = dc.heff_readoff(zak.dzt(yp, M, N), K0, L0, a)
    exp = np.zeros((M, N), complex)
    for hp, a_, b_ in zip(h, dk, dl):
        exp[K0 + a_, L0 + b_] += hp
    assert np.abs(heff - exp).max() < 1e-12
    pl = dc.threshold_paths(heff, K0, L0, 1e-6)
    assert sorted(zip(pl.dk, pl.dl)) == sorted(zip(dk, dl))


def test_pilot_readoff_through_independent_transmitter():
    """The same read-off on a pilot frame made by synth (its own IDZT and channel)."""
    M, N = 16, 16
    h = np.array([0.8 + 0.1j, -0.3 + 0.4j])
    dk = np.array([0, 2])
    dl = np.array([1, -2])
    a = np.sqrt(M * N)
    Xp = np.zeros((M, N), complex)
    Xp[M // 2, N // 2] = a
    yp = synth.channel_integer(synth.idzt(Xp), h, dk, dl)
    heff = dc.heff_readoff(zak.dzt(yp, M, N), M // 2, N // 2, a)
    pl = dc.threshold_paths(heff, M // 2, N // 2, 1e-6)
    # q = (L0 + dl) M + (K0 + dk): (2, -2) -> 106 comes before (0, 1) -> 152
    assert list(pl.dk) == [2, 0] and list(pl.dl) == [-2, 1]
    np.testing.assert_allclose(pl.h, [h[1], h[0]], atol=1e-12)


def test_threshold_order_and_truncation_brute_force():
    g = np.random.default_rng(9)
    M, N = 8, 4
    heff = (g.standard_normal((M, N)) + 1j * g.standard_normal((M, N))) * 0.1
    heff[3, 1] = 0.5
    heff[0, 3] = 0.5  # equal magnitude tie
    theta = 0.12
    heff[5, 2] = -theta  # exactly at the threshold: Eq. heff_thres's strict inequality drops it
    pl = dc.threshold_paths(heff, M // 2, N // 2, theta)
    expect = [q for q in range(M * N) if abs(heff[q % M, q // M]) > theta]
    assert list(pl.lp * M + pl.kp) == expect
    assert 2 * M + 5 not in expect
    assert not pl.truncated
    for p_max in (1, 2, 3, len(expect) - 1):
        pt = dc.threshold_paths(heff, M // 2, N // 2, theta, p_max=p_max)
        ranked = sorted(expect, key=lambda q: (-abs(heff[q % M, q // M]), q))[:p_max]
        assert list(pt.lp * M + pt.kp) == sorted(ranked)
        assert pt.truncated
    # region restriction for an embedded pilot: delay offsets [0, 2] only
    reg = dc.readoff_region(M, N, M // 2, N // 2, (0, 2))
    pr = dc.threshold_paths(heff, M // 2, N // 2, theta, region=reg)
    assert all(0 <= d <= 2 for d in pr.dk)
