"""GPU tests of the serving loop (zotfs_server_*): continuous batching of frames of mixed
shapes, antenna counts and QAM orders.  Served frames of every class the server routes are
checked against the FP64 oracle (path lists against its effective channel, LLRs and hard bits
against its CGA and demapper run on the served lists); each served frame's results are also
bitwise those of the same frame run alone through zotfs_rx; memory-based admission holds
frames back until released outputs make room; arrival, admission and completion times are
consistent."""

import time

import numpy as np
import pytest
import torch

import synth
from oracle import ddchannel as dc, zak
from tests.gpu_util import (TOL_LLR, TOL_X, check_path_list, dev, hard_bit_mismatches, oracle_on_lists,
                             rel_l2, served_plan, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()
    yield


SHAPES = [(32, 16), (64, 32), (128, 16), (64, 64), (128, 32)]
ANTS = [(1, 1), (2, 2), (4, 4)]
QAMS = [4, 16, 64]


def _frames(n, seed, shapes=SHAPES, ants=ANTS):
    g = np.random.default_rng(seed)
    out = []
    for i in range(n):
        M, N = shapes[int(g.integers(0, len(shapes)))]
        nrx, ntx = ants[int(g.integers(0, len(ants)))]
        Q = QAMS[int(g.integers(0, len(QAMS)))]
        b = synth.fractional_batch(1, seed=seed * 1000 + i, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx, n_paths=8,
                                   snr_db=(int(g.integers(0, 31)),))
        out.append(dict(M=M, N=N, nrx=nrx, ntx=ntx, Q=Q, b=b, yp=to_dev(b["y_pilot_td"][0]),
                        yd=to_dev(b["y_data_td"][0]), iters=10))
    return out


def _req(Server, tag, fr):
    b = fr["b"]
    return Server.request(tag, fr["yp"], fr["yd"], fr["M"], fr["N"], fr["nrx"], fr["ntx"], fr["Q"], fr["iters"],
                          float(b["noise_var"][0]), float(b["theta"][0]))


def _drain(srv, n, timeout_s=120.0, release=False):
    got = {}
    t0 = time.time()
    while len(got) < n:
        for c in srv.poll():
            got[c.tag] = (c.status, c.arrival_ns, c.admit_ns, c.done_ns, c.n_lists)
            if release:
                srv.release(c.tag)
        assert time.time() - t0 < timeout_s, f"only {len(got)} of {n} frames completed"
        time.sleep(0.001)
    return got


def test_served_mix_equals_alone():
    from paper_2604_02266_gb300 import Plan, Server
    frames = _frames(36, seed=11)
    srv = Server(p_max=64, max_wave_frames=8, waves_in_flight=3, keep_llr=True, arena_bytes=256 << 20, max_M=128,
                 max_N=64, max_ant=4)
    try:
        # half up front, half while the first waves run
        srv.submit([_req(Server, i, fr) for i, fr in enumerate(frames[:18])])
        srv.submit([_req(Server, i + 18, fr) for i, fr in enumerate(frames[18:])])
        got = _drain(srv, len(frames))
        st = srv.stats()
        assert st["waves"] >= 3 and st["admitted"] == len(frames)
        for i, fr in enumerate(frames):
            status, t_arr, t_adm, t_done, nl = got[i]
            assert status in (0, 6), (i, status)
            assert t_arr <= t_adm <= t_done
            M, N, nrx, ntx, Q = fr["M"], fr["N"], fr["nrx"], fr["ntx"], fr["Q"]
            bps = int(np.log2(Q))
            served = srv.read(i, ntx, M * N, bps, nrx * ntx, llr=True)
            plan = served_plan(M, N, nrx, ntx, Q)
            b = fr["b"]
            alone = plan.rx(fr["yp"][None], fr["yd"][None], to_dev(b["noise_var"]), to_dev(b["theta"]), fr["iters"], 1,
                            want_paths=True, want_llr=True)
            assert np.array_equal(served["bits"], alone["bits"].cpu().numpy().reshape(-1)), i
            assert np.array_equal(served["llr"], alone["llr"].cpu().numpy().reshape(-1)), i
            assert np.array_equal(served["count"], alone["paths"].count.cpu().numpy()), i
            srv.release(i)
        assert srv.stats()["arena_in_use"] == 0
    finally:
        srv.close()


# One frame of every class the server routes differently: SISO frames on one CTA's shared
# memory and on the large-frame kernel (256 x 64, 256 x 32), MIMO frames that fit one CTA
# (2x2 32x16, 4x4 64x16) and MIMO frames too large for it, which the server runs on 2-CTA
# clusters (2x2 and 4x4 at 128x64); all three QAM orders; 8-path channels; two frames ask
# for the CG stopping test.  (M, N, n_rx, n_tx, Q, SNR dB, cg_eps)
ORACLE_CLASSES = [(64, 32, 1, 1, 16, 12, 0.0), (32, 16, 2, 2, 4, 25, 0.0), (64, 16, 4, 4, 64, 30, 0.0),
                  (128, 64, 2, 2, 16, 20, 0.0), (128, 64, 4, 4, 64, 28, 0.0), (256, 64, 1, 1, 64, 30, 0.0),
                  (256, 32, 1, 1, 4, 5, 0.0), (128, 32, 1, 1, 16, 18, 0.05), (64, 64, 2, 2, 16, 22, 0.05)]


def test_served_frames_match_oracle():
    """Every served class against the FP64 oracle: the served path lists are valid for the
    oracle's effective channel (taps above the threshold listed, gains to FP32 accuracy), and
    the oracle's CGA + max-log demapper run on exactly those lists give the served LLRs to
    1e-3 relative L2 and the served hard bits wherever the decision is not within FP32
    rounding of a boundary."""
    from paper_2604_02266_gb300 import Server
    frames = []
    for i, (M, N, nrx, ntx, Q, snr, eps) in enumerate(ORACLE_CLASSES):
        b = synth.fractional_batch(1, seed=7100 + i, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx, n_paths=8, snr_db=(snr,))
        frames.append(dict(M=M, N=N, nrx=nrx, ntx=ntx, Q=Q, eps=eps, b=b, yp=to_dev(b["y_pilot_td"][0]),
                           yd=to_dev(b["y_data_td"][0]), iters=10))
    srv = Server(p_max=64, max_wave_frames=4, waves_in_flight=3, keep_llr=True, arena_bytes=256 << 20, max_M=256,
                 max_N=64, max_ant=4)
    try:
        reqs = [Server.request(i, fr["yp"], fr["yd"], fr["M"], fr["N"], fr["nrx"], fr["ntx"], fr["Q"], fr["iters"],
                               float(fr["b"]["noise_var"][0]), float(fr["b"]["theta"][0]), cg_eps=fr["eps"])
                for i, fr in enumerate(frames)]
        srv.submit(reqs[:4])
        srv.submit(reqs[4:])  # while the first waves run
        got = _drain(srv, len(frames))
        for i, fr in enumerate(frames):
            M, N, nrx, ntx, Q, b = fr["M"], fr["N"], fr["nrx"], fr["ntx"], fr["Q"], fr["b"]
            assert got[i][0] in (0, 6), (i, got[i][0])
            nl, bps, MN = nrx * ntx, int(np.log2(Q)), M * N
            served = srv.read(i, ntx, MN, bps, nl, llr=True)
            lam, theta = float(b["noise_var"][0]), float(b["theta"][0])
            dk = served["dk"].reshape(nl, -1)
            dl = served["dl"].reshape(nl, -1)
            h = served["h"].reshape(nl, -1).astype(complex)
            lists = []
            for r in range(nrx):
                for t in range(ntx):
                    li = r * ntx + t
                    P = int(served["count"][li])
                    lst = (dk[li, :P].astype(int), dl[li, :P].astype(int), h[li, :P])
                    heff = dc.heff_readoff(zak.dzt(b["y_pilot_td"][0, t, r].astype(complex), M, N), M // 2, N // 2,
                                           b["a_pilot"])
                    check_path_list(M, N, lst, heff, theta, 64)
                    lists.append(lst)
            y_dd = np.concatenate([zak.vec(zak.dzt(b["y_data_td"][0, r].astype(complex), M, N)) for r in range(nrx)])
            _, llr_ref = oracle_on_lists(lists, y_dd, lam, Q, fr["iters"], M, N, nrx, ntx, cg_eps=fr["eps"])
            err = rel_l2(served["llr"], llr_ref.reshape(-1))
            assert err < TOL_LLR, (ORACLE_CLASSES[i], err)
            assert hard_bit_mismatches(served["bits"], llr_ref, lam, Q) == 0, ORACLE_CLASSES[i]
            srv.release(i)
    finally:
        srv.close()


def test_memory_based_admission_backpressure():
    """An arena that holds only a few frames' outputs: frames wait and are admitted as earlier
    frames are released; every frame completes and the arena never overflows."""
    from paper_2604_02266_gb300 import Server
    frames = _frames(20, seed=12, shapes=[(64, 32)], ants=[(1, 1)])
    per_frame = 64 * 32 * 6 // 8 + 4 * 256 + 64 * 12  # upper bound of one SISO 64x32 frame's outputs
    arena = 3 * 8192
    srv = Server(p_max=64, max_wave_frames=16, waves_in_flight=2, arena_bytes=arena, max_M=64, max_N=32, max_ant=1)
    try:
        srv.submit([_req(Server, i, fr) for i, fr in enumerate(frames)])
        got = _drain(srv, len(frames), release=True)
        st = srv.stats()
        assert all(v[0] in (0, 6) for v in got.values())
        assert st["arena_high_water"] <= arena
        assert st["waves"] >= len(frames) * per_frame // arena
        assert st["completed"] == st["released"] == len(frames)
    finally:
        srv.close()


def test_frame_larger_than_arena_is_rejected():
    from paper_2604_02266_gb300 import Server, ENOMEM
    fr = _frames(1, seed=13, shapes=[(128, 32)], ants=[(4, 4)])[0]
    srv = Server(p_max=64, arena_bytes=4096, max_M=128, max_N=32, max_ant=4)
    try:
        srv.submit([_req(Server, 7, fr)])
        got = _drain(srv, 1)
        assert got[7][0] == ENOMEM
        assert srv.stats()["rejected_too_large"] == 1
    finally:
        srv.close()


def test_replay_poisson_arrivals():
    """Native Poisson replay: every frame completes, latencies are positive and ordered."""
    from paper_2604_02266_gb300 import Server
    frames = _frames(64, seed=14, shapes=[(32, 16), (64, 32)], ants=[(1, 1), (2, 2)])
    rate = 20000.0
    arrivals = np.cumsum(np.random.default_rng(5).exponential(1.0 / rate, size=len(frames)))
    srv = Server(p_max=64, max_wave_frames=64, waves_in_flight=4, arena_bytes=64 << 20, max_M=64, max_N=32,
                 max_ant=2)
    try:
        srv.replay([_req(Server, i, fr) for i, fr in enumerate(frames)], arrivals)
        got = _drain(srv, len(frames), release=True)
        lat = np.array([(v[3] - v[1]) * 1e-6 for v in got.values()])
        assert (lat > 0).all()
        arr = np.array([got[i][1] for i in range(len(frames))])
        assert (np.diff(arr) >= 0).all()  # arrival stamps follow the schedule
    finally:
        srv.close()


def test_light_frames_have_their_own_queue():
    """With light_work set, small frames queue and run in their own wave slots: every frame
    completes with the same results as alone, and the heavy frames never delay the light
    ones' admission behind them."""
    from paper_2604_02266_gb300 import Plan, Server
    frames = _frames(24, seed=15, shapes=[(32, 16), (128, 64)], ants=[(1, 1), (4, 4)])
    srv = Server(p_max=64, max_wave_frames=4, waves_in_flight=4, keep_llr=True, arena_bytes=256 << 20, max_M=128,
                 max_N=64, max_ant=4, light_work=2048)
    try:
        srv.submit([_req(Server, i, fr) for i, fr in enumerate(frames)])
        got = _drain(srv, len(frames))
        for i, fr in enumerate(frames):
            assert got[i][0] in (0, 6), (i, got[i][0])
            M, N, nrx, ntx, Q = fr["M"], fr["N"], fr["nrx"], fr["ntx"], fr["Q"]
            served = srv.read(i, ntx, M * N, int(np.log2(Q)), nrx * ntx, llr=True)
            b = fr["b"]
            alone = served_plan(M, N, nrx, ntx, Q).rx(fr["yp"][None], fr["yd"][None], to_dev(b["noise_var"]),
                                               to_dev(b["theta"]), fr["iters"], 1, want_llr=True)
            assert np.array_equal(served["bits"], alone["bits"].cpu().numpy().reshape(-1)), i
            assert np.array_equal(served["llr"], alone["llr"].cpu().numpy().reshape(-1)), i
            srv.release(i)
        light = [i for i, fr in enumerate(frames) if fr["M"] * fr["N"] * fr["nrx"] * fr["ntx"] <= 2048]
        heavy = [i for i in range(len(frames)) if i not in light]
        assert light and heavy
        # all were submitted together: the light frames' admissions do not wait for heavy ones
        assert max(got[i][2] for i in light) <= max(got[i][3] for i in heavy)
    finally:
        srv.close()


def test_served_frames_with_stopping_test_equal_alone():
    """zotfs_request.cg_eps reaches the frame's kernel: served frames that ask for the CG
    stopping test equal the same frames run alone with that plan option, bit for bit."""
    from paper_2604_02266_gb300 import Server
    frames = _frames(8, seed=17, shapes=[(64, 32), (64, 64)], ants=[(1, 1), (4, 4)])
    eps = 0.05
    srv = Server(p_max=64, max_wave_frames=8, waves_in_flight=2, keep_llr=True, arena_bytes=256 << 20, max_M=128,
                 max_N=64, max_ant=4)
    try:
        reqs = []
        for i, fr in enumerate(frames):
            b = fr["b"]
            reqs.append(Server.request(i, fr["yp"], fr["yd"], fr["M"], fr["N"], fr["nrx"], fr["ntx"], fr["Q"],
                                       fr["iters"], float(b["noise_var"][0]), float(b["theta"][0]), cg_eps=eps))
        srv.submit(reqs)
        got = _drain(srv, len(frames))
        for i, fr in enumerate(frames):
            assert got[i][0] in (0, 6), (i, got[i][0])
            M, N, nrx, ntx, Q = fr["M"], fr["N"], fr["nrx"], fr["ntx"], fr["Q"]
            served = srv.read(i, ntx, M * N, int(np.log2(Q)), nrx * ntx, llr=True)
            b = fr["b"]
            alone = served_plan(M, N, nrx, ntx, Q, cg_eps=eps).rx(fr["yp"][None], fr["yd"][None],
                                                                   to_dev(b["noise_var"]), to_dev(b["theta"]),
                                                                   fr["iters"], 1, want_llr=True)
            assert np.array_equal(served["llr"], alone["llr"].cpu().numpy().reshape(-1)), i
            assert np.array_equal(served["bits"], alone["bits"].cpu().numpy().reshape(-1)), i
            srv.release(i)
    finally:
        srv.close()
