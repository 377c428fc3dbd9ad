"""GPU parity of the paper-scale grid receiver (frames with M > 256 or M N > 16384, up to the
paper's 16384 x 32 operating point: one frame at a time on the whole GPU, a cooperative
kernel whose CTAs meet at grid barriers) against the FP64 oracle: Zak transform, read-off
(with and without truncation), operator applies, Algorithm 1 with estimated or given lists,
demapping, and independence of each frame's result from the others in the call."""

import numpy as np
import pytest
import torch

import synth
from oracle import zak, ddchannel as dc, equalizer as eq, qam
from tests.gpu_util import (TOL_LIN, TOL_LLR, TOL_X, check_path_list, dev, fill_paths, random_pathlist, rel_l2,
                            to_dev)
from tests.test_gpu_rx import _check_frames, _run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()
    yield


def Plan(*a, **k):
    from paper_2604_02266_gb300 import Plan as P
    return P(*a, **k)


@pytest.mark.parametrize("M,N,Q", [(1024, 32, 16), (512, 64, 4), (4096, 16, 64), (2048, 8, 16)])
def test_grid_rx_vs_oracle(M, N, Q):
    """(2048, 8): M > 256 with M N = 16384 -- the shortest Doppler axis, whose extension holds
    the rows twice over."""
    F = 2
    b = synth.fractional_batch(F, seed=9700 + M + N, M=M, N=N, Q=Q, snr_db=(10, 25))
    plan = Plan(M, N, 1, 1, Q)
    out = _run(plan, b, 10, F)
    torch.cuda.synchronize()
    assert set(out["status"].cpu().numpy().tolist()) <= {0, 6}
    wx, wl, mm = _check_frames(b, out, range(F), M, N, 1, 1, Q, 10, plan.p_max)
    assert wx < TOL_X and wl < TOL_LLR and mm == 0, (wx, wl, mm)


@pytest.mark.parametrize("ctas", [1, 2])
def test_grid_rx_ctas_per_sm(ctas):
    """The grid receiver at one and at two CTAs per SM (the grid barrier's arrival count and
    the per-CTA partials follow the grid size)."""
    M, N, Q, F = 1024, 32, 16, 2
    b = synth.fractional_batch(F, seed=9750 + ctas, M=M, N=N, Q=Q, snr_db=(12, 28))
    plan = Plan(M, N, 1, 1, Q)
    plan.set_tuning(ctas_per_sm=ctas)
    out = _run(plan, b, 10, F)
    torch.cuda.synchronize()
    assert set(out["status"].cpu().numpy().tolist()) <= {0, 6}
    wx, wl, mm = _check_frames(b, out, range(F), M, N, 1, 1, Q, 10, plan.p_max)
    assert wx < TOL_X and wl < TOL_LLR and mm == 0, (wx, wl, mm)


def test_grid_rx_paper_operating_point_16384x32():
    """One frame at the paper's headline grid (M, N) = (16384, 32), 16-QAM: 524288 DD bins,
    4 MB per FP32 vector."""
    M, N, Q = 16384, 32, 16
    b = synth.fractional_batch(1, seed=9800, M=M, N=N, Q=Q, snr_db=(20,))
    plan = Plan(M, N, 1, 1, Q)
    out = _run(plan, b, 10, 1)
    torch.cuda.synchronize()
    assert set(out["status"].cpu().numpy().tolist()) <= {0, 6}
    wx, wl, mm = _check_frames(b, out, range(1), M, N, 1, 1, Q, 10, plan.p_max)
    assert wx < TOL_X and wl < TOL_LLR and mm == 0, (wx, wl, mm)


@pytest.mark.parametrize("p_max", [1, 8, 256])
def test_grid_estimate_truncation(p_max):
    """zotfs_estimate on the grid receiver: threshold, stable compaction and (when more taps
    pass than p_max) the exact p_max largest, from histograms over the whole grid."""
    M, N, F = 1024, 32, 2
    b = synth.fractional_batch(F, seed=9900 + p_max, M=M, N=N, Q=16, snr_db=(30,))
    plan = Plan(M, N, 1, 1, 16, p_max=p_max)
    paths = plan.estimate(to_dev(b["y_pilot_td"]), to_dev(b["theta"]), F)
    lists = paths.to_host()
    st = paths.status.cpu().numpy()
    for f in range(F):
        heff = dc.heff_readoff(zak.dzt(b["y_pilot_td"][f, 0, 0].astype(complex), M, N), M // 2, N // 2,
                               b["a_pilot"])
        check_path_list(M, N, lists[f], heff, float(b["theta"][f]), p_max)
        ref = dc.threshold_paths(heff, M // 2, N // 2, float(b["theta"][f]), p_max)
        if ref.truncated:
            assert st[f] == 6 and len(lists[f][0]) == p_max


@pytest.mark.parametrize("theta_scale", [1e-3, 0.05])
def test_grid_estimate_many_passing_taps(theta_scale):
    """A threshold so low that more taps pass than the CTAs select among in shared memory
    (every tap at 1e-3; thousands at 0.05): the grid-wide radix select and compaction take
    over and still give the exact p_max largest in ascending q."""
    M, N, F, p_max = 1024, 32, 2, 64
    b = synth.fractional_batch(F, seed=9910, M=M, N=N, Q=16, snr_db=(10, 30))
    theta = (b["theta"] * theta_scale).astype(np.float32)
    plan = Plan(M, N, 1, 1, 16, p_max=p_max)
    paths = plan.estimate(to_dev(b["y_pilot_td"]), to_dev(theta), F)
    lists = paths.to_host()
    st = paths.status.cpu().numpy()
    for f in range(F):
        heff = dc.heff_readoff(zak.dzt(b["y_pilot_td"][f, 0, 0].astype(complex), M, N), M // 2, N // 2,
                               b["a_pilot"])
        n_pass = int((np.abs(heff) > float(theta[f])).sum())
        assert n_pass > p_max
        check_path_list(M, N, lists[f], heff, float(theta[f]), p_max)
        assert st[f] == 6 and len(lists[f][0]) == p_max


def test_grid_dzt():
    M, N, n = 2048, 16, 3
    g = np.random.default_rng(9901)
    y = (g.standard_normal((n, M * N)) + 1j * g.standard_normal((n, M * N))).astype(np.complex64)
    Y = Plan(M, N, 1, 1, 16).dzt(to_dev(y)).cpu().numpy()
    for i in range(n):
        assert rel_l2(Y[i], zak.vec(zak.dzt(y[i].astype(complex), M, N))) < TOL_LIN


def test_grid_ss_apply():
    M, N, F = 1024, 32, 2
    g = np.random.default_rng(9902)
    plan = Plan(M, N, 1, 1, 16)
    lists = [random_pathlist(g, M, N, 30) for _ in range(F)]
    paths = fill_paths(plan.new_paths(F), lists, plan.p_max)
    v = (g.standard_normal((F, 1, M * N)) + 1j * g.standard_normal((F, 1, M * N))).astype(np.complex64)
    fwd = plan.ss_apply(paths, to_dev(v), F).cpu().numpy()
    adj = plan.ss_apply(paths, to_dev(v), F, adjoint=True).cpu().numpy()
    for f in range(F):
        vf = v[f, 0].astype(complex)
        assert rel_l2(fwd[f, 0], eq.ss_forward(lists[f], vf)) < TOL_LIN
        assert rel_l2(adj[f, 0], eq.ss_adjoint(lists[f], vf)) < TOL_LIN


@pytest.mark.parametrize("y_is_dd", [False, True])
def test_grid_equalize_given_lists(y_is_dd):
    from tests.test_gpu_stages import _cg_case
    M, N, F, iters = 1024, 32, 2, 10
    b, grids = _cg_case(M, N, F, 20, seed=9903 + int(y_is_dd))
    plan = Plan(M, N, 1, 1, 16)
    paths = fill_paths(plan.new_paths(F), [g[0][0] for g in grids], plan.p_max)
    y_dd = np.stack([zak.vec(zak.dzt(b["y_data_td"][f, 0].astype(complex), M, N))[None] for f in range(F)])
    y = y_dd.astype(np.complex64) if y_is_dd else b["y_data_td"]
    x = plan.equalize(to_dev(y), paths, to_dev(b["noise_var"]), iters, F, y_is_dd=y_is_dd).cpu().numpy()
    for f in range(F):
        ref = eq.cga(grids[f], y_dd[f, 0], float(b["noise_var"][f]), iters)
        assert rel_l2(x[f].reshape(-1), ref) < TOL_X, f


def test_grid_demap():
    M, N, Q, F = 1024, 32, 64, 2
    g = np.random.default_rng(9904)
    pts = qam.constellation(Q)
    x = (pts[g.integers(0, Q, size=(F, 1, M * N))] + 0.1 * (g.standard_normal((F, 1, M * N)) +
                                                            1j * g.standard_normal((F, 1, M * N)))).astype(np.complex64)
    lam = np.array([0.05, 0.5], np.float32)
    L, B = Plan(M, N, 1, 1, Q).demap(to_dev(x), to_dev(lam), F)
    L, B = L.cpu().numpy(), B.cpu().numpy()
    for f in range(F):
        ref = qam.maxlog_llr(x[f, 0].astype(complex), float(lam[f]), Q)
        assert rel_l2(L[f, 0], ref) < TOL_LLR
        bits_ref = qam.hard_bits_from_llr(ref).reshape(-1)
        got = np.unpackbits(B[f, 0], bitorder="little")
        clear = np.abs(ref.reshape(-1)) * float(lam[f]) > 1e-4 * (2 * qam.pam_levels(Q)[0]) ** 2
        assert (got[clear] == bits_ref[clear]).all()


def test_grid_frames_in_one_call_equal_frames_alone():
    """The kernel takes a call's frames one after another on the whole grid: each frame's
    outputs are bitwise those of the same frame in a call of its own."""
    M, N, Q, F = 1024, 32, 16, 3
    b = synth.fractional_batch(F, seed=9905, M=M, N=N, Q=Q)
    plan = Plan(M, N, 1, 1, Q)
    whole = _run(plan, b, 10, F)
    for f in range(F):
        sub = {k: (v[f:f + 1] if isinstance(v, np.ndarray) and v.ndim > 0 and v.shape[0] == F else v)
               for k, v in b.items()}
        one = _run(plan, sub, 10, 1)
        torch.cuda.synchronize()
        for key in ("x_hat", "llr", "bits", "status"):
            assert torch.equal(whole[key][f:f + 1], one[key]), (f, key)


def test_grid_shapes_are_siso_only():
    from paper_2604_02266_gb300 import ZotfsError
    with pytest.raises(ZotfsError):
        Plan(1024, 32, 2, 2, 16)
    with pytest.raises(ZotfsError):
        Plan(16384, 64, 1, 1, 16)  # M N above 524288


def test_grid_embedded_pilot_is_unsupported():
    from paper_2604_02266_gb300 import PILOT_EMBEDDED, ZotfsError
    M, N, Q = 1024, 32, 4
    b = synth.fractional_batch(1, seed=9906, M=M, N=N, Q=Q)
    plan = Plan(M, N, 1, 1, Q, pilot_mode=PILOT_EMBEDDED)
    yd = to_dev(b["y_data_td"])
    with pytest.raises(ZotfsError):
        plan.rx(yd, yd, to_dev(b["noise_var"]), to_dev(b["theta"]), 10, 1)


@pytest.mark.parametrize("M,N,ctas", [(1024, 32, 2), (4096, 16, 2), (2048, 32, 1)])
def test_grid_windowed_and_global_gathers_agree(M, N, ctas):
    """The CG gathers read shared-memory windows of the extensions when every path's |dk| is
    within the launch's cap, else the global extensions.  Adding a zero-gain tap at the far
    delay M/2 - 1 changes no value but sends the frame down the global route: x is bitwise
    the same, and both match the oracle.  A second list adds a real tap 20 delays out (a wide
    window, read across the delay wrap by the first and last CTAs)."""
    F, iters = 2, 10
    b, grids = _cg_case_grid(M, N, F, seed=9960 + M + ctas)
    plan = Plan(M, N, 1, 1, 16, p_max=128)  # room for the estimated 64 taps and one more
    plan.set_tuning(ctas_per_sm=ctas)
    y = to_dev(b["y_data_td"])
    nv = to_dev(b["noise_var"])
    near = [g[0][0] for g in grids]
    far = []
    wide = []
    for pl in near:
        dk = np.append(pl.dk, M // 2 - 1)
        dl = np.append(pl.dl, 0)
        far.append(dc.PathList.from_offsets(M, N, M // 2, N // 2, np.append(pl.h, 0j), dk, dl))
        rng = np.random.default_rng(int(abs(pl.h[0]) * 1e6) % 1000)
        k_new = -20 if (-20, 3) not in set(zip(pl.dk.tolist(), pl.dl.tolist())) else 20
        wide.append(dc.PathList.from_offsets(M, N, M // 2, N // 2,
                                             np.append(pl.h, 0.05 * (rng.standard_normal() + 1j)).astype(np.complex64)
                                             .astype(complex), np.append(pl.dk, k_new), np.append(pl.dl, 3)))
    xs = {}
    for name, lists in (("near", near), ("far", far), ("wide", wide)):
        paths = fill_paths(plan.new_paths(F), lists, plan.p_max)
        xs[name] = plan.equalize(y, paths, nv, iters, F).cpu().numpy()
    assert np.array_equal(xs["near"], xs["far"])
    y_dd = [zak.vec(zak.dzt(b["y_data_td"][f, 0].astype(complex), M, N)) for f in range(F)]
    for name, lists in (("near", near), ("wide", wide)):
        for f in range(F):
            ref = eq.cga([[lists[f]]], y_dd[f], float(b["noise_var"][f]), iters)
            assert rel_l2(xs[name][f].reshape(-1), ref) < TOL_X, (name, f)


def test_grid_large_p_max_tables_in_global_memory():
    """p_max 256 at M = 16384: the CG's per-CTA coefficient tables (p_max x 54 columns) do not
    fit shared memory, so they go to global scratch and the gathers take the global route.  An
    equalisation with given lists and a read-off both still match the oracle."""
    M, N, F, iters = 16384, 16, 1, 10
    g = np.random.default_rng(9970)
    plan = Plan(M, N, 1, 1, 16, p_max=256)
    b = synth.fractional_batch(F, seed=9971, M=M, N=N, Q=16, snr_db=(20,))
    # a compact list of 24 taps near the origin (what a read-off gives), complex64 gains
    cand = [(a, c) for a in range(-4, 8) for c in range(-3, 3)]
    pick = g.choice(len(cand), size=24, replace=False)
    dk = np.array([cand[i][0] for i in pick])
    dl = np.array([cand[i][1] for i in pick])
    h = ((g.standard_normal(24) + 1j * g.standard_normal(24)) / np.sqrt(48)).astype(np.complex64).astype(complex)
    lists = [dc.PathList.from_offsets(M, N, M // 2, N // 2, h, dk, dl)]
    paths = fill_paths(plan.new_paths(F), lists, plan.p_max)
    x = plan.equalize(to_dev(b["y_data_td"]), paths, to_dev(b["noise_var"]), iters, F).cpu().numpy()
    y_dd = zak.vec(zak.dzt(b["y_data_td"][0, 0].astype(complex), M, N))
    ref = eq.cga([[lists[0]]], y_dd, float(b["noise_var"][0]), iters)
    assert rel_l2(x[0].reshape(-1), ref) < TOL_X
    est = plan.estimate(to_dev(b["y_pilot_td"]), to_dev(b["theta"]), F).to_host()
    heff = dc.heff_readoff(zak.dzt(b["y_pilot_td"][0, 0, 0].astype(complex), M, N), M // 2, N // 2, b["a_pilot"])
    check_path_list(M, N, est[0], heff, float(b["theta"][0]), 256)


def _cg_case_grid(M, N, F, seed):
    from tests.test_gpu_stages import _cg_case
    return _cg_case(M, N, F, 20, seed=seed)
