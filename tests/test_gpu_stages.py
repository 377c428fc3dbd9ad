"""GPU parity of the individual receiver stages against the FP64 oracle, through the C ABI:
Zak transform, structured-sparse applies, pilot read-off/thresholding, CGA, demapping."""

import numpy as np
import pytest
import torch

import synth
from oracle import zak, ddchannel as dc, equalizer as eq, qam, receiver
from tests.gpu_util import (TOL_LIN, TOL_LLR, TOL_X, check_path_list, dev, fill_paths, pathlist_from_lib,
                            random_pathlist, rel_l2, round_c64, to_dev)

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16), (16, 8), (32, 16), (64, 32), (32, 64), (128, 32), (64, 64), (128, 16)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()
    yield


def Plan(*a, **k):
    from paper_2604_02266_gb300 import Plan as P
    return P(*a, **k)


# ------------------------------------------------------------------------ Zak transform

@pytest.mark.parametrize("M,N", SHAPES)
@pytest.mark.parametrize("radix", [2, 4])
def test_dzt(M, N, radix):
    g = np.random.default_rng(M * 7 + N)
    n = 7  # ragged count, several CTAs
    y = (g.standard_normal((n, M * N)) + 1j * g.standard_normal((n, M * N))).astype(np.complex64)
    plan = Plan(M, N, 1, 1, 16)
    plan.set_tuning(fft_radix=radix)
    Y = plan.dzt(to_dev(y)).cpu().numpy()
    for i in range(n):
        ref = zak.vec(zak.dzt(y[i].astype(complex), M, N))
        assert rel_l2(Y[i], ref) < TOL_LIN


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_dzt_16bit_storage(dtype):
    from paper_2604_02266_gb300 import C32_F16, C32_BF16
    M, N = 64, 32
    g = np.random.default_rng(3)
    y = g.standard_normal((5, M * N, 2)).astype(np.float32)
    tdt = torch.float16 if dtype == "f16" else torch.bfloat16
    yt = torch.from_numpy(y).to(tdt)
    yq = yt.float().numpy()  # the values the library sees
    plan = Plan(M, N, 1, 1, 16, in_dtype=C32_F16 if dtype == "f16" else C32_BF16)
    Y = plan.dzt(yt.to(dev())).cpu().numpy()
    for i in range(5):
        ref = zak.vec(zak.dzt(yq[i, :, 0] + 1j * yq[i, :, 1], M, N))
        assert rel_l2(Y[i], ref) < TOL_LIN


def test_dzt_fp64():
    from paper_2604_02266_gb300 import C128, COMPUTE_FP64
    M, N = 64, 32
    g = np.random.default_rng(9)
    y = g.standard_normal((3, M * N)) + 1j * g.standard_normal((3, M * N))
    plan = Plan(M, N, 1, 1, 16, compute=COMPUTE_FP64, in_dtype=C128)
    for radix in (2, 4):
        plan.set_tuning(fft_radix=radix)
        Y = plan.dzt(to_dev(y)).cpu().numpy()
        for i in range(3):
            assert rel_l2(Y[i], zak.vec(zak.dzt(y[i], M, N))) < 1e-13


def test_dzt_empty_batch():
    plan = Plan(64, 32, 1, 1, 16)
    y = torch.zeros(0, 64 * 32, dtype=torch.complex64, device=dev())
    out = torch.zeros(0, 64 * 32, dtype=torch.complex64, device=dev())
    plan.dzt(y, out=out)
    torch.cuda.synchronize()


# ---------------------------------------------------------- structured-sparse operator

@pytest.mark.parametrize("M,N,P", [(16, 16, 5), (64, 32, 64), (32, 64, 17), (128, 32, 40), (16, 8, 1)])
def test_ss_apply_siso(M, N, P):
    g = np.random.default_rng(P + M)
    F = 3
    plan = Plan(M, N, 1, 1, 16)
    lists = [random_pathlist(g, M, N, min(P, M * N)) for _ in range(F)]
    paths = fill_paths(plan.new_paths(F), lists, plan.p_max)
    v = (g.standard_normal((F, 1, M * N)) + 1j * g.standard_normal((F, 1, M * N))).astype(np.complex64)
    fwd = plan.ss_apply(paths, to_dev(v), F).cpu().numpy()
    adj = plan.ss_apply(paths, to_dev(v), F, adjoint=True).cpu().numpy()
    for f in range(F):
        vf = v[f, 0].astype(complex)
        assert rel_l2(fwd[f, 0], eq.ss_forward(lists[f], vf)) < TOL_LIN
        assert rel_l2(adj[f, 0], eq.ss_adjoint(lists[f], vf)) < TOL_LIN


def test_ss_apply_fp64():
    from paper_2604_02266_gb300 import C128, COMPUTE_FP64
    M, N, F = 32, 16, 2
    g = np.random.default_rng(19)
    plan = Plan(M, N, 2, 2, 16, compute=COMPUTE_FP64, tap_dtype=C128)
    grids = [[[random_pathlist(g, M, N, 7) for _ in range(2)] for _ in range(2)] for _ in range(F)]
    flat = [pl for fr in grids for row in fr for pl in row]
    paths = fill_paths(plan.new_paths(F), flat, plan.p_max)
    v = g.standard_normal((F, 2, M * N)) + 1j * g.standard_normal((F, 2, M * N))
    fwd = plan.ss_apply(paths, to_dev(v), F).cpu().numpy()
    adj = plan.ss_apply(paths, to_dev(v), F, adjoint=True).cpu().numpy()
    for f in range(F):
        op = eq.StackedOperator(grids[f])
        assert rel_l2(fwd[f].reshape(-1), op.forward(v[f].reshape(-1))) < 1e-13
        assert rel_l2(adj[f].reshape(-1), op.adjoint(v[f].reshape(-1))) < 1e-13


def test_ss_apply_matches_dense_hdd():
    """Independent of the oracle's SS formulas: compare with Eq. Hdd's dense matrix."""
    M, N = 16, 8
    g = np.random.default_rng(11)
    plan = Plan(M, N, 1, 1, 16)
    pl = random_pathlist(g, M, N, 9)
    paths = fill_paths(plan.new_paths(1), [pl], plan.p_max)
    Hd = dc.dense_H(dc.heff_from_paths(pl), M // 2, N // 2)
    v = (g.standard_normal((1, 1, M * N)) + 1j * g.standard_normal((1, 1, M * N))).astype(np.complex64)
    fwd = plan.ss_apply(paths, to_dev(v), 1).cpu().numpy()[0, 0]
    adj = plan.ss_apply(paths, to_dev(v), 1, adjoint=True).cpu().numpy()[0, 0]
    assert rel_l2(fwd, Hd @ v[0, 0].astype(complex)) < TOL_LIN
    assert rel_l2(adj, Hd.conj().T @ v[0, 0].astype(complex)) < TOL_LIN


@pytest.mark.parametrize("nrx,ntx,M,N", [(2, 2, 32, 32), (2, 1, 64, 16), (1, 2, 32, 16), (4, 4, 32, 16), (3, 2, 16, 16)])
def test_ss_apply_mimo(nrx, ntx, M, N):
    g = np.random.default_rng(nrx * 10 + ntx)
    F = 2
    plan = Plan(M, N, nrx, ntx, 16)
    grids = [[[random_pathlist(g, M, N, 6) for _ in range(ntx)] for _ in range(nrx)] for _ in range(F)]
    flat = [pl for fr in grids for row in fr for pl in row]
    paths = fill_paths(plan.new_paths(F), flat, plan.p_max)
    v = (g.standard_normal((F, ntx, M * N)) + 1j * g.standard_normal((F, ntx, M * N))).astype(np.complex64)
    u = (g.standard_normal((F, nrx, M * N)) + 1j * g.standard_normal((F, nrx, M * N))).astype(np.complex64)
    fwd = plan.ss_apply(paths, to_dev(v), F).cpu().numpy()
    adj = plan.ss_apply(paths, to_dev(u), F, adjoint=True).cpu().numpy()
    for f in range(F):
        op = eq.StackedOperator(grids[f])
        assert rel_l2(fwd[f].reshape(-1), op.forward(v[f].reshape(-1).astype(complex))) < TOL_LIN
        assert rel_l2(adj[f].reshape(-1), op.adjoint(u[f].reshape(-1).astype(complex))) < TOL_LIN


def test_ss_apply_zero_paths_and_bad_entries():
    from paper_2604_02266_gb300 import EINVAL, OK
    M, N = 32, 16
    plan = Plan(M, N, 1, 1, 16)
    paths = plan.new_paths(2)
    paths.count.copy_(torch.tensor([0, 2], dtype=torch.int32))
    paths.dk[plan.p_max:plan.p_max + 2] = torch.tensor([1, M], dtype=torch.int16)  # second entry out of range
    paths.dl[plan.p_max:plan.p_max + 2] = torch.tensor([0, 0], dtype=torch.int16)
    paths.h[plan.p_max:plan.p_max + 2] = torch.tensor([1 + 0j, 1 + 0j], dtype=torch.complex64)
    v = torch.ones(2, 1, M * N, dtype=torch.complex64, device=dev())
    st = torch.full((2,), -1, dtype=torch.int32, device=dev())
    out = plan.ss_apply(paths, v, 2, status=st).cpu().numpy()
    assert np.abs(out[0]).max() == 0.0
    assert st.cpu().tolist() == [OK, EINVAL]


# ------------------------------------------------------------------- channel estimation

@pytest.mark.parametrize("snr", [0, 10, 20, 30])
def test_estimate_separate_pilot(snr):
    M, N, F = 64, 32, 12
    b = synth.fractional_batch(F, seed=500 + snr, M=M, N=N, Q=16, snr_db=(snr,))
    plan = Plan(M, N, 1, 1, 16)
    paths = plan.estimate(to_dev(b["y_pilot_td"]), to_dev(b["theta"]), F)
    lists = paths.to_host()
    st = paths.status.cpu().numpy()
    for f in range(F):
        heff = dc.heff_readoff(zak.dzt(b["y_pilot_td"][f, 0, 0].astype(complex), M, N), M // 2, N // 2,
                               b["a_pilot"])
        check_path_list(M, N, lists[f], heff, float(b["theta"][f]), plan.p_max)
        ref = dc.threshold_paths(heff, M // 2, N // 2, float(b["theta"][f]), plan.p_max)
        assert (st[f] == 6) == ref.truncated or abs(len(lists[f][0]) - ref.P) <= 1


@pytest.mark.parametrize("p_max", [1, 7, 64, 256])
def test_estimate_truncation(p_max):
    M, N, F = 32, 16, 6
    b = synth.fractional_batch(F, seed=77, M=M, N=N, Q=16, snr_db=(30,))
    plan = Plan(M, N, 1, 1, 16, p_max=p_max)
    paths = plan.estimate(to_dev(b["y_pilot_td"]), to_dev(b["theta"]), F)
    lists = paths.to_host()
    for f in range(F):
        heff = dc.heff_readoff(zak.dzt(b["y_pilot_td"][f, 0, 0].astype(complex), M, N), M // 2, N // 2,
                               b["a_pilot"])
        check_path_list(M, N, lists[f], heff, float(b["theta"][f]), p_max)


def test_estimate_embedded_pilot_c1():
    from paper_2604_02266_gb300 import PILOT_EMBEDDED
    frs = [synth.integer_embedded_frame(s) for s in range(40, 48)]
    M = N = 16
    plan = Plan(M, N, 1, 1, 4, pilot_mode=PILOT_EMBEDDED, a_pilot=frs[0]["a_pilot"], guard=2)
    y = np.stack([fr["y_data_td"] for fr in frs]).astype(np.complex64)
    th = np.array([fr["theta"] for fr in frs], np.float32)
    paths = plan.estimate(to_dev(y), to_dev(th), len(frs))
    lists = paths.to_host()
    region = dc.readoff_region(M, N, 8, 8, (0, 2))
    for f, fr in enumerate(frs):
        heff = dc.heff_readoff(zak.dzt(y[f].astype(complex), M, N), 8, 8, fr["a_pilot"])
        check_path_list(M, N, lists[f], heff, float(th[f]), plan.p_max, region=region)
        assert sorted(zip(lists[f][0], lists[f][1])) == sorted(zip(fr["delays"], fr["dopplers"]))


# -------------------------------------------------------------------------- equaliser

def _cg_case(M, N, F, snr, seed, nrx=1, ntx=1, Q=16, iters=10, dtype=np.complex64):
    b = synth.fractional_batch(F, seed=seed, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx, snr_db=(snr,), dtype=dtype)
    grids = []
    for f in range(F):
        grid = [[receiver.estimate(b["y_pilot_td"][f, t, r].astype(complex), M, N, M // 2, N // 2, b["a_pilot"],
                                   float(b["theta"][f]), 64) for t in range(ntx)] for r in range(nrx)]
        for row in grid:
            for pl in row:
                pl.h = round_c64(pl.h)
        grids.append(grid)
    return b, grids


@pytest.mark.parametrize("M,N,snr", [(64, 32, 0), (64, 32, 15), (64, 32, 30), (16, 16, 20), (32, 64, 25),
                                     (128, 32, 20), (64, 64, 10)])
def test_equalize_siso_vs_oracle_cga(M, N, snr):
    F, iters = 6, 10
    b, grids = _cg_case(M, N, F, snr, seed=900 + M + snr)
    plan = Plan(M, N, 1, 1, 16)
    paths = fill_paths(plan.new_paths(F), [g[0][0] for g in grids], plan.p_max)
    st = torch.full((F,), -1, dtype=torch.int32, device=dev())
    x = plan.equalize(to_dev(b["y_data_td"]), paths, to_dev(b["noise_var"]), iters, F, status=st).cpu().numpy()
    assert (st.cpu().numpy() == 0).all()
    for f in range(F):
        y_dd = zak.vec(zak.dzt(b["y_data_td"][f, 0].astype(complex), M, N))
        ref = eq.cga(grids[f][0][0], y_dd, float(b["noise_var"][f]), iters)
        assert rel_l2(x[f, 0], ref) < TOL_X, f"frame {f}"


def test_equalize_dd_input_and_iteration_counts():
    M, N, F = 64, 32, 4
    b, grids = _cg_case(M, N, F, 20, seed=31)
    plan = Plan(M, N, 1, 1, 16)
    paths = fill_paths(plan.new_paths(F), [g[0][0] for g in grids], plan.p_max)
    ydd = np.stack([zak.vec(zak.dzt(b["y_data_td"][f, 0].astype(complex), M, N)) for f in range(F)])
    ydd = ydd.astype(np.complex64)[:, None, :]
    for iters in (0, 1, 3, 30):
        x = plan.equalize(to_dev(ydd), paths, to_dev(b["noise_var"]), iters, F, y_is_dd=True).cpu().numpy()
        for f in range(F):
            ref = eq.cga(grids[f][0][0], ydd[f, 0].astype(complex), float(b["noise_var"][f]), iters)
            if iters == 0:
                assert np.abs(x[f, 0]).max() == 0.0
            else:
                assert rel_l2(x[f, 0], ref) < TOL_X, (iters, f)


@pytest.mark.parametrize("nrx,ntx,M,N", [(2, 2, 32, 32), (2, 2, 64, 16), (4, 4, 32, 16), (2, 1, 32, 32)])
def test_equalize_mimo(nrx, ntx, M, N):
    F, iters = 3, 10
    b, grids = _cg_case(M, N, F, 20, seed=70 + nrx + M, nrx=nrx, ntx=ntx)
    plan = Plan(M, N, nrx, ntx, 16)
    flat = [pl for g in grids for row in g for pl in row]
    paths = fill_paths(plan.new_paths(F), flat, plan.p_max)
    x = plan.equalize(to_dev(b["y_data_td"]), paths, to_dev(b["noise_var"]), iters, F).cpu().numpy()
    for f in range(F):
        y_dd = np.concatenate([zak.vec(zak.dzt(b["y_data_td"][f, r].astype(complex), M, N)) for r in range(nrx)])
        ref = eq.cga(grids[f], y_dd, float(b["noise_var"][f]), iters)
        assert rel_l2(x[f].reshape(-1), ref) < TOL_X


def test_equalize_fp64_vs_oracle_cga():
    """FP64 plan: 30 iterations on a 64x32 batch agree with the oracle to FP64 rounding."""
    from paper_2604_02266_gb300 import C128, COMPUTE_FP64
    M, N, F, iters = 64, 32, 4, 30
    b, grids = _cg_case(M, N, F, 25, seed=4242, dtype=np.complex128)
    plan = Plan(M, N, 1, 1, 16, compute=COMPUTE_FP64, in_dtype=C128, tap_dtype=C128)
    paths = fill_paths(plan.new_paths(F), [g[0][0] for g in grids], plan.p_max)
    x = plan.equalize(to_dev(b["y_data_td"]), paths, to_dev(b["noise_var"]), iters, F).cpu().numpy()
    for f in range(F):
        y_dd = zak.vec(zak.dzt(b["y_data_td"][f, 0], M, N))
        ref = eq.cga(grids[f][0][0], y_dd, float(b["noise_var"][f]), iters)
        assert rel_l2(x[f, 0], ref) < 1e-9


def test_equalize_single_path_closed_form():
    """One path: CG's first step is exact, x = H^H y / (|h|^2 + lambda)."""
    M, N = 32, 16
    plan = Plan(M, N, 1, 1, 16)
    pl = dc.PathList.from_offsets(M, N, M // 2, N // 2, round_c64([0.6 - 0.3j]), [-7], [5])
    paths = fill_paths(plan.new_paths(1), [pl], plan.p_max)
    g = np.random.default_rng(1)
    y = (g.standard_normal(M * N) + 1j * g.standard_normal(M * N)).astype(np.complex64)
    lam = np.array([0.05], np.float32)
    x = plan.equalize(to_dev(y[None, None]), paths, to_dev(lam), 3, 1, y_is_dd=True).cpu().numpy()[0, 0]
    exp = eq.ss_adjoint(pl, y.astype(complex)) / (abs(pl.h[0]) ** 2 + float(lam[0]))
    assert rel_l2(x, exp) < TOL_X


# ------------------------------------------------------------------------------ demap

@pytest.mark.parametrize("Q", [4, 16, 64])
def test_demap_vs_bruteforce(Q):
    M, N, F = 32, 16, 3
    g = np.random.default_rng(Q)
    pts = qam.constellation(Q)
    x = pts[g.integers(0, Q, size=(F, 1, M * N))] + 0.15 * (g.standard_normal((F, 1, M * N)) +
                                                           1j * g.standard_normal((F, 1, M * N)))
    x = x.astype(np.complex64)
    lam = np.array([0.02, 0.1, 1.0], np.float32)
    plan = Plan(M, N, 1, 1, Q)
    L, B = plan.demap(to_dev(x), to_dev(lam), F)
    L = L.cpu().numpy()
    B = B.cpu().numpy()
    for f in range(F):
        ref = qam.maxlog_llr(x[f, 0].astype(complex), float(lam[f]), Q)
        assert rel_l2(L[f, 0], ref) < TOL_LLR
        bits_ref = qam.hard_bits_from_llr(ref).reshape(-1)
        got = np.unpackbits(B[f, 0], bitorder="little")
        dmin2 = (2 * qam.pam_levels(Q)[0]) ** 2
        clear = (np.abs(ref.reshape(-1)) * float(lam[f]) > 1e-4 * dmin2)
        assert (got[clear] == bits_ref[clear]).all()


def test_demap_mimo_layout():
    M, N, F, Q = 16, 16, 2, 16
    g = np.random.default_rng(5)
    x = (g.standard_normal((F, 3, M * N)) + 1j * g.standard_normal((F, 3, M * N))).astype(np.complex64)
    lam = np.array([0.1, 0.3], np.float32)
    plan = Plan(M, N, 2, 3, Q)
    L, B = plan.demap(to_dev(x), to_dev(lam), F)
    for f in range(F):
        for t in range(3):
            ref = qam.maxlog_llr(x[f, t].astype(complex), float(lam[f]), Q)
            assert rel_l2(L[f, t].cpu().numpy(), ref) < TOL_LLR
