"""GPU edge cases of the fused receiver: no tap above the threshold, zero CG iterations, a
frame with non-finite samples among clean ones, the smallest grid, and independence of the
per-frame results from the order in which the persistent CTAs take the frames."""

import ctypes

import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import TOL_LLR, TOL_X, dev, to_dev
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


def _rx(plan, b, iters, theta=None, y_data=None):
    th = to_dev(b["theta"] if theta is None else theta)
    yd = to_dev(b["y_data_td"]) if y_data is None else y_data
    return plan.rx(to_dev(b["y_pilot_td"]), yd, to_dev(b["noise_var"]), th, iters, len(b["noise_var"]),
                   want_paths=True, want_x=True, want_llr=True)


def test_rx_no_tap_above_threshold():
    """theta above every read-off magnitude: empty path lists, x_hat = 0, status OK, and the
    LLRs and bits of x = 0 as the oracle computes them (the Gray bits that separate inner
    from outer levels are not ties at 0)."""
    M, N, Q, F = 64, 32, 16, 4
    b = dict(synth.fractional_batch(F, seed=71, M=M, N=N, Q=Q))
    b["theta"] = np.full(F, 1e6, np.float32)
    plan = Plan(M, N, 1, 1, Q)
    out = _rx(plan, b, 10)
    torch.cuda.synchronize()
    assert (out["paths"].count.cpu().numpy() == 0).all()
    assert (out["status"].cpu().numpy() == 0).all()
    assert not out["x_hat"].abs().any()
    wx, wl, mm = _check_frames(b, out, range(F), M, N, 1, 1, Q, 10, plan.p_max)
    assert wx == 0.0 and wl < TOL_LLR and mm == 0, (wx, wl, mm)


def test_rx_zero_iterations():
    """Algorithm 1 with no iteration returns x = 0 whatever the paths; the lists still match the
    oracle's read-off."""
    M, N, Q, F = 32, 32, 4, 4
    b = synth.fractional_batch(F, seed=72, M=M, N=N, Q=Q)
    plan = Plan(M, N, 1, 1, Q)
    out = _rx(plan, b, 0)
    torch.cuda.synchronize()
    assert not out["x_hat"].abs().any()
    assert not out["bits"].any()
    wx, wl, mm = _check_frames(b, out, range(F), M, N, 1, 1, Q, 0, plan.p_max)
    assert wx == 0.0 and mm == 0


def test_rx_nonfinite_frame_is_flagged_and_isolated():
    """A NaN sample in one data frame sets that frame's status to ZOTFS_ENONFINITE; every other
    frame's outputs are bitwise those of the same batch without the NaN."""
    from paper_2604_02266_gb300 import ENONFINITE
    M, N, Q, F = 64, 32, 16, 8
    b = synth.fractional_batch(F, seed=73, M=M, N=N, Q=Q)
    plan = Plan(M, N, 1, 1, Q)
    clean = _rx(plan, b, 10)
    yd = to_dev(b["y_data_td"]).clone()
    yd[3, 0, 100] = complex(float("nan"), 0.0)
    dirty = _rx(plan, b, 10, y_data=yd)
    torch.cuda.synchronize()
    st = dirty["status"].cpu().numpy()
    assert st[3] == ENONFINITE
    others = [f for f in range(F) if f != 3]
    assert (st[others] == clean["status"].cpu().numpy()[others]).all()
    for key in ("x_hat", "llr", "bits"):
        assert torch.equal(dirty[key][others], clean[key][others]), key


@pytest.mark.parametrize("M,N,Q", [(16, 8, 4), (16, 16, 64), (256, 8, 16)])
def test_rx_small_and_ragged_grids(M, N, Q):
    b = synth.fractional_batch(3, seed=74 + M + N, M=M, N=N, Q=Q, delay_max=2, doppler_max=1)
    plan = Plan(M, N, 1, 1, Q)
    out = _run(plan, b, 10, 3)
    torch.cuda.synchronize()
    wx, wl, mm = _check_frames(b, out, range(3), M, N, 1, 1, Q, 10, plan.p_max)
    assert wx < TOL_X and wl < TOL_LLR and mm == 0, (wx, wl, mm)


def test_rx_results_do_not_depend_on_frame_order():
    """A launch with more frames than resident CTAs takes them heaviest first; per-frame
    results are bitwise those of the same frames run in small launches in index order."""
    M, N, Q, F = 64, 32, 16, 400
    b = synth.fractional_batch(F, seed=75, M=M, N=N, Q=Q)
    plan = Plan(M, N, 1, 1, Q)
    whole = _rx(plan, b, 10)
    parts = []
    for s in range(0, F, 50):
        sub = {k: (v[s:s + 50] if isinstance(v, np.ndarray) and v.ndim > 0 and v.shape[0] == F else v)
               for k, v in b.items()}
        parts.append(_rx(plan, sub, 10))
    torch.cuda.synchronize()
    for key in ("x_hat", "llr", "bits", "status"):
        assert torch.equal(whole[key], torch.cat([p[key] for p in parts])), key
    assert torch.equal(whole["paths"].count, torch.cat([p["paths"].count for p in parts]))


def test_bounded_waits_give_up_with_etimeout():
    """Failure detection without a fault: the mbarrier wait of the bulk copies and the grid
    barrier of the paper-scale receiver, each run against a condition nothing satisfies, give
    up after their poll limit and report ZOTFS_ETIMEOUT; the context stays usable (a receiver
    call afterwards matches the oracle)."""
    from paper_2604_02266_gb300 import ETIMEOUT, _zotfs as Z
    for which in (0, 1):
        st = torch.full((1,), -1, dtype=torch.int32, device=dev())
        Z.check(Z.zotfs_check_bounded_wait(which, 1 << 14, ctypes.c_void_p(st.data_ptr()), None))
        torch.cuda.synchronize()
        assert st.item() == ETIMEOUT, which
    M, N, Q, F = 32, 16, 16, 2
    b = synth.fractional_batch(F, seed=76, M=M, N=N, Q=Q)
    out = _run(Plan(M, N, 1, 1, Q), b, 10, F)
    torch.cuda.synchronize()
    wx, wl, mm = _check_frames(b, out, range(F), M, N, 1, 1, Q, 10, 64)
    assert wx < TOL_X and wl < TOL_LLR and mm == 0, (wx, wl, mm)


def test_cg_ratio_matches_ieee_division():
    """The CG's alpha / beta division (one Newton-Raphson step on an FP32 reciprocal, in FP64)
    gives the float that IEEE double division rounded to float gives, on a million random
    pairs over wide magnitude ranges; a disagreement can only come from a quotient within
    2^-44 of a float rounding boundary, and is then one unit in the last place.  Zero, tiny and
    huge divisors take the exact path."""
    import ctypes as C
    from paper_2604_02266_gb300 import _zotfs as Z
    g = np.random.default_rng(123)
    n = 1 << 20
    a = (g.uniform(0.5, 2.0, n) * 10.0 ** g.uniform(-20, 20, n)) * g.choice([-1.0, 1.0], n)
    b = (g.uniform(0.5, 2.0, n) * 10.0 ** g.uniform(-25, 25, n)) * g.choice([-1.0, 1.0], n)
    b[:6] = [0.0, 1e-35, -1e-40, 1e35, 3e-300, 1.0]
    a[:6] = [1.0, 1.0, 2.0, 5.0, 1e-290, 0.0]
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    q = torch.empty(n, dtype=torch.float32, device="cuda")
    assert Z.zotfs_check_cg_ratio(C.c_void_p(ad.data_ptr()), C.c_void_p(bd.data_ptr()), C.c_void_p(q.data_ptr()), n,
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream)) == Z.OK
    got = q.cpu().numpy()
    with np.errstate(divide="ignore", over="ignore"):
        ref = np.where(b == 0.0, 0.0, a / np.where(b == 0.0, 1.0, b)).astype(np.float32)
    diff = got.view(np.int32).astype(np.int64) - ref.view(np.int32).astype(np.int64)
    assert np.abs(diff).max() <= 1
    assert int((diff != 0).sum()) <= 4, int((diff != 0).sum())
    assert got[0] == 0.0 and got[5] == 0.0
