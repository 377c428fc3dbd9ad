"""GPU parity of the CG's optional residual-norm stopping test (zotfs_options.cg_eps, the
relative form of the original CGA's test described in Sec. IV-C): every kernel route stops
each frame at the iteration the FP64 oracle stops it, with the threshold chosen away from
every frame's squared-residual ratios so that FP32 rounding cannot move a decision."""

import numpy as np
import pytest
import torch

import synth
from oracle import zak, equalizer as eq
from tests.gpu_util import TOL_LLR, TOL_X, dev, pathlist_from_lib, to_dev
from tests.test_gpu_rx import _check_frames, _run

pytestmark = pytest.mark.gpu

ITERS = 10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()
    yield


def _plan(M, N, nrx, ntx, Q, cluster, **opts):
    from paper_2604_02266_gb300 import Plan
    plan = Plan(M, N, nrx, ntx, Q, **opts)
    plan.set_tuning(cluster=cluster)
    return plan


def _histories(b, lists, M, N, nrx, ntx, F):
    """Oracle ||c||^2 / ||b||^2 after 0..ITERS iterations, per frame, on the library's lists."""
    out = []
    for f in range(F):
        grid = [[pathlist_from_lib(M, N, *lists[(f * nrx + r) * ntx + t]) for t in range(ntx)] for r in range(nrx)]
        y_dd = np.concatenate([zak.vec(zak.dzt(b["y_data_td"][f, r].astype(complex), M, N)) for r in range(nrx)])
        _, hist = eq.cga(grid, y_dd, float(b["noise_var"][f]), ITERS, history=True)
        out.append(np.array(hist) / hist[0])
    return out


def _safe_eps(hists):
    """A threshold at least 5 % away from every ratio of every frame, that stops some frame
    before the iteration cap and leaves another to run longer."""
    for eps in (0.3, 0.2, 0.1, 0.07, 0.05, 0.03, 0.02, 0.01, 0.005, 0.003, 0.002, 0.001):
        e2 = eps * eps
        if any(np.min(np.abs(h / e2 - 1.0)) < 0.05 for h in hists):
            continue
        stops = [int(np.argmax(h <= e2)) if np.any(h <= e2) else ITERS + 1 for h in hists]
        if min(stops) <= ITERS - 2 and max(stops) > min(stops):
            return eps
    pytest.skip("no threshold separates these frames' residual ratios")


ROUTES = {  # name: (M, N, n_rx, n_tx, cluster, plain)
    "shared_memory": (64, 32, 1, 1, 0, False),
    "plain_form": (64, 32, 1, 1, 0, True),
    "cluster_receiver": (64, 32, 1, 1, 2, False),
    "large_frame": (128, 64, 1, 1, 1, False),
    "clustered_large_frame": (64, 32, 4, 4, 2, False),
    "paper_scale_grid": (1024, 32, 1, 1, 0, False),
}


@pytest.mark.parametrize("route", sorted(ROUTES))
def test_stopping_test_vs_oracle(route):
    M, N, nrx, ntx, cluster, plain = ROUTES[route]
    Q = 16
    F = 3 if plain else (4 if nrx > 1 or M * N > 4096 else 12)
    if M * N > 16384:
        F = 3
    b = synth.fractional_batch(F, seed=9400 + M + nrx, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx,
                               snr_db=(0, 10, 20, 30))
    first = _run(_plan(M, N, nrx, ntx, Q, cluster), b, ITERS, F, plain=plain)
    hists = _histories(b, first["paths"].to_host(), M, N, nrx, ntx, F)
    eps = _safe_eps(hists)
    plan = _plan(M, N, nrx, ntx, Q, cluster, cg_eps=eps)
    out = _run(plan, b, ITERS, F, plain=plain)
    torch.cuda.synchronize()
    assert set(out["status"].cpu().numpy().tolist()) <= {0, 6}
    wx, wl, mm = _check_frames(b, out, range(F), M, N, nrx, ntx, Q, ITERS, plan.p_max, cg_eps=eps)
    assert wx < TOL_X and wl < TOL_LLR and mm == 0, (eps, wx, wl, mm)
    # the test changed something: some frame's x differs from the fixed-iteration run
    assert not torch.equal(out["x_hat"], first["x_hat"])


def test_stopping_test_edges():
    """eps = 0 is the fixed-iteration run bit for bit; eps >= 1 stops before the first
    iteration (x = 0); a negative or non-finite eps is rejected."""
    from paper_2604_02266_gb300 import ZotfsError
    M, N, Q, F = 64, 32, 16, 6
    b = synth.fractional_batch(F, seed=9500, M=M, N=N, Q=Q)
    ref = _run(_plan(M, N, 1, 1, Q, 0), b, ITERS, F)
    zero = _run(_plan(M, N, 1, 1, Q, 0, cg_eps=0.0), b, ITERS, F)
    one = _run(_plan(M, N, 1, 1, Q, 0, cg_eps=1.0), b, ITERS, F)
    torch.cuda.synchronize()
    for key in ("x_hat", "llr", "bits", "status"):
        assert torch.equal(zero[key], ref[key]), key
    assert not one["x_hat"].abs().any()
    for bad in (-0.1, float("nan"), float("inf")):
        with pytest.raises(ZotfsError):
            _plan(M, N, 1, 1, Q, 0, cg_eps=bad)


def test_stopping_test_per_frame_in_a_batch():
    """zotfs_frame_desc.cg_eps is per frame: frames of one bucket with different thresholds
    (and none) each stop where the oracle stops them."""
    from paper_2604_02266_gb300 import Batch
    M, N, Q, F = 64, 32, 16, 8
    b = synth.fractional_batch(F, seed=9600, M=M, N=N, Q=Q, snr_db=(5, 15, 25))
    first = _run(_plan(M, N, 1, 1, Q, 0), b, ITERS, F)
    lists = first["paths"].to_host()
    hists = _histories(b, lists, M, N, 1, 1, F)
    eps = _safe_eps(hists)
    per = [eps if f % 2 == 0 else 0.0 for f in range(F)]
    bps = 4
    xs = [torch.zeros(1, M * N, dtype=torch.complex64, device=dev()) for _ in range(F)]
    bits = [torch.zeros(1, M * N * bps // 8, dtype=torch.uint8, device=dev()) for _ in range(F)]
    frames = [dict(M=M, N=N, n_rx=1, n_tx=1, qam=Q, iters=ITERS, pilot_mode=0, guard=2, p_max=64, in_dtype=0,
                   noise_var=float(b["noise_var"][f]), theta=float(b["theta"][f]), a_pilot=float(b["a_pilot"]),
                   cg_eps=per[f], y_pilot=to_dev(b["y_pilot_td"][f]), y_data=to_dev(b["y_data_td"][f]),
                   x_hat=xs[f], bits=bits[f]) for f in range(F)]
    status = torch.full((F,), -1, dtype=torch.int32, device=dev())
    Batch(frames).run(status)
    torch.cuda.synchronize()
    assert set(status.cpu().numpy().tolist()) <= {0, 6}
    for f in range(F):
        grid = [[pathlist_from_lib(M, N, *lists[f])]]
        y_dd = zak.vec(zak.dzt(b["y_data_td"][f, 0].astype(complex), M, N))
        ref = eq.cga(grid, y_dd, float(b["noise_var"][f]), ITERS, eps=per[f])
        x = xs[f].cpu().numpy().reshape(-1)
        assert np.linalg.norm(x - ref) <= TOL_X * np.linalg.norm(ref), f
