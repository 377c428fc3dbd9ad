"""GPU parity of the cluster receiver (zotfs_tuning.cluster = 2 or 4: one frame on a
thread-block cluster whose CTAs exchange the CG vectors through distributed shared memory)
against the FP64 oracle, and its agreement with the one-CTA receiver."""

import numpy as np
import pytest
import torch

import synth
from oracle import equalizer as eq, zak
from tests.gpu_util import TOL_LLR, TOL_X, dev, fill_paths, pathlist_from_lib, rel_l2, to_dev
from tests.test_gpu_rx import _check_frames

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()
    yield


def _plan(M, N, Q, cluster):
    from paper_2604_02266_gb300 import Plan
    plan = Plan(M, N, 1, 1, Q)
    plan.set_tuning(cluster=cluster)
    return plan


def _rx(plan, b, iters):
    F = len(b["noise_var"])
    return plan.rx(to_dev(b["y_pilot_td"]), to_dev(b["y_data_td"]), to_dev(b["noise_var"]), to_dev(b["theta"]),
                   iters, F, want_paths=True, want_x=True, want_llr=True)


@pytest.mark.parametrize("M,N,Q,C", [(64, 32, 16, 2), (64, 32, 16, 4), (128, 64, 16, 4), (32, 16, 64, 2),
                                     (128, 32, 4, 4)])
def test_cluster_rx_vs_oracle(M, N, Q, C):
    F = 6
    b = synth.fractional_batch(F, seed=81 + C + M, M=M, N=N, Q=Q, snr_db=(0, 10, 20, 30))
    plan = _plan(M, N, Q, C)
    out = _rx(plan, b, 10)
    torch.cuda.synchronize()
    assert set(out["status"].cpu().numpy().tolist()) <= {0, 6}
    wx, wl, mm = _check_frames(b, out, range(F), M, N, 1, 1, Q, 10, plan.p_max)
    assert wx < TOL_X and wl < TOL_LLR and mm == 0, (wx, wl, mm)


def test_cluster_matches_one_cta_receiver():
    """Same path lists bit for bit (the read-off is the same code on the same grid); the CG
    results agree to FP32 rounding (the cluster sums its reductions in another order)."""
    M, N, Q, F = 64, 32, 16, 40
    b = synth.fractional_batch(F, seed=88, M=M, N=N, Q=Q)
    one = _rx(_plan(M, N, Q, 0), b, 10)
    clu = _rx(_plan(M, N, Q, 4), b, 10)
    torch.cuda.synchronize()
    for key in ("count", "dk", "dl", "h"):
        assert torch.equal(getattr(one["paths"], key), getattr(clu["paths"], key)), key
    assert torch.equal(one["status"], clu["status"])
    assert rel_l2(clu["x_hat"].cpu().numpy(), one["x_hat"].cpu().numpy()) < 2 * TOL_X


def test_cluster_equalize_given_lists():
    """zotfs_equalize (time-domain data frames) with the cluster receiver on caller-provided
    path lists."""
    from tests.gpu_util import random_pathlist
    M, N, F = 64, 64, 4
    g = np.random.default_rng(89)
    plan = _plan(M, N, 16, 2)
    lists = [random_pathlist(g, M, N, 20) for _ in range(F)]
    paths = fill_paths(plan.new_paths(F), lists, plan.p_max)
    y = (g.standard_normal((F, 1, M * N)) + 1j * g.standard_normal((F, 1, M * N))).astype(np.complex64)
    lam = np.full(F, 0.05, np.float32)
    x = plan.equalize(to_dev(y), paths, to_dev(lam), 12, F).cpu().numpy()
    for f in range(F):
        y_dd = zak.vec(zak.dzt(y[f, 0].astype(complex), M, N))
        ref = eq.cga([[lists[f]]], y_dd, float(lam[f]), 12)
        assert rel_l2(x[f].reshape(-1), ref) < TOL_X, f


def test_automatic_cluster_for_large_frames_at_low_load():
    """With the default tuning, a SISO frame too large for the one-CTA shared-memory kernel
    (128x64) runs on a 2-CTA cluster when the call leaves SMs idle: bit for bit the same as
    asking for cluster = 2, and within tolerance of the large-frame kernel (cluster = 1)."""
    M, N, Q, F = 128, 64, 16, 2
    b = synth.fractional_batch(F, seed=90, M=M, N=N, Q=Q)
    auto = _rx(_plan(M, N, Q, 0), b, 10)
    two = _rx(_plan(M, N, Q, 2), b, 10)
    big = _rx(_plan(M, N, Q, 1), b, 10)
    torch.cuda.synchronize()
    for key in ("x_hat", "llr", "bits", "status"):
        assert torch.equal(auto[key], two[key]), key
    assert rel_l2(auto["x_hat"].cpu().numpy(), big["x_hat"].cpu().numpy()) < 2 * TOL_X


def test_cluster_request_leaves_embedded_pilot_frames_to_one_cta():
    """The cluster receivers take separate pilot frames only (an embedded pilot is removed from
    the data grid before the CG, which they do not do): zotfs_equalize on an embedded-pilot
    plan that asks for a cluster runs the one-CTA kernel, bit for bit."""
    from paper_2604_02266_gb300 import PILOT_EMBEDDED, Plan
    M, N, Q, F = 64, 32, 16, 4
    b = synth.fractional_batch(F, seed=91, M=M, N=N, Q=Q)
    yd, nv = to_dev(b["y_data_td"]), to_dev(b["noise_var"])
    xs = []
    for cl in (1, 2):
        plan = Plan(M, N, 1, 1, Q, pilot_mode=PILOT_EMBEDDED, a_pilot=b["a_pilot"], guard=2)
        plan.set_tuning(cluster=cl)
        if cl == 1:
            paths = plan.rx(yd, yd, nv, to_dev(b["theta"]), 10, F, want_paths=True)["paths"]
        xs.append(plan.equalize(yd, paths, nv, 10, F))
    torch.cuda.synchronize()
    assert torch.equal(xs[0], xs[1])
