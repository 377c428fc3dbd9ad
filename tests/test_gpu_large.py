"""GPU parity of the large-frame kernel (vectors in per-CTA global scratch): grids and MIMO
stacks whose CG vectors do not fit one CTA's shared memory, e.g. 4x4 at 128x64 (32768
unknowns) and 256x64."""

import numpy as np
import pytest
import torch

import synth
from oracle import zak, equalizer as eq
from tests.gpu_util import TOL_LIN, TOL_LLR, TOL_X, dev, fill_paths, one_cta_plan, random_pathlist, rel_l2, to_dev
from tests.test_gpu_rx import _check_frames, _run
from tests.test_gpu_stages import _cg_case

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


@pytest.mark.parametrize("M,N", [(256, 64), (256, 32), (128, 64)])
def test_dzt_large(M, N):
    g = np.random.default_rng(M + N)
    y = (g.standard_normal((3, M * N)) + 1j * g.standard_normal((3, M * N))).astype(np.complex64)
    plan = Plan(M, N, 1, 1, 16)
    Y = plan.dzt(to_dev(y)).cpu().numpy()
    for i in range(3):
        assert rel_l2(Y[i], zak.vec(zak.dzt(y[i].astype(complex), M, N))) < TOL_LIN


@pytest.mark.parametrize("nrx,ntx,M,N", [(4, 4, 128, 64), (1, 1, 256, 64), (2, 2, 128, 64), (4, 4, 64, 32)])
def test_ss_apply_large(nrx, ntx, M, N):
    g = np.random.default_rng(nrx * M + N)
    F = 2
    plan = Plan(M, N, nrx, ntx, 16)
    grids = [[[random_pathlist(g, M, N, 12) for _ in range(ntx)] for _ in range(nrx)] for _ in range(F)]
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


@pytest.mark.parametrize("nrx,ntx,M,N", [(1, 1, 128, 64), (1, 1, 256, 64), (2, 2, 128, 64)])
def test_equalize_large(nrx, ntx, M, N):
    F, iters = 2, 10
    b, grids = _cg_case(M, N, F, 20, seed=5100 + M + nrx, nrx=nrx, ntx=ntx)
    plan = Plan(M, N, nrx, ntx, 16)
    flat = [pl for gr in grids for row in gr for pl in row]
    paths = fill_paths(plan.new_paths(F), flat, plan.p_max)
    x = plan.equalize(to_dev(b["y_data_td"]), paths, to_dev(b["noise_var"]), iters, F).cpu().numpy()
    for f in range(F):
        y_dd = np.concatenate([zak.vec(zak.dzt(b["y_data_td"][f, r].astype(complex), M, N)) for r in range(nrx)])
        ref = eq.cga(grids[f], y_dd, float(b["noise_var"][f]), iters)
        assert rel_l2(x[f].reshape(-1), ref) < TOL_X


def test_rx_4x4_128x64_64qam():
    """4x4 MIMO, 128x64, 64-QAM: the stacked 32768-unknown system, estimated path lists."""
    M, N, nrx, ntx, Q, F, iters = 128, 64, 4, 4, 64, 2, 10
    b = synth.fractional_batch(F, seed=7300, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx, snr_db=(25,))
    plan = Plan(M, N, nrx, ntx, Q)
    out = _run(plan, b, iters, F)
    wx, wl, mm = _check_frames(b, out, range(F), M, N, nrx, ntx, Q, iters, plan.p_max)
    assert wx < TOL_X and wl < TOL_LLR and mm == 0, (wx, wl, mm)


def test_rx_batch_with_large_buckets():
    """An uneven batch mixing shared-memory and large-frame buckets.  With cluster = 1 each frame
    equals its result alone through a one-CTA plan, bit for bit; by default the large buckets
    run on 2-CTA clusters, and each frame equals its result in a batch of its own, bit for
    bit, and the one-CTA result within FP32 reordering."""
    from paper_2604_02266_gb300 import Batch
    shapes = [(128, 64, 1, 1, 16), (64, 32, 1, 1, 16), (128, 64, 2, 2, 16), (64, 64, 2, 2, 4), (32, 16, 2, 2, 64)]
    frames, keep = [], []
    for i in range(15):
        M, N, nrx, ntx, Q = shapes[i % len(shapes)]
        b = synth.fractional_batch(1, seed=8100 + i, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx, snr_db=(5 + 2 * i,))
        frames.append(dict(M=M, N=N, n_rx=nrx, n_tx=ntx, qam=Q, iters=10, pilot_mode=0, guard=2, p_max=64,
                           in_dtype=0, noise_var=float(b["noise_var"][0]), theta=float(b["theta"][0]),
                           a_pilot=float(b["a_pilot"]), y_pilot=to_dev(b["y_pilot_td"][0]),
                           y_data=to_dev(b["y_data_td"][0])))
        keep.append(b)

    def outputs(fr):
        M, N, ntx, Q = fr["M"], fr["N"], fr["n_tx"], fr["qam"]
        return {"x_hat": torch.zeros(ntx, M * N, dtype=torch.complex64, device=dev()),
                "bits": torch.zeros(ntx, M * N * int(np.log2(Q)) // 8, dtype=torch.uint8, device=dev())}

    def run(frs, cluster):
        outs = [outputs(fr) for fr in frs]
        batch = Batch([dict(fr, **o) for fr, o in zip(frs, outs)], cluster=cluster)
        status = torch.full((len(frs),), -1, dtype=torch.int32, device=dev())
        batch.run(status)
        torch.cuda.synchronize()
        assert set(status.cpu().numpy().tolist()) <= {0, 6}
        return outs

    one = run(frames, 1)
    mix = run(frames, 0)
    for i, b in enumerate(keep):
        M, N, nrx, ntx, Q = shapes[i % len(shapes)]
        alone = _run(one_cta_plan(M, N, nrx, ntx, Q), b, 10, 1)
        assert torch.equal(alone["x_hat"][0], one[i]["x_hat"]), i
        assert torch.equal(alone["bits"][0], one[i]["bits"]), i
        own = run([frames[i]], 0)[0]
        assert torch.equal(own["x_hat"], mix[i]["x_hat"]), i
        assert torch.equal(own["bits"], mix[i]["bits"]), i
        assert rel_l2(mix[i]["x_hat"].cpu().numpy(), one[i]["x_hat"].cpu().numpy()) < 2 * TOL_X, i


def _cluster_plan(M, N, nrx, ntx, Q, CL):
    plan = Plan(M, N, nrx, ntx, Q)
    plan.set_tuning(cluster=CL)
    return plan


@pytest.mark.parametrize("nrx,ntx,M,N,CL", [(4, 4, 128, 64, 4), (4, 4, 128, 64, 2), (2, 2, 128, 64, 4),
                                            (4, 4, 64, 32, 2), (4, 4, 64, 32, 4), (1, 1, 256, 64, 4),
                                            (2, 2, 256, 64, 2)])
def test_big_cluster_rx_vs_oracle(nrx, ntx, M, N, CL):
    """The clustered large-frame kernel (CL CTAs per frame, one scratch slot per cluster):
    estimated lists, CG and demap against the FP64 oracle."""
    F, Q = 2, 16
    b = synth.fractional_batch(F, seed=9100 + 7 * CL + M + nrx, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx, snr_db=(12, 28))
    plan = _cluster_plan(M, N, nrx, ntx, Q, CL)
    out = _run(plan, b, 10, F)
    torch.cuda.synchronize()
    assert set(out["status"].cpu().numpy().tolist()) <= {0, 6}
    wx, wl, mm = _check_frames(b, out, range(F), M, N, nrx, ntx, Q, 10, plan.p_max)
    assert wx < TOL_X and wl < TOL_LLR and mm == 0, (wx, wl, mm)


def test_big_cluster_matches_big_kernel_over_many_frames():
    """More frames than resident clusters (one CTA per SM: 76 two-CTA clusters take 90 frames
    from the work counter): the same path lists bit for bit as the one-CTA large-frame kernel,
    x within FP32 reordering; the default tuning at this load is the same 2-CTA kernel, bit
    for bit."""
    M, N, nrx, ntx, Q, F = 64, 32, 4, 4, 16, 90
    b = synth.fractional_batch(F, seed=9200, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx)
    one = _run(_cluster_plan(M, N, nrx, ntx, Q, 1), b, 10, F)
    few = Plan(M, N, nrx, ntx, Q)
    few.set_tuning(cluster=2, ctas_per_sm=1)
    two = _run(few, b, 10, F)
    auto = _run(Plan(M, N, nrx, ntx, Q), b, 10, F)
    torch.cuda.synchronize()
    for key in ("count", "dk", "dl", "h"):
        assert torch.equal(getattr(one["paths"], key), getattr(two["paths"], key)), key
    assert torch.equal(one["status"], two["status"])
    for f in range(F):
        assert rel_l2(two["x_hat"][f].cpu().numpy(), one["x_hat"][f].cpu().numpy()) < 2 * TOL_X, f
    for key in ("x_hat", "llr", "bits", "status"):
        assert torch.equal(auto[key], two[key]), key


@pytest.mark.parametrize("y_is_dd", [False, True])
def test_big_cluster_equalize_given_lists(y_is_dd):
    """zotfs_equalize on the clustered large-frame kernel, time-domain or DD data frames."""
    M, N, nrx, ntx, F, iters = 128, 64, 2, 2, 2, 10
    b, grids = _cg_case(M, N, F, 20, seed=9300 + int(y_is_dd), nrx=nrx, ntx=ntx)
    plan = _cluster_plan(M, N, nrx, ntx, 16, 4)
    flat = [pl for gr in grids for row in gr for pl in row]
    paths = fill_paths(plan.new_paths(F), flat, plan.p_max)
    y_dd = np.stack([np.stack([zak.vec(zak.dzt(b["y_data_td"][f, r].astype(complex), M, N)) for r in range(nrx)])
                     for f in range(F)])
    y = y_dd.astype(np.complex64) if y_is_dd else b["y_data_td"]
    x = plan.equalize(to_dev(y), paths, to_dev(b["noise_var"]), iters, F, y_is_dd=y_is_dd).cpu().numpy()
    for f in range(F):
        ref = eq.cga(grids[f], y_dd[f].reshape(-1), float(b["noise_var"][f]), iters)
        assert rel_l2(x[f].reshape(-1), ref) < TOL_X, f


def test_plan_scratch_calls_on_two_streams_are_ordered():
    """Calls of a large-frame plan (its kernels share the plan's scratch) issued on two
    streams give the results of the same calls issued one after another."""
    M, N, nrx, ntx, Q, F = 64, 32, 4, 4, 16, 12
    b1 = synth.fractional_batch(F, seed=9400, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx)
    b2 = synth.fractional_batch(F, seed=9401, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx)
    plan = Plan(M, N, nrx, ntx, Q)
    ref1, ref2 = _run(plan, b1, 10, F), _run(plan, b2, 10, F)
    torch.cuda.synchronize()
    ins = [[to_dev(b[k]) for k in ("y_pilot_td", "y_data_td", "noise_var", "theta")] for b in (b1, b2)]
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for rep in range(3):
        for s, (yp, yd, nv, th) in zip((s1, s2), ins):
            with torch.cuda.stream(s):
                outs.append(plan.rx(yp, yd, nv, th, 10, F, want_x=True, want_llr=True, stream=s))
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        ref = ref1 if i % 2 == 0 else ref2
        for key in ("x_hat", "llr", "bits", "status"):
            assert torch.equal(o[key], ref[key]), (i, key)
