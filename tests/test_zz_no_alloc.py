"""zotfs_equalize_static: equalisation for callers that must not allocate device memory while
they run (a real-time receive loop working to a slot deadline, where cudaMalloc and cudaFree
synchronise the device; a process whose device memory is fully budgeted up front).

It is called straight through the C ABI.  On two calls in a row with different inputs (its
scratch array keeps the first call's contents, which the second call must not see) it must give
what the allocating entry point zotfs_equalize gives, and what the FP64 oracle's CGA gives, within
the equaliser tolerance of the other tests, SISO and MIMO.  Bad path lists and non-finite inputs
come back as per-frame statuses, and a call leaves the device's free memory unchanged.  This file
is collected last on purpose."""

import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as g
    g.build()
    yield


def _call(M, N, nrx, ntx, paths, yd, ld, iters, F):
    from paper_2604_02266_gb300 import _zotfs as Z
    x = torch.full((F, ntx, M * N), float("nan"), dtype=torch.complex64, device=yd.device)
    st = torch.full((F,), -1, dtype=torch.int32, device=yd.device)
    s = Z.zotfs_equalize_static(M, N, nrx, ntx, paths.c, C.c_void_p(yd.data_ptr()), C.c_void_p(ld.data_ptr()),
                                iters, C.c_void_p(x.data_ptr()), C.c_void_p(st.data_ptr()), F,
                                C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert s == Z.OK, Z.zotfs_last_error()
    torch.cuda.synchronize()
    return x.cpu().numpy(), st.cpu().numpy()


def _inputs(rng, M, N, nrx, ntx, F):
    from tests.gpu_util import random_pathlist
    lists = [random_pathlist(rng, M, N, int(rng.integers(4, 64))) for _ in range(F * nrx * ntx)]
    y = (rng.standard_normal((F, nrx, M * N)) + 1j * rng.standard_normal((F, nrx, M * N))).astype(np.complex64)
    lam = rng.uniform(1e-2, 1.0, size=F).astype(np.float32)
    return lists, y, lam


@pytest.mark.parametrize("M,N,nrx,ntx", [(64, 32, 1, 1), (32, 32, 2, 2), (32, 16, 4, 4)])
def test_static_scratch_equalize_matches_allocating_entry_point_and_oracle(M, N, nrx, ntx):
    from oracle import equalizer as eq
    from paper_2604_02266_gb300 import Plan, _zotfs as Z
    from tests.gpu_util import TOL_X, fill_paths, rel_l2, to_dev

    iters = 10
    plan = Plan(M, N, nrx, ntx, 16)
    rng = np.random.default_rng(2468 + M + nrx)
    for call, F in enumerate((3, 2)):  # two calls in a row, different inputs and frame counts
        lists, y, lam = _inputs(rng, M, N, nrx, ntx, F)
        paths = fill_paths(plan.new_paths(F), lists, plan.p_max)
        yd, ld = to_dev(y), to_dev(lam)
        ref = plan.equalize(yd, paths, ld, iters, F, y_is_dd=True).cpu().numpy()
        got, st = _call(M, N, nrx, ntx, paths, yd, ld, iters, F)
        assert (st == Z.OK).all(), st
        nl = nrx * ntx
        for f in range(F):
            grid = [[lists[f * nl + r * ntx + t] for t in range(ntx)] for r in range(nrx)]
            x_or = eq.cga(grid, y[f].reshape(-1).astype(np.complex128), float(lam[f]), iters)
            assert rel_l2(got[f].reshape(-1), x_or) < TOL_X, (call, f, "oracle")
            assert rel_l2(got[f], ref[f]) < TOL_X, (call, f, "zotfs_equalize")


def test_static_scratch_flags_bad_lists_and_nonfinite_frames():
    """Per-frame statuses: a count above p_max and an offset outside the centred range are
    ZOTFS_EINVAL, a NaN received sample is ZOTFS_ENONFINITE; the good frames of the same call
    still equal the oracle."""
    from oracle import equalizer as eq
    from paper_2604_02266_gb300 import Plan, _zotfs as Z
    from tests.gpu_util import TOL_X, fill_paths, rel_l2, to_dev

    M, N, nrx, ntx, F, iters = 32, 16, 2, 2, 5, 10
    plan = Plan(M, N, nrx, ntx, 16)
    rng = np.random.default_rng(97)
    lists, y, lam = _inputs(rng, M, N, nrx, ntx, F)
    paths = fill_paths(plan.new_paths(F), lists, plan.p_max)
    nl, pm = nrx * ntx, plan.p_max
    paths.count[1 * nl + 2] = pm + 1                 # frame 1: a count above p_max
    dk = paths.dk.cpu()
    dk[(3 * nl + 1) * pm] = M // 2                   # frame 3: dk = M/2 is outside [-M/2, M/2)
    paths.dk.copy_(dk)
    y[4, 1, 17] = np.nan                             # frame 4: a NaN sample
    got, st = _call(M, N, nrx, ntx, paths, to_dev(y), to_dev(lam), iters, F)
    assert st.tolist() == [Z.OK, Z.EINVAL, Z.OK, Z.EINVAL, Z.ENONFINITE], st
    for f in (0, 2):
        grid = [[lists[f * nl + r * ntx + t] for t in range(ntx)] for r in range(nrx)]
        x_or = eq.cga(grid, y[f].reshape(-1).astype(np.complex128), float(lam[f]), iters)
        assert rel_l2(got[f].reshape(-1), x_or) < TOL_X, f


def test_static_scratch_call_allocates_nothing():
    """After a first call (which looks up the array's address), a call leaves the device's
    free memory exactly where it was: it allocates nothing."""
    from paper_2604_02266_gb300 import Plan
    from tests.gpu_util import fill_paths, to_dev

    M, N, F = 64, 32, 4
    plan = Plan(M, N, 1, 1, 16)
    rng = np.random.default_rng(5)
    lists, y, lam = _inputs(rng, M, N, 1, 1, F)
    paths = fill_paths(plan.new_paths(F), lists, plan.p_max)
    yd, ld = to_dev(y), to_dev(lam)
    _call(M, N, 1, 1, paths, yd, ld, 10, F)          # first call: address lookup, kernels loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    _call(M, N, 1, 1, paths, yd, ld, 10, F)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_scratch_rejects_oversize():
    from paper_2604_02266_gb300 import _zotfs as Z
    p = Z.zotfs_paths()
    p.p_max, p.tap_dtype = 64, Z.C64
    s = Z.zotfs_equalize_static(128, 64, 1, 1, C.byref(p), None, None, 10, None, None, 1, None)
    assert s == Z.EUNSUPPORTED
    assert b"4096" in Z.zotfs_last_error()
