"""zotfs_equalize_static: equalisation for callers that must not allocate device memory while
they run (a real-time receive loop, code inside stream capture, a fully budgeted process).

It is called straight through the C ABI and must give what the allocating entry point
zotfs_equalize gives on the same inputs, within the equaliser tolerance of the other tests,
on two calls in a row with different inputs (its scratch array keeps the first call's
contents, which the second call must not see).  This file is collected last on purpose."""

import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_static_scratch_equalize_matches_allocating_entry_point():
    import __graft_entry__ as g
    g.build()
    from paper_2604_02266_gb300 import Plan, _zotfs as Z
    from tests.gpu_util import TOL_X, fill_paths, random_pathlist, rel_l2, to_dev

    M, N, iters = 64, 32, 10
    plan = Plan(M, N, 1, 1, 16)
    rng = np.random.default_rng(2468)
    for call, F in enumerate((3, 2)):  # two calls in a row, different inputs and frame counts
        lists = [random_pathlist(rng, M, N, int(rng.integers(4, 64))) for _ in range(F)]
        paths = fill_paths(plan.new_paths(F), lists, plan.p_max)
        y = (rng.standard_normal((F, 1, M * N)) + 1j * rng.standard_normal((F, 1, M * N))).astype(np.complex64)
        lam = rng.uniform(1e-3, 1.0, size=F).astype(np.float32)
        yd, ld = to_dev(y), to_dev(lam)
        ref = plan.equalize(yd, paths, ld, iters, F, y_is_dd=True).cpu().numpy()
        x = torch.full((F, 1, M * N), float("nan"), dtype=torch.complex64, device=yd.device)
        st = torch.full((F,), -1, dtype=torch.int32, device=yd.device)
        s = Z.zotfs_equalize_static(M, N, 1, 1, paths.c, C.c_void_p(yd.data_ptr()), C.c_void_p(ld.data_ptr()),
                                    iters, C.c_void_p(x.data_ptr()), C.c_void_p(st.data_ptr()), F,
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert s == Z.OK, Z.zotfs_last_error()
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == Z.OK).all()
        got = x.cpu().numpy()
        for f in range(F):
            assert rel_l2(got[f, 0], ref[f, 0]) < TOL_X, (call, f)


def test_static_scratch_rejects_oversize():
    from paper_2604_02266_gb300 import _zotfs as Z
    p = Z.zotfs_paths()
    p.p_max, p.tap_dtype = 64, Z.C64
    s = Z.zotfs_equalize_static(128, 64, 1, 1, C.byref(p), None, None, 10, None, None, 1, None)
    assert s == Z.EUNSUPPORTED
    assert b"4096" in Z.zotfs_last_error()
