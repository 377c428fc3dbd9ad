"""Allocation failures injected on the host (zotfs_debug_fail_alloc): plan, batch, server and
autotuner creation fail cleanly at every allocation they make -- ZOTFS_ENOMEM, no handle,
nothing left allocated -- and a batch created once the injection is off runs bit for bit like
one created normally.  No device work fails: the injected allocation is refused before CUDA
is asked."""

import ctypes

import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import dev, to_dev

pytestmark = pytest.mark.gpu

LEAK_BYTES = 8 << 20  # device-memory slack of the leak checks (allocation granularity)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()
    yield
    from paper_2604_02266_gb300 import _zotfs as Z
    Z.zotfs_debug_fail_alloc(-1)


def _fail_each(create, limit=160):
    """Run create(handle) with its k-th allocation failing, for k = 0, 1, ... until it
    succeeds.  Every failure must be ENOMEM and leave no handle; returns (k, handle)."""
    from paper_2604_02266_gb300 import _zotfs as Z
    for k in range(limit):
        assert Z.zotfs_debug_fail_alloc(k) == Z.OK
        h = ctypes.c_void_p()
        try:
            st = create(h)
        finally:
            Z.zotfs_debug_fail_alloc(-1)
        if st == Z.OK:
            assert h.value, k
            return k, h
        assert st == Z.ENOMEM, (k, st, Z.zotfs_last_error())
        assert h.value is None, k
    raise AssertionError(f"creation still failing after {limit} injected failures")


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("shape,reps,min_allocs", [((64, 32, 1, 1), 24, 6), ((128, 64, 4, 4), 2, 7),
                                                   ((16384, 32, 1, 1), 1, 7)])
def test_plan_creation_fails_cleanly_at_every_allocation(shape, reps, min_allocs):
    from paper_2604_02266_gb300 import _zotfs as Z
    M, N, nrx, ntx = shape

    def create(h):
        return Z.zotfs_plan_create(M, N, nrx, ntx, 0, 16, ctypes.byref(h))

    # one plan made and freed first, so that state the runtime creates lazily is not a leak
    h = ctypes.c_void_p()
    assert create(h) == Z.OK and Z.zotfs_plan_destroy(h) == Z.OK
    free0 = _free_bytes()
    for _ in range(reps):  # repeated so that leaked small tables would add up
        k, h = _fail_each(create)
        assert k >= min_allocs, k
        assert Z.zotfs_plan_destroy(h) == Z.OK
    assert free0 - _free_bytes() < LEAK_BYTES


def _frames(shapes, n, seed):
    g = np.random.default_rng(seed)
    frames, outs = [], []
    for i in range(n):
        M, N, nrx, ntx, Q = shapes[i % len(shapes)]
        b = synth.fractional_batch(1, seed=seed * 100 + i, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx,
                                   snr_db=(int(g.integers(0, 31)),))
        bps = int(np.log2(Q))
        o = {"x": torch.zeros(ntx, M * N, dtype=torch.complex64, device=dev()),
             "llr": torch.zeros(ntx, M * N, bps, device=dev()),
             "bits": torch.zeros(ntx, M * N * bps // 8, dtype=torch.uint8, device=dev()),
             "pc": torch.zeros(nrx * ntx, dtype=torch.int32, device=dev()),
             "pdk": torch.zeros(nrx * ntx * 64, dtype=torch.int16, device=dev()),
             "pdl": torch.zeros(nrx * ntx * 64, dtype=torch.int16, device=dev()),
             "ph": torch.zeros(nrx * ntx * 64, dtype=torch.complex64, device=dev())}
        # path outputs: all four or none
        frames.append(dict(M=M, N=N, n_rx=nrx, n_tx=ntx, qam=Q, iters=10, pilot_mode=0, guard=2, p_max=64,
                           in_dtype=0, noise_var=float(b["noise_var"][0]), theta=float(b["theta"][0]),
                           a_pilot=float(b["a_pilot"]), y_pilot=to_dev(b["y_pilot_td"][0]),
                           y_data=to_dev(b["y_data_td"][0]), x_hat=o["x"], llr=o["llr"], bits=o["bits"],
                           path_count=o["pc"], path_dk=o["pdk"], path_dl=o["pdl"], path_h=o["ph"]))
        outs.append(o)
    return frames, outs


def test_batch_creation_fails_cleanly_and_the_batch_still_runs():
    """Shape groups of the one-CTA kernel and a large-frame group (128x64 2x2, with its own
    global scratch); the batch created after the failures equals one created normally."""
    from paper_2604_02266_gb300 import Batch, _zotfs as Z
    frames, outs = _frames([(64, 32, 1, 1, 16), (128, 64, 2, 2, 16), (32, 16, 1, 1, 4)], 6, seed=41)
    n = len(frames)
    ref = Batch(frames)
    st_ref = torch.full((n,), -1, dtype=torch.int32, device=dev())
    ref.run(st_ref)
    torch.cuda.synchronize()
    expect = [{k: v.clone() for k, v in o.items()} for o in outs]
    for o in outs:
        for v in o.values():
            v.zero_()
    arr, keep = Batch.descriptors(frames)

    def create(h):
        return Z.zotfs_batch_create(arr, n, None, ctypes.byref(h))

    free0 = _free_bytes()
    for _ in range(3):
        k, h = _fail_each(create)
        assert k >= 5, k  # descriptors, ids, counters, two tables per shape, large-frame scratch
        assert Z.zotfs_batch_destroy(h) == Z.OK
    assert free0 - _free_bytes() < LEAK_BYTES
    k, h = _fail_each(create)
    st = torch.full((n,), -1, dtype=torch.int32, device=dev())
    try:
        assert Z.zotfs_rx_batch(h, ctypes.c_void_p(st.data_ptr()), None) == Z.OK
        torch.cuda.synchronize()
    finally:
        assert Z.zotfs_batch_destroy(h) == Z.OK
    assert torch.equal(st, st_ref)
    for o, e in zip(outs, expect):
        for key in o:
            assert torch.equal(o[key], e[key]), key
    del keep, ref


def test_server_creation_fails_cleanly_at_every_allocation():
    """Per-shape tables, the output arena and every wave's pinned and device buffers."""
    from paper_2604_02266_gb300 import _zotfs as Z
    opts = Z.zotfs_server_opts(p_max=64, max_wave_frames=16, waves_in_flight=2, keep_llr=0, arena_bytes=64 << 20,
                               max_M=128, max_N=64, max_ant=2, light_work=0)

    def create(h):
        return Z.zotfs_server_create(ctypes.byref(opts), ctypes.byref(h))

    h = ctypes.c_void_p()
    assert create(h) == Z.OK and Z.zotfs_server_destroy(h) == Z.OK
    free0 = _free_bytes()
    k, h = _fail_each(create)
    assert k >= 2 * 10 + 1, k  # tables of every shape up to 128x64, the arena, the waves' buffers
    assert Z.zotfs_server_destroy(h) == Z.OK
    assert free0 - _free_bytes() < LEAK_BYTES


def test_autotune_setup_failure_is_enomem():
    from paper_2604_02266_gb300 import Batch, _zotfs as Z
    frames, outs = _frames([(64, 32, 1, 1, 16)], 2, seed=43)
    arr, keep = Batch.descriptors(frames)
    res = (Z.zotfs_tuning_result * 1)()
    n = ctypes.c_int(-1)
    for k in (0, 1):
        assert Z.zotfs_debug_fail_alloc(k) == Z.OK
        try:
            st = Z.zotfs_autotune(arr, len(frames), None, res, 1, ctypes.byref(n), None)
        finally:
            Z.zotfs_debug_fail_alloc(-1)
        assert st == Z.ENOMEM, (k, st, Z.zotfs_last_error())
        assert n.value == 0
    del keep, outs
