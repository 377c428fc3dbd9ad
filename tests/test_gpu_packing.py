"""GPU tests of frames packed into one CTA (zotfs_tuning.frames_per_cta): the shared-memory
frame kernel launched with a two-dimensional block runs several frames side by side in one CTA,
each on its own threads, slice of shared memory and named barrier.  Packed frames give bitwise
the results of one frame per CTA (through a plan and through an uneven batch), match the FP64
oracle, and the autotuner's candidates include the packings."""

import numpy as np
import pytest
import torch

import synth
from tests.gpu_util import TOL_LLR, TOL_X, to_dev
from tests.test_gpu_graph_tune import _frames, _snapshot, _zero
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


@pytest.mark.parametrize("M,N,nrx,ntx,Q", [(32, 16, 1, 1, 16), (16, 16, 1, 1, 4), (16, 8, 1, 1, 64),
                                           (32, 16, 2, 2, 16), (64, 16, 1, 1, 16)])
@pytest.mark.parametrize("fpc", [2, 4])
def test_packed_frames_equal_one_frame_per_cta_and_oracle(M, N, nrx, ntx, Q, fpc):
    F = 23  # not a multiple of the packing: the last CTA's rows run out of frames unevenly
    b = synth.fractional_batch(F, seed=6100 + M + N + fpc + nrx, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx,
                               snr_db=(5, 15, 25, 30))
    one = Plan(M, N, nrx, ntx, Q)
    ref = _run(one, b, 10, F)
    packed = Plan(M, N, nrx, ntx, Q)
    packed.set_tuning(frames_per_cta=fpc)
    assert packed.tuning()["frames_per_cta"] == fpc
    out = _run(packed, b, 10, F)
    torch.cuda.synchronize()
    for key in ("x_hat", "llr", "bits", "status"):
        assert torch.equal(out[key], ref[key]), key
    assert torch.equal(out["paths"].count, ref["paths"].count)
    wx, wl, mm = _check_frames(b, out, range(0, F, 3), M, N, nrx, ntx, Q, 10, packed.p_max)
    assert wx < TOL_X and wl < TOL_LLR and mm == 0, (wx, wl, mm)


def test_packed_buckets_in_an_uneven_batch_equal_unpacked():
    from paper_2604_02266_gb300 import Batch
    shapes = [(32, 16, 1, 1, 16), (16, 16, 1, 1, 4), (32, 16, 2, 2, 64), (64, 32, 1, 1, 16)]
    frames, keep = _frames(shapes, 40, seed=811)
    st = torch.empty(len(frames), dtype=torch.int32, device="cuda")
    Batch(frames).run(st)
    torch.cuda.synchronize()
    ref = _snapshot(keep)
    _zero(keep)
    tuning = [((M, N, r, t), {"frames_per_cta": 4 if M * N <= 512 else 2}) for (M, N, r, t, _) in shapes]
    Batch(frames, tuning=tuning).run(st)
    torch.cuda.synchronize()
    for i, (_, o) in enumerate(keep):
        for k, v in o.items():
            assert torch.equal(v, ref[i][k]), (i, k)
    assert set(st.cpu().numpy().tolist()) <= {0, 6}


def test_autotuner_times_packings_of_small_frames():
    from paper_2604_02266_gb300 import autotune, Batch
    frames, keep = _frames([(32, 16, 1, 1, 16), (16, 16, 1, 1, 4)], 16, seed=812)
    res = autotune(frames, warmup=1, reps=2, max_frames=8)
    assert len(res) == 2
    for r in res:
        assert r["frames_per_cta"] in (0, 1, 2, 4)  # 0: the default shape won
        assert r["n_candidates"] >= 6
    tuning = [((r["M"], r["N"], r["n_rx"], r["n_tx"]), r) for r in res]
    st = torch.empty(len(frames), dtype=torch.int32, device="cuda")
    Batch(frames, tuning=tuning).run(st)
    torch.cuda.synchronize()
    for i, (b, o) in enumerate(keep):
        M, N, Q = b["M"], b["N"], b["Q"]
        out = {"paths": None, "x_hat": o["x"][None], "llr": o["llr"][None], "bits": o["bits"][None]}

        class _P:  # the frame's own lists, in the Paths.to_host layout
            @staticmethod
            def to_host():
                cnt = int(o["pc"][0])
                return [(o["pdk"][:cnt].cpu().numpy().astype(int), o["pdl"][:cnt].cpu().numpy().astype(int),
                         o["ph"][:cnt].cpu().numpy().astype(complex))]
        out["paths"] = _P
        wx, wl, mm = _check_frames(b, out, [0], M, N, 1, 1, Q, 10, 64)
        assert wx < TOL_X and wl < TOL_LLR and mm == 0, (i, wx, wl, mm)
