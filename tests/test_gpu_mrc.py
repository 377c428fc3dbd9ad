"""GPU parity of SS-MRC (zotfs_equalize_mrc) against the FP64 oracle (oracle/mrc.py).

Both sides run on identical inputs: the library's estimated path lists (taps as stored) and
the same received frames.  The equaliser feeds hard decisions back, so its result is a
discontinuous function of the arithmetic: the test frames are chosen where no decision of the
oracle's sweeps lies within FP32 rounding of a boundary, and there the GPU's soft estimate must
match the oracle's to the equaliser tolerance and its decisions exactly."""

import ctypes as C

import numpy as np
import pytest
import torch

import synth
from oracle import mrc, qam, zak
from tests.gpu_util import TOL_X, pathlist_from_lib, rel_l2, to_dev

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


def _decisions(x, Q):
    pts = qam.constellation(Q)
    return pts[np.argmin(np.abs(np.asarray(x).reshape(-1)[:, None] - pts[None, :]) ** 2, axis=1)]


@pytest.mark.parametrize("M,N,Q,snr,iters", [(64, 32, 16, 24, 10), (32, 16, 4, 12, 10), (16, 8, 4, 20, 6),
                                             (128, 64, 16, 26, 5), (64, 64, 64, 30, 4), (256, 64, 4, 15, 3)])
def test_mrc_vs_oracle(M, N, Q, snr, iters):
    F = 4
    b = synth.fractional_batch(F, seed=9100 + M + N + Q, M=M, N=N, Q=Q, snr_db=(snr,))
    plan = Plan(M, N, 1, 1, Q)
    paths = plan.estimate(to_dev(b["y_pilot_td"]), to_dev(b["theta"]), F)
    st = torch.full((F,), -1, dtype=torch.int32, device="cuda")
    x = plan.equalize_mrc(to_dev(b["y_data_td"]), paths, iters, F, status=st).cpu().numpy()
    assert (st.cpu().numpy() == 0).all()
    lists = paths.to_host()
    for f in range(F):
        pl = pathlist_from_lib(M, N, *lists[f])
        y_dd = zak.vec(zak.dzt(b["y_data_td"][f, 0].astype(complex), M, N))
        ref, dec = mrc.mrc(pl, y_dd, iters, Q, return_decisions=True)
        assert rel_l2(x[f, 0], ref) < TOL_X, (f, rel_l2(x[f, 0], ref))
        assert np.array_equal(_decisions(x[f, 0], Q), dec), f


def test_mrc_dd_input_equals_td_input():
    M, N, Q, F, iters = 64, 32, 16, 3, 8
    b = synth.fractional_batch(F, seed=77, M=M, N=N, Q=Q, snr_db=(20,))
    plan = Plan(M, N, 1, 1, Q)
    paths = plan.estimate(to_dev(b["y_pilot_td"]), to_dev(b["theta"]), F)
    x_td = plan.equalize_mrc(to_dev(b["y_data_td"]), paths, iters, F).cpu().numpy()
    y_dd = plan.dzt(to_dev(b["y_data_td"].reshape(F, M * N)))
    x_dd = plan.equalize_mrc(y_dd, paths, iters, F, y_is_dd=True).cpu().numpy()
    assert rel_l2(x_dd, x_td) < TOL_X
    for f in range(F):
        assert np.array_equal(_decisions(x_dd[f], Q), _decisions(x_td[f], Q))


def test_mrc_noiseless_integer_4qam_bit_exact():
    M, N, Q, F = 32, 16, 4, 6
    b = synth.fractional_batch(F, seed=9, M=M, N=N, Q=Q, snr_db=(60,), integer=True)
    plan = Plan(M, N, 1, 1, Q)
    nv = to_dev(b["noise_var"])
    paths = plan.estimate(to_dev(b["y_pilot_td"]), to_dev(b["theta"]), F)
    x = plan.equalize_mrc(to_dev(b["y_data_td"]), paths, 4, F)
    _, bits = plan.demap(x, nv, F, llr=False)
    got = np.unpackbits(bits.cpu().numpy().reshape(F, -1), axis=1, bitorder="little")
    assert np.array_equal(got, b["bits"].reshape(F, -1))


def test_mrc_statuses_and_zero_iterations():
    from paper_2604_02266_gb300 import EINVAL, ENONFINITE, OK
    M, N, Q, F = 32, 16, 16, 4
    b = synth.fractional_batch(F, seed=31, M=M, N=N, Q=Q, snr_db=(20,))
    plan = Plan(M, N, 1, 1, Q)
    paths = plan.estimate(to_dev(b["y_pilot_td"]), to_dev(b["theta"]), F)
    y = b["y_data_td"].copy()
    y[3, 0, 5] = np.nan
    paths.count[1] = plan.p_max + 3
    dk = paths.dk.cpu()
    dk[2 * plan.p_max] = M // 2
    paths.dk.copy_(dk)
    st = torch.full((F,), -1, dtype=torch.int32, device="cuda")
    plan.equalize_mrc(to_dev(y), paths, 3, F, status=st)
    assert st.cpu().numpy().tolist() == [OK, EINVAL, EINVAL, ENONFINITE]
    x0 = plan.equalize_mrc(to_dev(y), paths, 0, F)
    assert (x0.cpu().numpy() == 0).all()


def test_mrc_rejects_mimo_plans():
    from paper_2604_02266_gb300 import EUNSUPPORTED, ZotfsError
    plan = Plan(32, 16, 2, 2, 16)
    paths = plan.new_paths(1)
    with pytest.raises(ZotfsError) as e:
        plan.equalize_mrc(torch.zeros(1, 2, 512, dtype=torch.complex64, device="cuda"), paths, 2, 1)
    assert e.value.status == EUNSUPPORTED
