"""GPU parity of pilot reuse (zotfs_rx_lists): one pilot frame's estimated path lists serve
the data frames that follow it through the same channel; each data frame is equalised and
demapped with its packet's lists, against the FP64 oracle, and bitwise equal to the
equalise-then-demap chain of the library's separate calls."""

import numpy as np
import pytest
import torch

import synth
from oracle import zak, ddchannel as dc, equalizer as eq, qam
from tests.gpu_util import TOL_LLR, TOL_X, check_path_list, dev, pathlist_from_lib, rel_l2, to_dev

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


def _packets_vs_oracle(M, N, nrx, ntx, Q, P, D, seed, cluster=0):
    b = synth.packet_batch(P, D, seed, M=M, N=N, Q=Q, n_rx=nrx, n_tx=ntx, snr_db=(8, 20, 30))
    plan = Plan(M, N, nrx, ntx, Q)
    plan.set_tuning(cluster=cluster)
    paths = plan.estimate(to_dev(b["y_pilot_td"]), to_dev(b["theta"]), P)
    F = P * D
    out = plan.rx_lists(to_dev(b["y_data_td"]), paths, to_dev(b["noise_var"]), 10, F,
                        path_ids=to_dev(b["path_ids"]), want_x=True, want_llr=True)
    torch.cuda.synchronize()
    assert set(out["status"].cpu().numpy().tolist()) <= {0}
    lists = paths.to_host()
    nl = nrx * ntx
    for p in range(P):  # the library's lists are valid read-offs of each packet's pilot
        for r in range(nrx):
            for t in range(ntx):
                heff = dc.heff_readoff(zak.dzt(b["y_pilot_td"][p, t, r].astype(complex), M, N), M // 2, N // 2,
                                       b["a_pilot"])
                check_path_list(M, N, lists[p * nl + r * ntx + t], heff, float(b["theta"][p]), plan.p_max)
    x = out["x_hat"].cpu().numpy()
    L = out["llr"].cpu().numpy()
    B = out["bits"].cpu().numpy()
    bps = int(np.log2(Q))
    for f in range(F):
        p = int(b["path_ids"][f])
        grid = [[pathlist_from_lib(M, N, *lists[p * nl + r * ntx + t]) for t in range(ntx)] for r in range(nrx)]
        y_dd = np.concatenate([zak.vec(zak.dzt(b["y_data_td"][f, r].astype(complex), M, N)) for r in range(nrx)])
        lam = float(b["noise_var"][f])
        ref = eq.cga(grid, y_dd, lam, 10)
        assert rel_l2(x[f].reshape(-1), ref) < TOL_X, f
        llr_ref = qam.maxlog_llr(ref, lam, Q)
        assert rel_l2(L[f].reshape(-1), llr_ref.reshape(-1)) < TOL_LLR, f
        bits = np.concatenate([np.unpackbits(B[f, t], bitorder="little") for t in range(ntx)])
        bref = qam.hard_bits_from_llr(llr_ref).reshape(-1)
        clear = np.abs(llr_ref.reshape(-1)) * lam > 1e-4 * (2 * qam.pam_levels(Q)[0]) ** 2
        assert (bits[clear] == bref[clear]).all(), f
        assert bits.size == ntx * M * N * bps
    return plan, b, paths, out


@pytest.mark.parametrize("M,N,nrx,ntx,Q,cluster", [(64, 32, 1, 1, 16, 0), (32, 16, 2, 2, 64, 0),
                                                   (64, 32, 4, 4, 16, 2), (1024, 32, 1, 1, 16, 0)])
def test_rx_lists_pilot_reuse_vs_oracle(M, N, nrx, ntx, Q, cluster):
    """Shared-memory kernel (SISO, 2x2), clustered large-frame kernel (4x4) and the
    paper-scale grid receiver (1024x32)."""
    P, D = (2, 2) if M * N * nrx * ntx > 16384 else (4, 3)
    _packets_vs_oracle(M, N, nrx, ntx, Q, P, D, seed=9950 + M + nrx, cluster=cluster)


def test_rx_lists_equals_equalize_then_demap():
    """More data frames than resident CTAs (frames taken heaviest first, by the path counts of
    each frame's list set): bitwise the equalize-then-demap chain on the lists repeated per
    data frame."""
    M, N, Q, P, D = 64, 32, 16, 48, 8
    b = synth.packet_batch(P, D, 9960, M=M, N=N, Q=Q)
    plan = Plan(M, N, 1, 1, Q)
    paths = plan.estimate(to_dev(b["y_pilot_td"]), to_dev(b["theta"]), P)
    F = P * D
    out = plan.rx_lists(to_dev(b["y_data_td"]), paths, to_dev(b["noise_var"]), 10, F,
                        path_ids=to_dev(b["path_ids"]), want_x=True, want_llr=True)
    ids = torch.from_numpy(b["path_ids"].astype(np.int64)).to(dev())
    full = plan.new_paths(F)  # the packets' lists repeated per data frame
    full.count.copy_(paths.count[ids])
    full.dk.copy_(paths.dk.view(P, -1)[ids].reshape(-1))
    full.dl.copy_(paths.dl.view(P, -1)[ids].reshape(-1))
    full.h.copy_(paths.h.view(P, -1)[ids].reshape(-1))
    x = plan.equalize(to_dev(b["y_data_td"]), full, to_dev(b["noise_var"]), 10, F)
    L, B = plan.demap(x, to_dev(b["noise_var"]), F)
    torch.cuda.synchronize()
    assert torch.equal(x, out["x_hat"])
    assert torch.equal(L, out["llr"])
    assert torch.equal(B, out["bits"])


def test_rx_lists_bad_list_id():
    from paper_2604_02266_gb300 import EINVAL
    M, N, Q, P, D = 32, 16, 4, 2, 2
    b = synth.packet_batch(P, D, 9970, M=M, N=N, Q=Q)
    plan = Plan(M, N, 1, 1, Q)
    paths = plan.estimate(to_dev(b["y_pilot_td"]), to_dev(b["theta"]), P)
    ids = b["path_ids"].copy()
    ids[1] = 7  # outside the two sets
    out = plan.rx_lists(to_dev(b["y_data_td"]), paths, to_dev(b["noise_var"]), 10, P * D, path_ids=to_dev(ids),
                        n_sets=P)
    good = plan.rx_lists(to_dev(b["y_data_td"]), paths, to_dev(b["noise_var"]), 10, P * D,
                         path_ids=to_dev(b["path_ids"]), n_sets=P)
    torch.cuda.synchronize()
    st = out["status"].cpu().numpy()
    assert st[1] == EINVAL and (st[[0, 2, 3]] == 0).all()
    for f in (0, 2, 3):
        assert torch.equal(out["bits"][f], good["bits"][f]), f


def test_rx_lists_without_ids_equals_fused_rx():
    """Without path_ids frame f takes list set f: with the lists the fused receiver estimated
    from the same pilots, the outputs are bitwise those of zotfs_rx (whose status also reports
    the read-off's truncations; loading a list truncates nothing)."""
    M, N, Q, F = 64, 32, 16, 16
    b = synth.fractional_batch(F, seed=9980, M=M, N=N, Q=Q)
    plan = Plan(M, N, 1, 1, Q)
    ref = plan.rx(to_dev(b["y_pilot_td"]), to_dev(b["y_data_td"]), to_dev(b["noise_var"]), to_dev(b["theta"]), 10, F,
                  want_paths=True, want_x=True, want_llr=True)
    out = plan.rx_lists(to_dev(b["y_data_td"]), ref["paths"], to_dev(b["noise_var"]), 10, F, want_x=True,
                        want_llr=True)
    torch.cuda.synchronize()
    for key in ("x_hat", "llr", "bits"):
        assert torch.equal(out[key], ref[key]), key
    assert (out["status"].cpu().numpy() == 0).all()
    assert set(ref["status"].cpu().numpy().tolist()) <= {0, 6}
