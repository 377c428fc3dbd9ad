"""Helpers shared by the GPU parity tests: moving synthetic inputs to the device, carrying
path lists between the oracle and the library, and the comparison rules.

Comparison rules:
* floating point results: relative L2 error against the FP64 oracle on identical inputs
  (x_hat <= 1e-5, LLRs <= 1e-3, Zak transform and operator applies <= 1e-5).  Ten FP32 CG
  iterations track the FP64 ones to ~1e-6 on the test frames.  The max-log LLR is a
  continuous, piecewise-linear function of x_hat, so its relative error follows x_hat's
  (2.9e-6 against 2.2e-6 in the mixed-precision tests); 1e-3 covers the x_hat bar with room
  and still catches a wrong label, sign or 1/lambda scale, which moves LLRs by O(1);
* decisions taken in floating point (a tap passing the threshold, the P_max-th largest
  tap, a hard bit) must agree wherever the oracle's margin exceeds the FP32 rounding the
  library's arithmetic can make; inside that margin either outcome is valid and the test
  checks the library's choice against the oracle's value instead.
"""

import numpy as np
import torch

from oracle import ddchannel as dc

TOL_X = 1e-5
TOL_LLR = 1e-3
TOL_LIN = 1e-5


def dev():
    return torch.device("cuda:0")


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def rel_l2(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def round_c64(h):
    return np.asarray(h, np.complex64).astype(np.complex128)


def fill_paths(paths_t, lists, p_max):
    """Write oracle PathLists (flat list, order [frame][rx][tx]) into a Paths container."""
    n = len(lists)
    cnt = np.zeros(n, np.int32)
    dk = np.zeros((n, p_max), np.int16)
    dl = np.zeros((n, p_max), np.int16)
    h = np.zeros((n, p_max), np.complex128)
    for i, pl in enumerate(lists):
        cnt[i] = pl.P
        dk[i, :pl.P] = pl.dk
        dl[i, :pl.P] = pl.dl
        h[i, :pl.P] = pl.h
    paths_t.count.copy_(torch.from_numpy(cnt))
    paths_t.dk.copy_(torch.from_numpy(dk.reshape(-1)))
    paths_t.dl.copy_(torch.from_numpy(dl.reshape(-1)))
    if paths_t.h.is_complex():
        paths_t.h.copy_(torch.from_numpy(h.reshape(-1)).to(paths_t.h.dtype))
    else:
        hh = np.stack([h.real, h.imag], -1).reshape(-1, 2)
        paths_t.h.copy_(torch.from_numpy(hh).to(paths_t.h.dtype))
    return paths_t


def pathlist_from_lib(M, N, dk, dl, h):
    """Oracle PathList from a list the library produced (taps exactly as stored)."""
    return dc.PathList.from_offsets(M, N, M // 2, N // 2, np.asarray(h, np.complex128), dk, dl)


def random_pathlist(g, M, N, P, edge=True):
    """P distinct integer offsets over the whole centred range (edges included when `edge`)."""
    cand = [(a, b) for a in range(-(M // 2), M // 2) for b in range(-(N // 2), N // 2)]
    pick = list(g.choice(len(cand), size=P, replace=False))
    if edge and P >= 3:
        pick[0] = cand.index((-(M // 2), -(N // 2)))
        pick[1] = cand.index((M // 2 - 1, N // 2 - 1))
        pick[2] = cand.index((M // 2 - 1, -(N // 2)))
        pick = list(dict.fromkeys(pick))
    dk = np.array([cand[c][0] for c in pick])
    dl = np.array([cand[c][1] for c in pick])
    h = (g.standard_normal(len(pick)) + 1j * g.standard_normal(len(pick))) / np.sqrt(2 * len(pick))
    return dc.PathList.from_offsets(M, N, M // 2, N // 2, round_c64(h), dk, dl)


def check_path_list(M, N, lib_list, heff, theta, p_max, region=None, rtol=1e-4):
    """Validate one library path list against the oracle's effective channel grid `heff`
    (uncentred pilot grid).  Returns the number of ambiguous taps.

    * every tap clearly above theta (margin > rtol) is listed unless truncation applies;
    * no tap clearly below theta is listed;
    * with truncation, the listed taps are the p_max largest up to the ambiguity margin;
    * entries are in ascending q and their gains match the oracle to FP32 accuracy.
    """
    dk, dl, h = lib_list
    K0, L0 = M // 2, N // 2
    mag = np.abs(heff)
    if region is None:
        region = np.ones((M, N), bool)
    kk = np.mod(K0 + dk, M)
    ll = np.mod(L0 + dl, N)
    q = ll * M + kk
    assert (np.diff(q) > 0).all(), "paths not in ascending q"
    assert region[kk, ll].all(), "path outside the read-off region"
    scale = max(mag.max(), 1e-30)
    np.testing.assert_allclose(h, heff[kk, ll], rtol=0, atol=2e-6 * scale)
    listed = np.zeros((M, N), bool)
    listed[kk, ll] = True
    passing = (mag > theta) & region
    amb = np.abs(mag - theta) <= rtol * theta
    n_amb = int((amb & region).sum())
    if passing.sum() <= p_max or len(dk) < p_max:
        # no truncation: the listed set is the passing set up to ambiguous taps
        bad = (listed != passing) & ~amb & region
        assert not bad.any(), f"{int(bad.sum())} unambiguous taps listed/omitted wrongly"
    else:
        assert len(dk) == p_max
        vals = np.sort(mag[passing])[::-1]
        vK = vals[p_max - 1]
        amb_k = np.abs(mag - vK) <= rtol * vK
        must = passing & (mag > vK) & ~amb_k & ~amb
        mustnot = ~passing | ((mag < vK) & ~amb_k)
        mustnot &= ~amb
        assert listed[must].all(), "a clearly top-P tap is missing"
        assert not listed[mustnot & region].any(), "a tap below the top-P cut is listed"
        n_amb += int((amb_k & passing).sum())
    return n_amb


def served_plan(M, N, nrx, ntx, Q, **opts):
    """A plan that runs a frame on the kernel the serving loop picks for it: MIMO frames too
    large for one CTA's shared memory on 2-CTA clusters, every other frame on one CTA."""
    from paper_2604_02266_gb300 import Plan
    plan = Plan(M, N, nrx, ntx, Q, **opts)
    plan.set_tuning(cluster=2 if nrx * ntx > 1 else 1)
    return plan


def one_cta_plan(M, N, nrx, ntx, Q, **opts):
    """A plan that runs every frame on one CTA (no cluster receiver): the kernels that uneven
    batches and the serving loop use, so their results can be compared bit for bit."""
    from paper_2604_02266_gb300 import Plan
    plan = Plan(M, N, nrx, ntx, Q, **opts)
    plan.set_tuning(cluster=1)
    return plan


def oracle_on_lists(lists, y_dd, lam, Q, iters, M, N, nrx, ntx, cg_eps=0.0):
    """The FP64 oracle's CGA (Algorithm 1) and max-log demapper (Eq. demod) on one frame,
    run with path lists the library produced (``lists`` in [rx][tx] order, each (dk, dl, h)
    as stored).  Returns (x_hat, LLRs [n_tx*MN, bps])."""
    from oracle import equalizer as eq, qam
    grid = [[pathlist_from_lib(M, N, *lists[r * ntx + t]) for t in range(ntx)] for r in range(nrx)]
    x = eq.cga(grid, y_dd, lam, iters, eps=cg_eps)
    return x, qam.maxlog_llr(x, lam, Q)


def hard_bit_mismatches(bits_packed, llr_ref, lam, Q):
    """Hard bits (LSB-first packed bytes of one frame) differing from the oracle's decisions,
    counted only where the oracle's LLR margin |LLR| lam exceeds 1e-4 d_min^2 (inside it
    either decision is valid)."""
    from oracle import qam
    bits = np.unpackbits(np.asarray(bits_packed, np.uint8).reshape(-1), bitorder="little")
    bref = qam.hard_bits_from_llr(llr_ref).reshape(-1)
    dmin2 = (2 * qam.pam_levels(Q)[0]) ** 2
    clear = np.abs(llr_ref.reshape(-1)) * lam > 1e-4 * dmin2
    assert bits.size == bref.size
    return int((bits[clear] != bref[clear]).sum())
