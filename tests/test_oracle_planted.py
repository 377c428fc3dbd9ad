"""Planted mistakes: each plausible slip in the oracle (a dropped term, a wrong sign, a
missing conjugate, a transposed operand) must break at least one of the pins above.
The mistakes are planted in the oracle, on the CPU, via monkeypatch."""

import numpy as np

from oracle import zak, ddchannel as dc, equalizer as eq, qam
from oracle.zak import _roots


def _physical(h, dk, dl, M, N):
    MN = M * N
    H = np.zeros((MN, MN), complex)
    for q in range(MN):
        e = np.zeros(MN, complex)
        e[q] = 1
        H[:, q] = zak.vec(zak.dzt(dc.td_channel_integer(zak.idzt(zak.unvec(e, M, N)), h, dk, dl, M, N), M, N))
    return H


def _case():
    M, N = 8, 4
    h = np.array([0.9 + 0.2j, -0.4 + 0.5j, 0.3 - 0.1j])
    dk = np.array([0, 3, -4])
    dl = np.array([1, -2, 0])
    return M, N, h, dk, dl, dc.PathList.from_offsets(M, N, M // 2, N // 2, h, dk, dl)


def _ss_ok():
    M, N, h, dk, dl, pl = _case()
    return np.abs(dc.ss_to_dense(pl) - _physical(h, dk, dl, M, N)).max() < 1e-12


def _dense_ok():
    M, N, h, dk, dl, pl = _case()
    return np.abs(dc.dense_H(dc.heff_from_paths(pl), M // 2, N // 2) - _physical(h, dk, dl, M, N)).max() < 1e-12


def test_pins_pass_unmodified():
    assert _ss_ok() and _dense_ok()


def test_dropped_wrap_term_is_caught(monkeypatch):
    def bad(paths, q, p=None):
        M, N = paths.M, paths.N
        q = np.asarray(q)
        k_q = q % M
        kp = paths.kp[:, None]
        lp = paths.lp[:, None]
        A = paths.K0 + k_q - kp
        return paths.h[:, None] * _roots((lp - paths.L0) * A, M * N)  # n l_pq M dropped
    monkeypatch.setattr(dc, "ss_coefficients", bad)
    assert not _ss_ok()


def test_wrong_offset_sign_is_caught(monkeypatch):
    orig = dc.ss_forward_map

    def bad(paths, q):
        flipped = dc.PathList(paths.M, paths.N, paths.K0, paths.L0, paths.h,
                              np.mod(2 * paths.K0 - paths.kp, paths.M), paths.lp)
        return orig(flipped, q)
    monkeypatch.setattr(dc, "ss_forward_map", bad)
    assert not _ss_ok()


def test_transposed_vectorisation_is_caught(monkeypatch):
    monkeypatch.setattr(zak, "vec", lambda X: np.asarray(X).reshape(-1, order="C"))
    monkeypatch.setattr(dc, "vec", lambda X: np.asarray(X).reshape(-1, order="C"))
    assert not _ss_ok()


def test_missing_zak_normalisation_is_caught(monkeypatch):
    orig = zak.dzt
    monkeypatch.setattr(zak, "dzt", lambda y, M, N: orig(y, M, N) * np.sqrt(N))
    x = np.random.default_rng(0).standard_normal(32) + 0j
    assert np.abs(zak.idzt(zak.dzt(x, 8, 4)) - x).max() > 1e-3


def test_wrong_dzt_sign_is_caught(monkeypatch):
    orig = zak.dzt
    monkeypatch.setattr(zak, "dzt", lambda y, M, N: np.conj(orig(np.conj(y), M, N)))
    assert not _dense_ok()


def test_missing_conjugate_in_adjoint_is_caught(monkeypatch):
    M, N, h, dk, dl, pl = _case()
    Hp = _physical(h, dk, dl, M, N)
    orig = dc.ss_coefficients
    monkeypatch.setattr(eq, "ss_coefficients", lambda paths, q, p=None: np.conj(orig(paths, q, p)))
    v = np.random.default_rng(1).standard_normal(M * N) + 1j
    assert np.abs(eq.ss_adjoint(pl, v) - Hp.conj().T @ v).max() > 1e-6


def test_dropped_regulariser_is_caught():
    """CG run on H^H H alone (lambda dropped) misses the Cholesky LMMSE solution."""
    M, N, h, dk, dl, pl = _case()
    Hd = dc.dense_H(dc.heff_from_paths(pl), M // 2, N // 2)
    y = np.random.default_rng(2).standard_normal(M * N) + 0j
    x_dir = eq.lmmse_direct(Hd, y, 0.5)
    x_bad, _ = eq.cg_to_convergence(pl, y, 0.0)
    assert np.linalg.norm(x_bad - x_dir) > 1e-3 * np.linalg.norm(x_dir)


def test_natural_binary_labels_are_caught(monkeypatch):
    monkeypatch.setattr(qam, "_gray", lambda i: i)
    pts = qam.constellation(16)
    bits = qam.label_bits(16)
    d = np.abs(pts[:, None] - pts[None, :])
    dmin = d[d > 1e-12].min()
    adj = [(bits[a] != bits[b]).sum() for a in range(16) for b in range(16) if abs(d[a, b] - dmin) < 1e-9]
    assert max(adj) > 1


# ------------------------------------------------- stopping test and iteration budget

def _stopping_pin_holds():
    """The pin of tests/test_oracle_equalizer.py's stopping test, as a predicate."""
    g = np.random.default_rng(21)
    M, N = 16, 16
    cand = [(a, b) for a in range(-3, 3) for b in range(-3, 3)]
    pick = g.choice(len(cand), size=5, replace=False)
    h = (g.standard_normal(5) + 1j * g.standard_normal(5)) / np.sqrt(10)
    pl = dc.PathList.from_offsets(M, N, M // 2, N // 2, h, [cand[c][0] for c in pick], [cand[c][1] for c in pick])
    Hd = dc.dense_H(dc.heff_from_paths(pl), M // 2, N // 2)
    lam = 0.02
    A = Hd.conj().T @ Hd + lam * np.eye(M * N)
    y = g.standard_normal(M * N) + 1j * g.standard_normal(M * N)
    b = Hd.conj().T @ y
    nb2 = float(np.vdot(b, b).real)
    _, hist = eq.cga(pl, y, lam, 12, history=True)
    k = 5
    eps = np.sqrt(np.sqrt(hist[k] * hist[k + 1]) / nb2)
    x = eq.cga(pl, y, lam, 12, eps=eps)
    r = b - A @ x
    rp = b - A @ eq.cga(pl, y, lam, k)
    return (float(np.vdot(r, r).real) <= eps * eps * nb2 and float(np.vdot(rp, rp).real) > eps * eps * nb2
            and np.array_equal(x, eq.cga(pl, y, lam, k + 1)))


def test_stopping_pin_passes_unmodified():
    assert _stopping_pin_holds()


def test_stopping_test_slips_are_caught(monkeypatch):
    """An absolute threshold (c_n <= eps^2, the form Sec. IV-C quotes for the original CGA, which
    scales with MN), or a test placed before the update of c, stops at another iteration."""
    orig = eq.cga

    def planted(absolute, before_update):
        def cga(paths, y, lam, iters, history=False, eps=0.0):
            if eps <= 0.0:
                return orig(paths, y, lam, iters, history)
            op = eq.as_operator(paths)
            b = op.adjoint(y)
            x = np.zeros_like(b)
            c = b.copy()
            p = b.copy()
            cn = float(np.vdot(c, c).real)
            stop_at = eps * eps * (1.0 if absolute else cn)
            prev = cn
            for _ in range(iters):
                if (prev if before_update else cn) <= stop_at:
                    break
                a = op.adjoint(op.forward(p)) + lam * p
                alpha = cn / float(np.vdot(p, a).real)
                x = x + alpha * p
                prev = cn
                c = c - alpha * a
                cn_new = float(np.vdot(c, c).real)
                p = c + (cn_new / cn) * p
                cn = cn_new
            return x
        return cga

    for absolute, before in ((True, False), (False, True)):
        monkeypatch.setattr(eq, "cga", planted(absolute, before))
        assert not _stopping_pin_holds(), (absolute, before)
    monkeypatch.setattr(eq, "cga", orig)


def test_iteration_criterion_slips_are_caught(monkeypatch):
    """Dividing by the new BER instead of the previous one, or dropping the zeta guard's max,
    changes a pinned convergence iteration."""
    from oracle import iterations as it

    def by_new(ber, eta=1e-2, zeta=1e-12):
        for xi in range(2, len(ber) + 1):
            prev, cur = ber[xi - 2], ber[xi - 1]
            if (prev - cur) / max(cur, zeta) < eta:
                return xi
        return len(ber)

    def no_guard(ber, eta=1e-2, zeta=1e-12):
        for xi in range(2, len(ber) + 1):
            prev, cur = ber[xi - 2], ber[xi - 1]
            r = (prev - cur) / prev if prev != 0.0 else 1.0
            if r < eta:
                return xi
        return len(ber)

    pinned = [([0.3, 0.1, 0.08, 0.07], 0.3, 3), ([0.0, 0.0, 0.0], 1e-2, 2), ([0.2, 0.1, 0.0999], 0.6, 2)]
    for fn in (by_new, no_guard):
        assert any(fn(b, eta) != want for b, eta, want in pinned), fn.__name__
    for b, eta, want in pinned:
        assert it.convergence_iteration(b, eta) == want


def test_swapped_antenna_pairing_is_caught(monkeypatch):
    """Pairing rx r with tx t's list as if it were (t, r) -- a transposed list grid -- breaks
    the noiseless MIMO pin."""
    from tests.test_oracle_equalizer import _mimo_bit_errors
    assert _mimo_bit_errors(2, 2, 50) == 0
    orig = eq.StackedOperator.__init__

    def transposed(self, grid):
        orig(self, [list(col) for col in zip(*grid)])
    monkeypatch.setattr(eq.StackedOperator, "__init__", transposed)
    assert _mimo_bit_errors(2, 2, 50) > 0


# ------------------------------------------------------------------- SS-MRC (oracle/mrc.py)

def _mrc_pins_ok():
    """The SS-MRC pins of tests/test_oracle_mrc.py on one case each."""
    from oracle import mrc
    from tests import test_oracle_mrc as T
    g = np.random.default_rng(7)
    M, N = 16, 8
    pl = T._paths(g, M, N, 6, edge=True)
    H = dc.dense_H(dc.heff_from_paths(pl), M // 2, N // 2)
    V = g.standard_normal((M, N)) + 1j * g.standard_normal((M, N))
    op_ok = np.abs(mrc.dt_to_dd(mrc.dt_apply(pl, mrc.dd_to_dt(V))) - zak.unvec(H @ zak.vec(V), M, N)).max() < 1e-12
    pl2 = T._paths(g, M, N, 6, edge=False)
    H2 = dc.dense_H(dc.heff_from_paths(pl2), M // 2, N // 2)
    x_tx = qam.constellation(4)[g.integers(0, 4, M * N)]
    y = H2 @ x_tx + 0.05 * (g.standard_normal(M * N) + 1j * g.standard_normal(M * N))
    soft, dec = mrc.mrc(pl2, y, 2, 4, return_decisions=True)
    soft_ref, dec_ref = T._dense_gauss_seidel_ls(H2, y, M, N, 2, 4)
    ls_ok = np.abs(soft - soft_ref).max() < 1e-9 and np.array_equal(dec, dec_ref)
    return bool(op_ok), bool(ls_ok)


def test_mrc_pins_pass_unmodified():
    assert _mrc_pins_ok() == (True, True)


def test_mrc_wrong_time_shift_is_caught(monkeypatch):
    from oracle import mrc
    orig = mrc.branch_gain

    def bad(paths_d, k, d, M, N):
        G, kt, f = orig(paths_d, k, d, M, N)
        return G, kt, -f  # the wrap into the previous time block taken the wrong way
    monkeypatch.setattr(mrc, "branch_gain", bad)
    assert _mrc_pins_ok() == (False, False)


def test_mrc_dropped_wrap_in_gain_phase_is_caught(monkeypatch):
    from oracle import mrc

    def bad(paths_d, k, d, M, N):
        hs, ls = paths_d
        kt, f = (k + d) % M, (k + d) // M
        n = np.arange(N)
        G = np.zeros(N, complex)
        for h, l in zip(hs, ls):
            G += h * np.exp(2j * np.pi * np.mod(l * (kt - d + n * M), M * N) / (M * N))  # f M term dropped
        return G, kt, f
    monkeypatch.setattr(mrc, "branch_gain", bad)
    assert not _mrc_pins_ok()[0]


def test_mrc_missing_conjugate_in_combining_is_caught(monkeypatch):
    from oracle import mrc

    def bad(gk, D, x_row, dy):
        g = np.zeros(len(x_row), complex)
        for G, kt, nt in gk:
            g += G * dy[kt, nt]
        c = np.asarray(x_row, complex).copy()
        ok = D > 0
        c[ok] += g[ok] / D[ok]
        return c
    monkeypatch.setattr(mrc, "combine_row", bad)
    assert _mrc_pins_ok()[1] is False


def test_mrc_dropped_decision_feedback_is_caught(monkeypatch):
    from oracle import mrc
    monkeypatch.setattr(mrc, "feed_back", lambda gk, delta, dy: None)
    assert _mrc_pins_ok()[1] is False
