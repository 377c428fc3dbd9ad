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
