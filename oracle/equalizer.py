"""LMMSE equalisation of y = H x + w in the DD domain, FP64.

Test infrastructure only (see :mod:`oracle`).

Passages followed:

* Eq. sparse_mvm / Eq. D_definition: u[q] = sum_p D_{p,q} v[c_p(q)];
* Eq. sparse_herm_mvm: u[r] = sum_p conj(D_{p,q_p(r)}) v[q_p(r)];
* Algorithm 1 (Sec. IV-C, compute-aware CGA): CG on (H^H H + lambda I) x = H^H y with the
  two MVMs per iteration, scalar lambda, fixed iteration count, no early exit; optionally the
  residual-norm stopping test that Sec. IV-C describes for the original CGA (stop once the
  squared residual norm falls below a threshold), read as relative: ||c||^2 <= eps^2 ||b||^2;
* Eq. lmmse (Sec. III-B "Equalization"): x = (H^H H + R_n)^-1 H^H y with R_n = lambda I,
  solved by Cholesky as the paper suggests.

MIMO stacking (not in the paper): the unknown is x = [x_0; ...; x_{n_tx-1}] and
(Hv)_r = sum_t H_rt v_t, (H^H u)_t = sum_r H_rt^H u_r, one path list per (r, t).
"""

import numpy as np

from .ddchannel import ss_forward_map, ss_inverse_map, ss_coefficients, dense_H, heff_from_paths


def ss_forward(paths, v):
    """u = H v through the structured-sparse form, Eq. sparse_mvm (gather, multiply, reduce over p)."""
    MN = paths.M * paths.N
    v = np.asarray(v, np.complex128)
    q = np.arange(MN)
    cols = ss_forward_map(paths, q)
    D = ss_coefficients(paths, q)
    u = np.zeros(MN, np.complex128)
    for p in range(paths.P):
        u += D[p] * v[cols[p]]
    return u


def ss_adjoint(paths, v):
    """u = H^H v through the structured-sparse form, Eq. sparse_herm_mvm, with the inverse
    map of Eq. herm_mapping and the coefficient of the mapped row."""
    MN = paths.M * paths.N
    v = np.asarray(v, np.complex128)
    r = np.arange(MN)
    rows = ss_inverse_map(paths, r)
    u = np.zeros(MN, np.complex128)
    for p in range(paths.P):
        D_row = ss_coefficients(paths, rows[p], p)
        u += np.conj(D_row) * v[rows[p]]
    return u


class StackedOperator:
    """H for an n_rx x n_tx system with one path list per (r, t) pair (MIMO stacking)."""

    def __init__(self, path_grid):
        self.paths = path_grid  # list (rx) of lists (tx) of PathList
        self.n_rx = len(path_grid)
        self.n_tx = len(path_grid[0])
        self.MN = path_grid[0][0].M * path_grid[0][0].N

    def forward(self, v):
        v = np.asarray(v, np.complex128).reshape(self.n_tx, self.MN)
        out = np.zeros((self.n_rx, self.MN), np.complex128)
        for r in range(self.n_rx):
            for t in range(self.n_tx):
                out[r] += ss_forward(self.paths[r][t], v[t])
        return out.reshape(-1)

    def adjoint(self, u):
        u = np.asarray(u, np.complex128).reshape(self.n_rx, self.MN)
        out = np.zeros((self.n_tx, self.MN), np.complex128)
        for t in range(self.n_tx):
            for r in range(self.n_rx):
                out[t] += ss_adjoint(self.paths[r][t], u[r])
        return out.reshape(-1)

    def dense(self):
        """Dense stacked matrix built block by block from Eq. Hdd (tiny sizes only)."""
        blocks = [[dense_H(heff_from_paths(p), p.K0, p.L0) for p in row] for row in self.paths]
        return np.block(blocks)


def as_operator(paths):
    """Wrap a single PathList or an n_rx x n_tx grid of them as a StackedOperator."""
    if isinstance(paths, StackedOperator):
        return paths
    if isinstance(paths, (list, tuple)):
        return StackedOperator(paths)
    return StackedOperator([[paths]])


def cga(paths, y, lam, iters, history=False, eps=0.0):
    """Compute-aware CGA, Algorithm 1, in FP64.

    b = H^H y, x = 0, c = b, p = b, c_n = ||c||^2; then for each of ``iters`` iterations:
    a_p = H^H (H p) + lambda p; alpha = c_n / (p^H a_p); x += alpha p; c -= alpha a_p;
    c_n' = ||c||^2; p = c + (c_n'/c_n) p; c_n = c_n'.

    Readings where Algorithm 1 is silent: p^H a_p is taken as its real part (the system
    matrix is Hermitian positive definite); alpha = 0 when p^H a_p = 0 and beta = 0 when
    c_n = 0, so a converged noiseless run stays finite.

    eps > 0 adds the residual-norm stopping test of the original CGA (Sec. IV-C, "Profiling-
    based fixed termination"), relative to ||b||^2: no further iteration once
    c_n <= eps^2 ||b||^2, tested before the first iteration and after each update of c.
    ``iters`` stays the cap.  eps = 0 is Algorithm 1 as printed (no early exit).
    """
    op = as_operator(paths)
    b = op.adjoint(y)
    x = np.zeros_like(b)
    c = b.copy()
    p = b.copy()
    cn = float(np.vdot(c, c).real)
    stop_at = eps * eps * cn if eps > 0.0 else -1.0
    hist = [cn]
    for _ in range(iters):
        if cn <= stop_at:
            break
        a = op.adjoint(op.forward(p)) + lam * p
        pa = float(np.vdot(p, a).real)
        alpha = cn / pa if pa != 0.0 else 0.0
        x = x + alpha * p
        c = c - alpha * a
        cn_new = float(np.vdot(c, c).real)
        beta = cn_new / cn if cn != 0.0 else 0.0
        p = c + beta * p
        cn = cn_new
        hist.append(cn)
    return (x, hist) if history else x


def cg_to_convergence(paths, y, lam, rel_tol=1e-24, max_iters=None):
    """Algorithm 1's iteration run until ||c||^2 <= rel_tol ||b||^2 (or MN n_tx steps)."""
    op = as_operator(paths)
    n = op.n_tx * op.MN
    max_iters = n if max_iters is None else max_iters
    b = op.adjoint(y)
    x = np.zeros_like(b)
    c = b.copy()
    p = b.copy()
    cn = float(np.vdot(c, c).real)
    cn0 = cn
    it = 0
    while it < max_iters and cn > rel_tol * cn0:
        a = op.adjoint(op.forward(p)) + lam * p
        pa = float(np.vdot(p, a).real)
        alpha = cn / pa if pa != 0.0 else 0.0
        x = x + alpha * p
        c = c - alpha * a
        cn_new = float(np.vdot(c, c).real)
        beta = cn_new / cn if cn != 0.0 else 0.0
        p = c + beta * p
        cn = cn_new
        it += 1
    return x, it


def lmmse_direct(H, y, lam):
    """Eq. lmmse by Cholesky: solve (H^H H + lambda I) x = H^H y."""
    H = np.asarray(H, np.complex128)
    A = H.conj().T @ H + lam * np.eye(H.shape[1])
    L = np.linalg.cholesky(A)
    z = np.linalg.solve(L, H.conj().T @ np.asarray(y, np.complex128))
    return np.linalg.solve(L.conj().T, z)


__all__ = ["ss_forward", "ss_adjoint", "StackedOperator", "as_operator", "cga",
           "cg_to_convergence", "lmmse_direct"]
