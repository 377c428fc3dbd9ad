"""BER-driven choice of the CG iteration budget (Sec. IV-C, "BER-driven iteration selection",
Eq. ber_convergence).  Test infrastructure only (see :mod:`oracle`).

The signed relative BER change between consecutive iterations is
    r_xi = (BER_{xi-1} - BER_xi) / max(BER_{xi-1}, zeta),
the BER has converged at the first xi >= 2 with r_xi < eta, and the iteration budget is the
largest convergence iteration over the profiled SNRs and grids (eta = 1e-2, zeta = 1e-12 in the
paper).
"""


def convergence_iteration(ber, eta=1e-2, zeta=1e-12):
    """``ber[i]`` is the BER after i + 1 iterations.  Returns the first iteration xi >= 2 (1-based)
    at which r_xi < eta, or the last profiled iteration if none."""
    for xi in range(2, len(ber) + 1):
        prev, cur = ber[xi - 2], ber[xi - 1]
        r = (prev - cur) / max(prev, zeta)
        if r < eta:
            return xi
    return len(ber)


def budget(curves, eta=1e-2, zeta=1e-12):
    """Largest convergence iteration over a set of BER-vs-iteration curves."""
    return max(convergence_iteration(c, eta, zeta) for c in curves)
