"""Offline choice of the CG iteration count from BER (Sec. IV-C, "BER-driven iteration
selection", Eq. ber_convergence): BER-vs-iteration curves measured with the library's
receiver on frames with known transmitted bits, the convergence iteration of each curve, and
the budget over SNRs and grids."""

import numpy as np
import torch

__all__ = ["ber_curve", "convergence_iteration", "iteration_budget"]


def convergence_iteration(ber, eta=1e-2, zeta=1e-12):
    """First iteration xi >= 2 (1-based; ``ber[i]`` is the BER after i + 1 iterations) where the
    signed relative BER change (BER_{xi-1} - BER_xi) / max(BER_{xi-1}, zeta) falls below eta --
    a negligible gain or a rebound; the last iteration if none does."""
    b = np.asarray(ber, float)
    if b.size < 2:
        return int(b.size)
    r = (b[:-1] - b[1:]) / np.maximum(b[:-1], zeta)
    hit = np.nonzero(r < eta)[0]
    return int(hit[0]) + 2 if hit.size else int(b.size)


def iteration_budget(curves, eta=1e-2, zeta=1e-12):
    """The largest convergence iteration over BER curves (SNRs, grids)."""
    return max(convergence_iteration(c, eta, zeta) for c in curves)


def ber_curve(plan, y_pilot_td, y_data_td, noise_var, theta, tx_bits, max_iters, stream=None):
    """BER after 1 .. max_iters CG iterations over a batch of SISO frames (device tensors as
    for ``Plan.rx``; ``tx_bits`` the transmitted bits [n_frames, MN bps], one byte per bit),
    from the hard decisions of the fused receiver."""
    n = int(noise_var.numel())
    ref = torch.as_tensor(tx_bits, device=y_data_td.device).reshape(n, -1).to(torch.uint8)
    out = plan._rx_outputs(n, y_data_td.device, False, False, False)
    shifts = torch.arange(8, device=y_data_td.device, dtype=torch.uint8)
    bers = []
    for it in range(1, max_iters + 1):
        plan.rx(y_pilot_td, y_data_td, noise_var, theta, it, n, out=out, stream=stream)
        packed = out[3].reshape(n, -1)
        got = ((packed.unsqueeze(-1) >> shifts) & 1).reshape(n, -1)  # LSB-first bit order
        bers.append(float((got != ref).float().mean().item()))
    return bers
