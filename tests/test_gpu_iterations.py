"""The BER-vs-iteration curves of the library's receiver (the input of the iteration budget,
Eq. ber_convergence) against the FP64 oracle's on the same Veh-A frames."""

import numpy as np
import pytest
import torch

import synth
from oracle import receiver
from tests.gpu_util import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()
    yield


def test_ber_curve_vs_oracle():
    from paper_2604_02266_gb300 import Plan
    from paper_2604_02266_gb300.iterations import ber_curve, convergence_iteration
    M, N, Q, F, K = 32, 32, 4, 6, 12
    b = synth.veh_a_batch(F, 9990, M=M, N=N, Q=Q, snr_db=(6, 12))
    plan = Plan(M, N, 1, 1, Q)
    curve = ber_curve(plan, to_dev(b["y_pilot_td"]), to_dev(b["y_data_td"]), to_dev(b["noise_var"]),
                      to_dev(b["theta"]), b["bits"], K)
    ref = []
    for it in range(1, K + 1):
        wrong = 0
        for f in range(F):
            out = receiver.receive(b["y_pilot_td"][f], b["y_data_td"][f], M, N, 1, 1, Q, float(b["noise_var"][f]),
                                   float(b["theta"][f]), it, b["a_pilot"], p_max=plan.p_max)
            wrong += int((out["bits"].reshape(-1) != b["bits"][f].reshape(-1)).sum())
        ref.append(wrong / (F * M * N * 2))
    # hard decisions agree except for symbols within FP32 rounding of a decision boundary
    assert np.abs(np.array(curve) - np.array(ref)).max() <= 20 / (F * M * N * 2), (curve, ref)
    assert 2 <= convergence_iteration(curve) <= K
