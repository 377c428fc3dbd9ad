"""Mixed precision on an uneven batch: frames of mixed shapes and antenna counts stored FP16
or BF16, FP32 arithmetic, FP64 CG scalars.  The error against the FP64 oracle is measured
twice per storage type:

- compute error: the oracle run on the *quantised* inputs with the library's own path lists
  (held to the FP32 parity bar: x_hat 1e-5, LLRs 1e-3, hard bits identical);
- storage + compute error: the oracle's full receiver on the *original* complex128 inputs
  (own estimate, own path lists), reported and held to a bound that the 16-bit rounding of
  the received samples sets (relative rounding 2^-11 for FP16, 2^-8 for BF16, amplified by
  the CG's conditioning at 10 iterations).

The table is printed (pytest -s) for the record."""

import numpy as np
import pytest
import torch

import synth
from oracle import receiver
from tests.gpu_util import TOL_LLR, TOL_X, dev, rel_l2
from tests.test_gpu_rx import _check_frames

pytestmark = pytest.mark.gpu

SHAPES = [(32, 16, 1), (64, 32, 1), (128, 64, 1), (64, 16, 2), (32, 64, 2), (128, 32, 2)]
Q, ITERS = 16, 10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()
    yield


def _quantised(b, tdt):
    yp = torch.view_as_real(torch.from_numpy(b["y_pilot_td"])).to(tdt).contiguous()
    yd = torch.view_as_real(torch.from_numpy(b["y_data_td"])).to(tdt).contiguous()
    bq = dict(b)
    bq["y_pilot_td"] = torch.view_as_complex(yp.float().contiguous()).numpy()
    bq["y_data_td"] = torch.view_as_complex(yd.float().contiguous()).numpy()
    return yp, yd, bq


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_uneven_16bit_batch_error_vs_oracle(storage):
    from paper_2604_02266_gb300 import C32_BF16, C32_F16, Batch, Paths
    code, tdt = {"fp16": (C32_F16, torch.float16), "bf16": (C32_BF16, torch.bfloat16)}[storage]
    frames, keep = [], []
    for i, (M, N, a) in enumerate(SHAPES * 2):
        b = synth.fractional_batch(1, seed=900 + i, M=M, N=N, Q=Q, n_rx=a, n_tx=a, snr_db=((10, 20, 30)[i % 3],))
        yp, yd, bq = _quantised(b, tdt)
        yp, yd = yp[0].to(dev()), yd[0].to(dev())
        bps = int(np.log2(Q))
        o = {"x": torch.zeros(a, M * N, dtype=torch.complex64, device=dev()),
             "llr": torch.zeros(a, M * N, bps, device=dev()),
             "bits": torch.zeros(a, M * N * bps // 8, dtype=torch.uint8, device=dev()),
             "pc": torch.zeros(a * a, dtype=torch.int32, device=dev()),
             "pdk": torch.zeros(a * a * 64, dtype=torch.int16, device=dev()),
             "pdl": torch.zeros(a * a * 64, dtype=torch.int16, device=dev()),
             "ph": torch.zeros(a * a * 64, dtype=torch.complex64, device=dev())}
        frames.append(dict(M=M, N=N, n_rx=a, n_tx=a, qam=Q, iters=ITERS, pilot_mode=0, guard=2, p_max=64,
                           in_dtype=code, noise_var=float(b["noise_var"][0]), theta=float(b["theta"][0]),
                           a_pilot=float(b["a_pilot"]), y_pilot=yp, y_data=yd, x_hat=o["x"], llr=o["llr"],
                           bits=o["bits"], path_count=o["pc"], path_dk=o["pdk"], path_dl=o["pdl"], path_h=o["ph"]))
        keep.append((b, bq, o, (M, N, a)))
    status = torch.full((len(frames),), -1, dtype=torch.int32, device=dev())
    Batch(frames).run(status)
    torch.cuda.synchronize()
    assert set(status.cpu().numpy().tolist()) <= {0, 6}

    rows = []
    bound = {"fp16": 5e-2, "bf16": 3e-1}[storage]
    for b, bq, o, (M, N, a) in keep:
        paths = Paths(a * a, 64, device=dev())
        paths.count.copy_(o["pc"])
        paths.dk.copy_(o["pdk"])
        paths.dl.copy_(o["pdl"])
        paths.h.copy_(o["ph"])
        out = {"paths": paths, "x_hat": o["x"][None], "llr": o["llr"][None], "bits": o["bits"][None]}
        wx, wl, mm = _check_frames(bq, out, [0], M, N, a, a, Q, ITERS, 64)  # compute error
        assert wx < TOL_X and wl < TOL_LLR and mm == 0, (storage, M, N, a, wx, wl, mm)
        ref = receiver.receive(b["y_pilot_td"][0], b["y_data_td"][0], M, N, a, a, Q, float(b["noise_var"][0]),
                               float(b["theta"][0]), ITERS, float(b["a_pilot"]), p_max=64)
        x = o["x"].cpu().numpy().reshape(-1)
        ex = rel_l2(x, ref["x_hat"])
        bits = np.concatenate([np.unpackbits(o["bits"][t].cpu().numpy(), bitorder="little") for t in range(a)])
        ber = float((bits != ref["bits"].reshape(-1)).mean())
        rows.append((M, N, a, float(b["noise_var"][0]), wx, wl, ex, ber))
    print(f"\n{storage}: M N ant noise_var | compute: x_relL2 llr_relL2 | storage+compute: x_relL2 bit_diff_rate")
    for r in rows:
        print("  %4d %3d %d %.2e | %.2e %.2e | %.2e %.2e" % r)
    print(f"  worst compute x {max(r[4] for r in rows):.2e}, worst storage+compute x {max(r[6] for r in rows):.2e}, "
          f"mean bit_diff_rate {np.mean([r[7] for r in rows]):.2e}")
    assert all(r[6] < bound for r in rows), [(r[:3], r[6]) for r in rows if r[6] >= bound]
