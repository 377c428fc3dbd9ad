"""The multi-rank bookkeeping of bench.py, on CPU with the gloo backend (world size 2): the
slowest rank's time is every rank's time, the whole-job rate counts every rank's shard, each
rank draws its own frames, and the reference arm runs on rank 0 only."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, times, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        t = bench.max_over_ranks(times[rank], ws)
        rate = bench.whole_job_rate(1024, ws, 10, t)
        import synth
        b = synth.fractional_batch(2, seed=bench.SEED + 1000 * rank, M=16, N=16, Q=4)
        np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([t, rate]))
        np.save(os.path.join(out_dir, f"y{rank}.npy"), b["y_data_td"])
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_max_time_and_whole_job_rate(tmp_path):
    ws, times = 2, [0.75, 1.25]
    mp.start_processes(_worker, args=(ws, _free_port(), times, str(tmp_path)), nprocs=ws, start_method="spawn")
    res = [np.load(tmp_path / f"r{r}.npy") for r in range(ws)]
    for t, rate in res:
        assert t == pytest.approx(max(times))  # every rank reports the slowest rank's time
        assert rate == pytest.approx(1024 * ws * 10 / max(times))  # all ranks' frames / that time
    y0, y1 = np.load(tmp_path / "y0.npy"), np.load(tmp_path / "y1.npy")
    assert y0.shape == y1.shape and not np.allclose(y0, y1)  # independent shards, no shared data


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(0.5, 1) == 0.5
    assert bench.whole_job_rate(1024, 1, 4, 2.0) == 2048.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")

    class Args:
        steps, warmup, ref_frames = 1, 3, 1

    assert bench.impl_reference(Args()) == 0
    assert capsys.readouterr().out == ""  # no work and no JSON line on other ranks
