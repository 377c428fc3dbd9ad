"""Benchmark of the fused Zak-OTFS receiver (SS-CGA) on the 64x32 16-QAM batch workload.

One step = the whole receiver (pilot Zak transforms, read-off and thresholding, data Zak
transform, 10 CGA iterations, max-log demapping to soft LLRs and hard bits) over a batch of 1024 frames of 64 delay x
32 Doppler bins, each with its own pilot frame, a 6-path fractional channel and an SNR drawn
from 0..30 dB, through the library's C ABI (zotfs_rx).  Inputs are synthetic (synth/) and
resident in HBM; 8 copies of the batch are rotated so the timed inputs exceed the 129 MB L2.

Reported (one JSON line on rank 0):
  value         frames/s over all ranks (device time, CUDA events)
  e2e           the same metric with pinned host inputs copied in and the LLRs, hard bits
                and statuses copied back inside the timed region
  plain_form    the plain single-frame FP32 form (one launch per stage) on the same frames
  roofline      the fused kernel against the FP32 FMA peak (algorithmic flops per launch)
  cpu_baseline  the FP64 oracle on the host cores, on a bounded sample of the same frames
  clocks        nvidia-smi samples taken during the timed region

`--impl reference` times the oracle alone (the reference arm of this workload).
"""

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, Q, FRAMES, ITERS = 64, 32, 16, 1024, 10
WORKLOAD = "SISO batch of 1024 frames, M=64, N=32, 16-QAM, separate pilot frame per frame, 6-path fractional " \
           "channel (delay U[0,4], Doppler U[-3,3] bins, exponential PDP), SNR 0..30 dB, threshold 3 sigma, " \
           "p_max 64, 10 CG iterations, complex FP32"
SEED = 2604


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device=None):
    """The maximum of a per-rank host number over all ranks (all_reduce MAX; the slowest
    rank's time defines the whole job's), or x itself on one rank."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, ws, steps, seconds):
    """Units per second of the whole job: every rank processes its own shard of
    units_per_rank_step units per step (weak scaling), timed by the slowest rank."""
    return units_per_rank_step * ws * steps / seconds


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# ------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling (200 ms) in the background during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- work model

PATH_HIST_EDGES = [0, 8, 16, 24, 32, 40, 48, 56, 64, 65]


def flops_per_frame(P, iters=ITERS, M=M, N=N, Q=Q):
    """Algorithmic flops of one frame: CGA (two SS applies of 8 flops per tap-element plus
    24 flops of vector updates per element and iteration, one adjoint for b), the two Zak
    transforms (5 MN log2 N each) and demapping (~4 flops per constellation level per axis)."""
    MN = M * N
    cg = MN * (iters * (16 * P + 24) + 8 * P + 4)
    dzt = 2 * 5 * MN * np.log2(N)
    demap = MN * 2 * 4 * int(np.sqrt(Q))
    return cg + dzt + demap


def hbm_bytes_per_frame(M=M, N=N, Q=Q, llr=True):
    """Algorithmic HBM bytes of one frame in the fused kernel: pilot + data TD frames in
    (complex64), float32 LLRs (when written), hard bits and the status word out (x_hat is
    not written in the timed step)."""
    MN = M * N
    bps = int(np.log2(Q))
    return 2 * MN * 8 + (MN * bps * 4 if llr else 0) + MN * bps // 8 + 4


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("common.cuh", "frame_engine.cuh", "frame_kernel.cuh", "frame_variant.cu"):
        with open(os.path.join(ROOT, "paper_2604_02266_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the fused kernel from the committed ncu summary, if it was
    taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "frame_kernel_64x32_batch1024.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    if vals.get("llr_written") != "yes":  # the timed step stores LLRs; a bits-only capture does not count
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ------------------------------------------------------------------------ oracle arm

def run_oracle(batch, frames):
    """Full FP64 oracle receiver on the given frame indices; returns seconds."""
    from oracle import receiver
    t0 = time.perf_counter()
    for f in frames:
        receiver.receive(batch["y_pilot_td"][f].astype(complex), batch["y_data_td"][f].astype(complex), M, N, 1, 1, Q,
                         float(batch["noise_var"][f]), float(batch["theta"][f]), ITERS, batch["a_pilot"], p_max=64)
    return time.perf_counter() - t0


def _oracle_chunk(yp, yd, nv, th, a_pilot):
    """Worker: the FP64 oracle receiver on a chunk of frames (returns the frame count)."""
    from oracle import receiver
    for f in range(len(yd)):
        receiver.receive(yp[f], yd[f], M, N, 1, 1, Q, float(nv[f]), float(th[f]), ITERS, a_pilot, p_max=64)
    return len(yd)


class OraclePool:
    """The FP64 oracle over frames on the host's cores: a pool of spawned worker processes,
    one frame chunk each, single-threaded BLAS per worker.  Started before timing."""

    def __init__(self, workers):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.workers = workers
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            self.ex = cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"))
            list(self.ex.map(abs, range(workers)))  # start every worker
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def run(self, batch, frames):
        """Seconds to run the oracle on `frames` (indices into batch) across the pool."""
        chunks = np.array_split(np.asarray(frames), self.workers)
        args = [(batch["y_pilot_td"][c].astype(complex), batch["y_data_td"][c].astype(complex),
                 batch["noise_var"][c], batch["theta"][c], batch["a_pilot"]) for c in chunks if len(c)]
        t0 = time.perf_counter()
        done = sum(f.result() for f in [self.ex.submit(_oracle_chunk, *a) for a in args])
        secs = time.perf_counter() - t0
        assert done == len(frames)
        return secs

    def close(self):
        self.ex.shutdown()


def host_cores():
    return max(1, min(16, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()))


def oracle_sample(n_frames, sample):
    idx = np.linspace(0, n_frames - 1, sample).astype(int)
    return idx


def impl_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import synth
    batch = synth.fractional_batch(FRAMES, seed=SEED, M=M, N=N, Q=Q)
    cores = host_cores()
    # frames per step: ref_frames per core, fewer for long runs so that the whole timed run
    # stays near a minute of the pool's time (one frame is ~0.1 s of one core)
    sample = max(1, min(args.ref_frames * cores, (60 * cores) // max(1, args.steps)))
    idx = oracle_sample(FRAMES, sample)
    pool = OraclePool(cores)
    try:
        for _ in range(args.warmup):
            pool.run(batch, idx[:min(cores, len(idx))])
        times = [pool.run(batch, idx) for _ in range(args.steps)]
    finally:
        pool.close()
    fps = sample * args.steps / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames_per_step": sample},
        "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} of the {FRAMES} frames per step (evenly spaced), full FP64 receiver, "
                                   f"{cores} worker processes"},
        "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


METRIC = "equalized Zak-OTFS frames/s + p50/p99 latency, 64x32 16-QAM, vs plain form"


# ------------------------------------------------------------------------- GPU arm

def impl_zotfs(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as ge
    if rank == 0:
        ge.build()
    if ws > 1:
        torch.distributed.barrier()
    ge.build()
    import synth
    from paper_2604_02266_gb300 import Plan, launch_count

    batch = synth.fractional_batch(FRAMES, seed=SEED + 1000 * rank, M=M, N=N, Q=Q)
    plan = Plan(M, N, 1, 1, Q)
    if args.threads:
        plan.set_tuning(threads_per_frame=args.threads, fft_radix=args.radix, ctas_per_sm=args.ctas)
    elif args.radix:
        plan.set_tuning(fft_radix=args.radix, ctas_per_sm=args.ctas)
    copies = 8  # 8 x 32 MB of TD frames > 129 MB L2
    yp = [torch.from_numpy(batch["y_pilot_td"]).to(dev) for _ in range(copies)]
    yd = [torch.from_numpy(batch["y_data_td"]).to(dev) for _ in range(copies)]
    nv = torch.from_numpy(batch["noise_var"]).to(dev)
    th = torch.from_numpy(batch["theta"]).to(dev)
    outs = plan._rx_outputs(FRAMES, dev, False, False, True)  # soft output: LLRs + hard bits
    outs_hard = plan._rx_outputs(FRAMES, dev, False, False, False)
    stream = torch.cuda.current_stream()

    # path counts of this batch (same data every step) for the flop count
    probe = plan.rx(yp[0], yd[0], nv, th, ITERS, FRAMES, want_paths=True)
    P = probe["paths"].count.cpu().numpy()
    status = probe["status"].cpu().numpy()
    total_flops = float(sum(flops_per_frame(int(p)) for p in P))
    # decoding quality of the batch (untimed): BER of the hard bits against the transmitted
    # bits, with the benchmark's p_max = 64 and with p_max = 256 (no list of this batch is cut)
    errs64 = bit_errors(probe["bits"].cpu().numpy(), batch["bits"], FRAMES)
    wide = Plan(M, N, 1, 1, Q, p_max=256)
    probe256 = wide.rx(yp[0], yd[0], nv, th, ITERS, FRAMES, want_paths=True)
    errs256 = bit_errors(probe256["bits"].cpu().numpy(), batch["bits"], FRAMES)
    P256 = probe256["paths"].count.cpu().numpy()
    nbits = FRAMES * M * N * int(np.log2(Q))
    quality = {"ber_p_max_64": float(errs64.sum()) / nbits, "ber_p_max_256": float(errs256.sum()) / nbits,
               "paths_p_max_256": {"mean": float(P256.mean()), "max": int(P256.max())},
               "ber_by_snr_db": {int(snr): {"p_max_64": float(errs64[batch["snr_db"] == snr].sum()) /
                                            max(1, int((batch["snr_db"] == snr).sum()) * M * N * int(np.log2(Q))),
                                            "p_max_256": float(errs256[batch["snr_db"] == snr].sum()) /
                                            max(1, int((batch["snr_db"] == snr).sum()) * M * N * int(np.log2(Q)))}
                                 for snr in (0, 10, 20, 30)}}
    del wide, probe256

    def step(i):
        plan.rx(yp[i % copies], yd[i % copies], nv, th, ITERS, FRAMES, out=outs)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches = 0
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t0 = time.perf_counter()
        for i in range(args.steps):
            ev[i][0].record(stream)
            step(i)
            launches += launch_count()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    step_ms = np.array([a.elapsed_time(b) for a, b in ev])
    dev_s = max_over_ranks(float(step_ms.sum()) / 1e3, ws, dev)
    value = whole_job_rate(FRAMES, ws, args.steps, dev_s)

    # ---- secondary: the same steps with hard bits only (no LLR store)
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(args.warmup):
        plan.rx(yp[i % copies], yd[i % copies], nv, th, ITERS, FRAMES, out=outs_hard)
    torch.cuda.synchronize()
    h0.record(stream)
    for i in range(args.steps):
        plan.rx(yp[i % copies], yd[i % copies], nv, th, ITERS, FRAMES, out=outs_hard)
    h1.record(stream)
    torch.cuda.synchronize()
    hard_s = max_over_ranks(h0.elapsed_time(h1) / 1e3, ws, dev)
    hard_only = {"value": whole_job_rate(FRAMES, ws, args.steps, hard_s), "unit": "frames/s",
                 "ms_per_step": 1e3 * hard_s / args.steps, "note": "hard bits and statuses only, no LLR store"}

    # ---- end to end: pinned host frames in, hard bits out, every step.  Two streams with their
    # own device buffers alternate, so one step's copies overlap the other's receiver (the way
    # a receive chain streams frames); every step still copies its own inputs and results.
    hp = torch.from_numpy(batch["y_pilot_td"]).pin_memory()
    hd = torch.from_numpy(batch["y_data_td"]).pin_memory()
    lanes = []
    for _ in range(2):
        o = plan._rx_outputs(FRAMES, dev, False, False, True)
        lanes.append({"s": torch.cuda.Stream(device=dev), "dp": torch.empty_like(yp[0]), "dd": torch.empty_like(yd[0]),
                      "out": o, "hl": torch.empty_like(o[2], device="cpu").pin_memory(),
                      "hb": torch.empty_like(o[3], device="cpu").pin_memory(),
                      "hs": torch.empty_like(o[4], device="cpu").pin_memory()})

    def e2e_step(i):
        ln = lanes[i % 2]
        with torch.cuda.stream(ln["s"]):
            ln["dp"].copy_(hp, non_blocking=True)
            ln["dd"].copy_(hd, non_blocking=True)
            plan.rx(ln["dp"], ln["dd"], nv, th, ITERS, FRAMES, out=ln["out"], stream=ln["s"])
            ln["hl"].copy_(ln["out"][2], non_blocking=True)
            ln["hb"].copy_(ln["out"][3], non_blocking=True)
            ln["hs"].copy_(ln["out"][4], non_blocking=True)

    for ln in lanes:
        ln["s"].wait_stream(stream)
    for i in range(max(2, args.warmup)):
        e2e_step(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for ln in lanes:
        ln["s"].wait_stream(stream)
    for i in range(args.steps):
        e2e_step(i)
    for ln in lanes:
        stream.wait_stream(ln["s"])
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, ws, dev)
    hl0, hb0, hs0 = lanes[0]["hl"], lanes[0]["hb"], lanes[0]["hs"]

    # ---- the same device-resident steps on the two streams (consecutive batches overlap)
    def dev_step(i):
        ln = lanes[i % 2]
        with torch.cuda.stream(ln["s"]):
            plan.rx(yp[i % copies], yd[i % copies], nv, th, ITERS, FRAMES, out=ln["out"], stream=ln["s"])

    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    p0.record(stream)
    for ln in lanes:
        ln["s"].wait_stream(stream)
    for i in range(args.steps):
        dev_step(i)
    for ln in lanes:
        stream.wait_stream(ln["s"])
    p1.record(stream)
    torch.cuda.synchronize()
    pipe_s = max_over_ranks(p0.elapsed_time(p1) / 1e3, ws, dev)
    pipelined = {"value": whole_job_rate(FRAMES, ws, args.steps, pipe_s), "unit": "frames/s",
                 "ms_per_step": 1e3 * pipe_s / args.steps,
                 "note": "inputs resident in HBM; consecutive batches on two streams overlap"}
    e2e = {"value": whole_job_rate(FRAMES, ws, args.steps, e2e_s), "unit": "frames/s",
           "h2d_bytes_per_step": int(hp.numel() * hp.element_size() + hd.numel() * hd.element_size()),
           "d2h_bytes_per_step": int(hl0.numel() * 4 + hb0.numel() + hs0.numel() * 4),
           "pipelined": "2 streams: step i+1's host-device copies overlap step i's receiver"}

    # ---- plain form: one frame at a time, one launch per stage
    n_plain = args.plain_frames
    pout = plan._rx_outputs(1, dev, False, False, True)
    lat = []
    for f in range(n_plain + 2):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        plan.rx(yp[0][f:f + 1], yd[0][f:f + 1], nv[f:f + 1], th[f:f + 1], ITERS, 1, out=pout, plain=True)
        b.record(stream)
        b.synchronize()
        if f >= 2:  # first two are warm-up
            lat.append(a.elapsed_time(b))
    lat = np.array(lat) if lat else np.array([np.nan])
    plain_fps = 1e3 * len(lat) / lat.sum() if n_plain > 0 else float("nan")

    # ---- roofline of the fused kernel (one launch per step)
    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = n_sm * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s
    kern_s = float(np.mean(step_ms)) / 1e3
    achieved = total_flops / kern_s / 1e12
    traffic = profiled_traffic()
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": traffic,
                "peak_source": f"{n_sm} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz (max SM clock, "
                               "MEASURED_PEAKS.json)",
                "hbm_GBps": hbm_bytes_per_frame() * FRAMES / kern_s / 1e9,
                "hbm_peak_GBps": float(peaks.get("hbm_gbs", 6800.0))}

    # ---- FP64 oracle on the host cores (bounded sample)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cores = host_cores()
        idx = oracle_sample(FRAMES, args.oracle_frames * cores)
        pool = OraclePool(cores)
        try:
            pool.run(batch, idx[:cores])  # warm-up
            secs = pool.run(batch, idx)
        finally:
            pool.close()
        one = oracle_sample(FRAMES, args.oracle_frames)
        secs1 = run_oracle(batch, one)
        cpu = {"value": len(idx) / secs, "unit": "frames/s", "cores": cores, "kind": "oracle",
               "sample": f"{len(idx)} of the {FRAMES} frames (evenly spaced), full FP64 receiver, {cores} worker "
                         f"processes (one frame chunk each); single core on {len(one)} frames: "
                         f"{len(one) / secs1:.2f} frames/s",
               "single_core_value": len(one) / secs1}

    if rank == 0:
        bps = int(np.log2(Q))
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_per_step_per_gpu": FRAMES, "M": M, "N": N, "qam": Q,
                       "iters": ITERS, "p_max": 64, "l2": "8 rotating input copies (256 MB) > L2",
                       "threads_per_frame": plan.tuning()["threads_per_frame"] or "library default",
                       "fft_radix": plan.tuning()["fft_radix"]},
            "mbit_s": value * M * N * bps / 1e6,
            "latency_ms": {"batch_p50": float(np.percentile(step_ms, 50)),
                           "batch_p99": float(np.percentile(step_ms, 99))},
            "plain_form": {"value": plain_fps, "unit": "frames/s", "frames": len(lat),
                           "frame_latency_p50_ms": float(np.percentile(lat, 50)),
                           "frame_latency_p99_ms": float(np.percentile(lat, 99))},
            "speedup_vs_plain": value / plain_fps / ws,
            "paths": {"mean": float(P.mean()), "min": int(P.min()), "max": int(P.max()),
                      "truncated_frames": int((status == 6).sum()),
                      # P_est histogram: [0, 8), [8, 16), ..., [56, 64), and exactly 64 (= p_max)
                      "hist_edges": PATH_HIST_EDGES,
                      "hist_counts": np.histogram(P, bins=PATH_HIST_EDGES)[0].tolist()},
            "decoding": quality,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "pipelined": pipelined,
            "hard_output_only": hard_only,
            "gpu_launches": launches,
            "clocks": clocks.summary(),
            "wall_s_timed": wall,
        }
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# ----------------------------------------------------------------- serving workload

SERVE_M, SERVE_N, SERVE_ANT, SERVE_Q = (32, 64, 128, 256), (16, 32, 64), (1, 2, 4), (4, 16, 64)
SERVE_WORKLOAD = ("serving loop: Poisson arrivals, M in {32,64,128,256}, N in {16,32,64}, 1x1/2x2/4x4, QAM in "
                  "{4,16,64}, all uniform, 8-path fractional channels, SNR 0..30 dB, 10 CG iterations, "
                  "0.5 ms deadline from arrival, outputs kept in a device arena until released")
DEADLINE_MS = 0.5
# latency classes of the serving report: M N n_rx n_tx in (lo, hi]
SERVE_WORK_BUCKETS = ((0, 2048), (2048, 8192), (8192, 32768), (32768, 131072), (131072, 1 << 30))


def impl_serve(args):
    """Continuous-batching server under Poisson load: one run per offered rate, reporting the
    completed frames/s, Mbit/s and the arrival-to-completion latency percentiles against the
    slot deadline.  Requests draw their frames from a device-resident pool of synthetic
    frames per (M, N, antennas, QAM) class."""
    import torch
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as ge
    ge.build()
    import synth
    from paper_2604_02266_gb300 import Server

    if args.serve_mix == "c2":  # the headline frame shape only: 64x32 SISO 16-QAM, 6 paths
        classes, n_paths = [(M, N, 1, Q)], 6
    else:
        classes, n_paths = [(m, n, a, q) for m in SERVE_M for n in SERVE_N for a in SERVE_ANT for q in SERVE_Q], 8
    pool = {}
    for ci, (m, n, a, q) in enumerate(classes):
        b = synth.fractional_batch(args.pool, seed=SEED + 7919 * ci, M=m, N=n, Q=q, n_rx=a, n_tx=a, n_paths=n_paths)
        pool[(m, n, a, q)] = (torch.from_numpy(b["y_pilot_td"]).to(dev), torch.from_numpy(b["y_data_td"]).to(dev),
                              b["noise_var"].astype(float), b["theta"].astype(float))
    light = args.light_work if args.serve_mix == "c5" else 0
    srv = Server(p_max=64, max_wave_frames=args.wave_frames, waves_in_flight=args.waves, keep_llr=False,
                 arena_bytes=4 << 30, max_M=256, max_N=64, max_ant=4, light_work=light)

    def make(n, g, tag0):
        reqs, meta = [], []
        for i in range(n):
            m, nn, a, q = classes[int(g.integers(0, len(classes)))]
            j = int(g.integers(0, args.pool))
            yp, yd, nv, th = pool[(m, nn, a, q)]
            reqs.append(Server.request(tag0 + i, yp[j], yd[j], m, nn, a, a, q, ITERS, nv[j], th[j]))
            meta.append((m, nn, a, q))
        return reqs, meta

    def drain(n, timeout_s):
        got = {}
        t0 = time.time()
        while len(got) < n:
            cs = srv.poll()
            for c in cs:
                got[c.tag] = (c.status, c.arrival_ns, c.admit_ns, c.done_ns)
                srv.release(c.tag)
            if time.time() - t0 > timeout_s:
                raise RuntimeError(f"serving run stalled: {len(got)} of {n} frames completed")
            if not cs:
                time.sleep(50e-6)
        return got

    g = np.random.default_rng(SEED)
    try:
        # warm-up: every class once (kernel attributes, first launches)
        warm = [Server.request(10**9 + i, pool[c][0][0], pool[c][1][0], *c[:3], c[2], c[3], ITERS,
                               pool[c][2][0], pool[c][3][0]) for i, c in enumerate(classes)]
        srv.submit(warm)
        drain(len(warm), 300)
        runs = []
        tag0 = 0
        for rate in args.rates:
            n = max(1, int(rate * args.duration))
            reqs, meta = make(n, g, tag0)
            arrivals = np.cumsum(g.exponential(1.0 / rate, size=n))
            th = threading.Thread(target=srv.replay, args=(reqs, arrivals))
            th.start()
            got = drain(n, 600)
            th.join()
            rows = [got[tag0 + i] for i in range(n)]
            tag0 += n
            st = np.array([r[0] for r in rows])
            arr = np.array([r[1] for r in rows], dtype=np.int64)
            adm = np.array([r[2] for r in rows], dtype=np.int64)
            done = np.array([r[3] for r in rows], dtype=np.int64)
            lat = (done - arr) * 1e-6
            wall = (done.max() - arr.min()) * 1e-9
            bits = sum(a * m * nn * int(np.log2(q)) for (m, nn, a, q) in meta)
            def lat_stats(sel):
                return {"frames": int(sel.sum()), "p50_ms": float(np.percentile(lat[sel], 50)),
                        "p99_ms": float(np.percentile(lat[sel], 99)),
                        "deadline_met": float((lat[sel] <= DEADLINE_MS).mean())}
            by_ant = {}
            for a in SERVE_ANT:
                sel = np.array([mt[2] == a for mt in meta])
                if sel.any():
                    by_ant[f"{a}x{a}"] = lat_stats(sel)
            # per class: work buckets of M N n_rx n_tx, and every SISO shape on its own
            work = np.array([m * nn * a * a for (m, nn, a, q) in meta])
            by_work = {}
            for lo, hi in SERVE_WORK_BUCKETS:
                sel = (work > lo) & (work <= hi)
                if sel.any():
                    by_work[f"({lo},{hi}]"] = lat_stats(sel)
            by_siso_shape = {}
            for (m, nn) in sorted({(mt[0], mt[1]) for mt in meta if mt[2] == 1}):
                sel = np.array([mt[0] == m and mt[1] == nn and mt[2] == 1 for mt in meta])
                by_siso_shape[f"{m}x{nn}"] = lat_stats(sel)
            runs.append({"offered_frames_s": rate, "frames": n, "completed_frames_s": n / wall,
                         "mbit_s": bits / wall / 1e6, "p50_ms": float(np.percentile(lat, 50)),
                         "p99_ms": float(np.percentile(lat, 99)), "deadline_met": float((lat <= DEADLINE_MS).mean()),
                         "queue_p99_ms": float(np.percentile((adm - arr) * 1e-6, 99)),
                         "status_ok_or_truncated": float(np.isin(st, (0, 6)).mean()), "by_antennas": by_ant,
                         "by_work": by_work, "by_siso_shape": by_siso_shape})
        stats = srv.stats()
    finally:
        srv.close()
    head = runs[0]
    workload = SERVE_WORKLOAD if args.serve_mix == "c5" else (
        "serving loop: Poisson arrivals of 64x32 SISO 16-QAM frames, separate pilot frame, 6-path fractional "
        "channel, SNR 0..30 dB, 10 CG iterations, 0.5 ms deadline from arrival")
    line = {"metric": "served Zak-OTFS frames/s + p50/p99 latency vs 0.5 ms deadline", "value": head["completed_frames_s"],
            "unit": "frames/s", "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "mix": args.serve_mix, "duration_s": args.duration,
                       "pool_frames_per_class": args.pool, "max_wave_frames": args.wave_frames,
                       "waves_in_flight": args.waves, "light_work": light},
            "runs": runs, "server_stats": stats}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------- mixed-precision uneven batch

MIXED_M, MIXED_N = (32, 64, 128), (16, 32, 64)
MIXED_FRAMES = 8192


def impl_mixed(args):
    """8192 frames of uneven shapes (M in {32,64,128} x N in {16,32,64}, SISO or 2x2 with
    probability 1/2), received frames stored FP16 or BF16, one uneven batch per storage type:
    autotuned launch shapes, and the whole batch replayed as one CUDA graph per step."""
    import torch
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as ge
    ge.build()
    import synth
    from paper_2604_02266_gb300 import C32_BF16, C32_F16, Batch, autotune, save_tuning

    g = np.random.default_rng(SEED)
    cls = [(int(g.choice(MIXED_M)), int(g.choice(MIXED_N)), 1 if g.random() < 0.5 else 2) for _ in range(MIXED_FRAMES)]
    groups = {}
    for i, c in enumerate(cls):
        groups.setdefault(c, []).append(i)
    data = {}
    for gi, (c, ids) in enumerate(sorted(groups.items())):
        m, n, a = c
        data[c] = synth.fractional_batch(len(ids), seed=SEED + 104729 * gi, M=m, N=n, Q=Q, n_rx=a, n_tx=a)
    out = {"storage": {}}
    for name, code, tdt in (("fp16", C32_F16, torch.float16), ("bf16", C32_BF16, torch.bfloat16)):
        frames, keep = [], []
        for c, ids in sorted(groups.items()):
            m, n, a = c
            b = data[c]
            yp = torch.view_as_real(torch.from_numpy(b["y_pilot_td"])).to(tdt).to(dev).contiguous()
            yd = torch.view_as_real(torch.from_numpy(b["y_data_td"])).to(tdt).to(dev).contiguous()
            bits = torch.zeros(len(ids), a, m * n * int(np.log2(Q)) // 8, dtype=torch.uint8, device=dev)
            keep += [yp, yd, bits]
            for j in range(len(ids)):
                frames.append(dict(M=m, N=n, n_rx=a, n_tx=a, qam=Q, iters=ITERS, pilot_mode=0, guard=2, p_max=64,
                                   in_dtype=code, noise_var=float(b["noise_var"][j]), theta=float(b["theta"][j]),
                                   a_pilot=float(b["a_pilot"]), y_pilot=yp[j], y_data=yd[j], bits=bits[j]))
        status = torch.zeros(len(frames), dtype=torch.int32, device=dev)
        tuning = autotune(frames, warmup=1, reps=3, max_frames=args.tune_frames)
        if args.tuning_file:
            save_tuning(args.tuning_file.replace("{dtype}", name), tuning, torch.cuda.get_device_name(dev))
        entries = [((t["M"], t["N"], t["n_rx"], t["n_tx"]), t) for t in tuning]

        def timed(run, steps):
            for _ in range(args.warmup):
                run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                run()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / steps

        plain_batch = Batch(frames)
        ms_default = timed(lambda: plain_batch.run(status), args.mixed_steps)
        del plain_batch
        tuned = Batch(frames, tuning=entries)
        ms_eager = timed(lambda: tuned.run(status), args.mixed_steps)
        graph = tuned.capture(status)
        ms_graph = timed(graph.launch, args.mixed_steps)
        st = status.cpu().numpy()
        # consecutive batches overlapped: a second batch of the same frames with its own outputs
        # and status, its graph replayed on a second stream, alternating with the first
        frames2 = [dict(f, bits=torch.empty_like(f["bits"])) for f in frames]
        status2 = torch.zeros_like(status)
        tuned2 = Batch(frames2, tuning=entries)
        graph2 = tuned2.capture(status2)
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

        def pair():
            with torch.cuda.stream(s1):
                graph.launch(stream=s1)
            with torch.cuda.stream(s2):
                graph2.launch(stream=s2)

        for _ in range(args.warmup):
            pair()
        torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record()
        s1.wait_stream(torch.cuda.current_stream())
        s2.wait_stream(torch.cuda.current_stream())
        for _ in range(args.mixed_steps // 2):
            pair()
        torch.cuda.current_stream().wait_stream(s1)
        torch.cuda.current_stream().wait_stream(s2)
        t_end.record()
        torch.cuda.synchronize()
        ms_pipelined = t_start.elapsed_time(t_end) / (2 * (args.mixed_steps // 2))
        graph.close()
        graph2.close()
        del tuned2, frames2
        bits_per_step = sum(len(ids) * a * m * n * int(np.log2(Q)) for (m, n, a), ids in groups.items())
        out["storage"][name] = {
            "frames_s": len(frames) / ms_graph * 1e3, "mbit_s": bits_per_step / ms_graph / 1e3,
            "frames_s_pipelined": len(frames) / ms_pipelined * 1e3, "ms_per_step_pipelined": ms_pipelined,
            "ms_per_step_graph": ms_graph, "ms_per_step_tuned_eager": ms_eager, "ms_per_step_default_eager": ms_default,
            "status_ok_or_truncated": float(np.isin(st, (0, 6)).mean()),
            "tuning": [{k: t[k] for k in ("M", "N", "n_rx", "n_tx", "threads_per_frame", "fft_radix", "ctas_per_sm", "cluster",
                                          "frames_per_cta", "sm_ms_per_frame", "ms_best", "ms_default")} for t in tuning]}
        del tuned, frames, keep
    head = out["storage"]["fp16"]
    line = {"metric": "equalized Zak-OTFS frames/s, uneven mixed-precision batch", "value": head["frames_s"],
            "unit": "frames/s", "n_gpus": 1, "steps": args.mixed_steps, "warmup": args.warmup,
            "ms_per_step": head["ms_per_step_graph"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 compute, fp16/bf16 storage", "data": "synthetic",
            "config": {"workload": "8192 frames, M in {32,64,128} x N in {16,32,64} uniform, SISO or 2x2 with "
                                   "probability 1/2, 16-QAM, 6-path fractional channels, SNR 0..30 dB, 10 CG "
                                   "iterations, frames stored FP16 / BF16, autotuned launch shapes, one CUDA graph "
                                   "per step", "frames": MIXED_FRAMES, "classes": len(groups)},
            **out}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------------- MIMO workload

def impl_mimo(args):
    """256 frames of a 4x4 stack at 128x64, 64-QAM (16 path lists per frame, 32768 stacked
    unknowns per CG): the large-frame kernels, whose vectors live in global scratch slots.  The
    headline runs the default tuning (the clustered kernel, 2 CTAs per frame at this load); the
    one-CTA kernel and the 4-CTA cluster are timed beside it, each also one frame per call
    (where the default takes 4 CTAs per frame)."""
    import torch
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as ge
    ge.build()
    import synth
    from paper_2604_02266_gb300 import Plan, launch_count
    Mm, Nm, Qm, A, F = 128, 64, 64, 4, 256
    b = synth.fractional_batch(F, seed=SEED + 3, M=Mm, N=Nm, Q=Qm, n_rx=A, n_tx=A)
    yp, yd = torch.from_numpy(b["y_pilot_td"]).to(dev), torch.from_numpy(b["y_data_td"]).to(dev)
    nv, th = torch.from_numpy(b["noise_var"]).to(dev), torch.from_numpy(b["theta"]).to(dev)
    steps = args.mimo_steps
    variants = {}
    head = None
    for name, cl, ctas in (("default", 0, 0), ("one_cta", 1, 0), ("cluster2", 2, 0), ("cluster4", 4, 0)):
        plan = Plan(Mm, Nm, A, A, Qm)
        plan.set_tuning(cluster=cl, ctas_per_sm=ctas)
        outs = plan._rx_outputs(F, dev, True, False, False)
        for _ in range(args.warmup):
            plan.rx(yp, yd, nv, th, ITERS, F, out=outs)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.rx(yp, yd, nv, th, ITERS, F, out=outs)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        launches = launch_count() * steps  # the library counts the launches of its last call
        one = plan._rx_outputs(1, dev, False, False, False)
        ts = []
        for f in range(12):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            plan.rx(yp[f:f + 1], yd[f:f + 1], nv[f:f + 1], th[f:f + 1], ITERS, 1, out=one)
            s1.record()
            s1.synchronize()
            ts.append(s0.elapsed_time(s1))
        variants[name] = {"ms_per_step": ms, "frames_s": F / ms * 1e3, "one_frame_p50_ms": float(np.median(ts[2:]))}
        if head is None:
            P = outs[0].count.cpu().numpy()
            st = outs[4].cpu().numpy()
            head = (ms, launches, P, st)
        del plan, outs, one
    ms, launches, P, st = head
    line = {"metric": "equalized Zak-OTFS frames/s, 4x4 MIMO 128x64 64-QAM", "value": F / ms * 1e3, "unit": "frames/s",
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "256 frames, 4x4 antennas, M=128, N=64, 64-QAM, 16 independent 6-path fractional "
                                   "channels per frame, separate pilot frame per tx antenna, SNR 0..30 dB, 10 CG "
                                   "iterations over 32768 stacked unknowns, complex FP32 with FP64 CG scalars"},
            "mbit_s": F * A * Mm * Nm * 6 / ms / 1e3, "paths_per_list": {"mean": float(P.mean()), "max": int(P.max())},
            "status_ok_or_truncated": float(np.isin(st, (0, 6)).mean()), "gpu_launches": launches,
            "variants": variants}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------- pilot-reuse workload

def impl_packets(args):
    """Pilot reuse: packets of one pilot frame and D data frames through the same channel (the
    headline 64x32 16-QAM shape); a step is the read-off of the packets' pilots (zotfs_estimate)
    and the fused data-frame receiver over all data frames with their packet's lists
    (zotfs_rx_lists)."""
    import torch
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as ge
    ge.build()
    import synth
    from paper_2604_02266_gb300 import Plan
    D = args.packet_data
    P = FRAMES // D
    b = synth.packet_batch(P, D, SEED + 77, M=M, N=N, Q=Q)
    plan = Plan(M, N, 1, 1, Q)
    yp, yd = torch.from_numpy(b["y_pilot_td"]).to(dev), torch.from_numpy(b["y_data_td"]).to(dev)
    nv, th = torch.from_numpy(b["noise_var"]).to(dev), torch.from_numpy(b["theta"]).to(dev)
    ids = torch.from_numpy(b["path_ids"]).to(dev)
    paths = plan.new_paths(P)
    F = P * D
    _, x, L, B, st = plan._rx_outputs(F, dev, False, False, False)

    def step():
        plan.estimate(yp, th, P, paths=paths)
        plan.rx_lists(yd, paths, nv, ITERS, F, path_ids=ids, n_sets=P, out=(x, L, B, st))

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    steps = args.steps or 200
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    s_ = st.cpu().numpy()
    # one packet per call (pilot read-off + its D data frames), device time against the 2T
    # deadline of the paper's real-time setting (T = N / delta_f = 1.07 ms at 30 kHz)
    one_paths = plan.new_paths(1)
    _, x1, L1, B1, st1 = plan._rx_outputs(D, dev, False, False, False)
    ids1 = torch.zeros(D, dtype=torch.int32, device=dev)
    ts = []
    for i in range(min(P, 64) + 3):
        pk = i % P
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        plan.estimate(yp[pk:pk + 1], th[pk:pk + 1], 1, paths=one_paths)
        plan.rx_lists(yd[pk * D:(pk + 1) * D], one_paths, nv[pk * D:(pk + 1) * D], ITERS, D, path_ids=ids1, n_sets=1,
                      out=(x1, L1, B1, st1))
        t1.record()
        t1.synchronize()
        if i >= 3:
            ts.append(t0.elapsed_time(t1))
    ts = np.array(ts)
    from paper_2604_02266_gb300 import numerology
    two_t_ms = numerology.packet_deadline(N, 30e3) * 1e3
    packet_ms = numerology.packet_deadline(N, 30e3, D) * 1e3
    line = {"metric": "equalized Zak-OTFS data frames/s with pilot reuse, 64x32 16-QAM", "value": F / ms * 1e3,
            "unit": "frames/s", "n_gpus": 1, "steps": steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{P} packets x (1 pilot frame + {D} data frames through the same 6-path fractional "
                                   "channel), M=64, N=32, 16-QAM, SNR 0..30 dB per packet, 10 CG iterations; a step "
                                   "is the pilots' read-off + the data frames' receiver", "packets": P,
                       "data_per_pilot": D},
            "mbit_s": F * M * N * 4 / ms / 1e3, "status_ok": float((s_ == 0).mean()), "gpu_launches_per_step": 3,
            "one_packet_per_call": {"p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
                                    "deadline_2T_ms": two_t_ms, "within_2T": float((ts <= two_t_ms).mean()),
                                    "packet_duration_ms": packet_ms, "packets": int(ts.size)},
            "data_per_pilot_at_100Hz": numerology.data_frames_per_pilot(100.0, N, 30e3)}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------- iteration-budget workload

def impl_iterations(args):
    """The BER-driven iteration budget (Sec. IV-C, Eq. ber_convergence) on Veh-A frames: BER
    after 1 .. 30 CG iterations of the fused receiver per (grid, SNR), the convergence
    iteration and the lowest-BER iteration of each curve, and the budget over all of them."""
    import torch
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as ge
    ge.build()
    import synth
    from paper_2604_02266_gb300 import Plan
    from paper_2604_02266_gb300.iterations import ber_curve, convergence_iteration, iteration_budget
    rows, curves = [], []
    t0 = time.time()
    for (m, n) in ((128, 32), (32, 32)):
        plan = Plan(m, n, 1, 1, 16)
        for snr in range(0, 31, 5):
            b = synth.veh_a_batch(args.iter_frames, SEED + 31 * m + snr, M=m, N=n, Q=16, snr_db=(snr,))
            c = ber_curve(plan, torch.from_numpy(b["y_pilot_td"]).to(dev), torch.from_numpy(b["y_data_td"]).to(dev),
                          torch.from_numpy(b["noise_var"]).to(dev), torch.from_numpy(b["theta"]).to(dev), b["bits"],
                          args.iter_max)
            curves.append(c)
            rows.append({"M": m, "N": n, "snr_db": snr, "converged_at": convergence_iteration(c),
                         "lowest_ber_at": int(np.argmin(c)) + 1, "ber_converged": c[convergence_iteration(c) - 1],
                         "ber_lowest": float(min(c)), "ber_at_10": c[9] if len(c) >= 10 else None})
    budget = iteration_budget(curves)
    line = {"metric": "BER-driven CG iteration budget (Eq. ber_convergence), Veh-A 16-QAM", "value": budget,
            "unit": "iterations", "n_gpus": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{args.iter_frames} Veh-A frames (Table vehAProf delays and powers, nu_max 100 Hz, "
                                   "delta_f 30 kHz) per (grid, SNR), grids 128x32 and 32x32, SNR 0..30 dB step 5, "
                                   f"1..{args.iter_max} CG iterations, eta 1e-2, zeta 1e-12",
                       "frames": args.iter_frames, "max_iters": args.iter_max},
            "paper_budget": 10, "rows": rows, "wall_s": time.time() - t0}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ BER vs SNR workload

def unpack_bits(packed, n_frames):
    """Packed hard bits (uint8, LSB first, as the library writes them) -> [n_frames, bits] 0/1."""
    a = np.asarray(packed, np.uint8).reshape(n_frames, -1)
    return np.unpackbits(a, axis=1, bitorder="little")


def bit_errors(packed, tx_bits, n_frames):
    """Bit errors per frame between the library's packed hard bits and the transmitted bits."""
    got = unpack_bits(packed, n_frames)
    ref = np.asarray(tx_bits, np.uint8).reshape(n_frames, -1)
    return (got != ref).sum(axis=1)


def _lmmse_bits(y_data_td, dk, dl, h, M, N, Q, lam):
    """Worker: the oracle's direct LMMSE (Eq. lmmse, dense Eq. Hdd from the given path list,
    Cholesky) on one SISO frame, and its hard bits (Eq. demod)."""
    from oracle import ddchannel as dc, equalizer as eq, qam, zak
    pl = dc.PathList.from_offsets(M, N, M // 2, N // 2, np.asarray(h, complex), dk, dl)
    H = dc.dense_H(dc.heff_from_paths(pl), M // 2, N // 2)
    y = zak.vec(zak.dzt(np.asarray(y_data_td, complex), M, N))
    x = eq.lmmse_direct(H, y, lam)
    return qam.hard_demod(x, Q)[1].reshape(-1).astype(np.uint8)


def ber_claims(rows, factor=2.0, min_errors=20, sigmas=3.0):
    """The paper's qualitative BER claims (SS-CGA matches LMMSE and beats SS-MRC) checked on
    the sweep's rows.  Ratios SS-CGA / LMMSE use only points where the pair rests on at least
    `min_errors` bit errors; "SS-CGA at or below SS-MRC" holds at a point unless SS-CGA's BER
    exceeds SS-MRC's by more than `sigmas` binomial standard deviations of the difference."""
    out = {"factor": factor, "sigmas": sigmas}
    for key in ("cga", "cga20"):
        ratios = [r[f"ber_{key}"] / r["ber_lmmse"] for r in rows
                  if min(r[f"ber_{key}"], r["ber_lmmse"]) * r["bits"] >= min_errors]
        out[f"worst_ratio_{key}_lmmse"] = max(ratios) if ratios else None
        out[f"{key}_within_factor_of_lmmse"] = (max(ratios) <= factor) if ratios else None
        out[f"{key}_points_compared"] = len(ratios)
    worse = []
    for r in rows:
        pc, pm, nb = r["ber_cga"], r["ber_mrc"], r["bits"]
        sd = np.sqrt((pc * (1 - pc) + pm * (1 - pm)) / nb)
        if pc - pm > sigmas * sd and (pc - pm) * nb >= 1:
            worse.append({k: r[k] for k in ("M", "N", "qam", "snr_db")})
    out["cga_at_or_below_mrc"] = not worse
    out["cga_worse_than_mrc_at"] = worse
    return out


def impl_equalizers(args):
    """SS-CGA and SS-MRC equalisation alone with given lists (each frame's list estimated from
    its pilot frame first, untimed): --eq-frames frames of 64x32 16-QAM, 10 iterations / sweeps,
    device time per call over 20 calls."""
    import torch
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as ge
    ge.build()
    import synth
    from paper_2604_02266_gb300 import Plan, launch_count
    M, N, F = 64, 32, args.eq_frames
    b = synth.fractional_batch(F, seed=SEED + 5, M=M, N=N, Q=Q)
    plan = Plan(M, N, 1, 1, Q)
    yd, nv = torch.from_numpy(b["y_data_td"]).to(dev), torch.from_numpy(b["noise_var"]).to(dev)
    paths = plan.estimate(torch.from_numpy(b["y_pilot_td"]).to(dev), torch.from_numpy(b["theta"]).to(dev), F)
    x = torch.empty(F, 1, M * N, dtype=torch.complex64, device=dev)

    def timed(fn, reps=20):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_cga = timed(lambda: plan.equalize(yd, paths, nv, ITERS, F, x_hat=x))
    ms_mrc = timed(lambda: plan.equalize_mrc(yd, paths, ITERS, F, x_hat=x))
    line = {"metric": "equaliser throughput with given lists (SS-MRC)", "value": F / ms_mrc * 1e3, "unit": "frames/s",
            "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{F} frames 64x32 16-QAM, lists estimated from the pilot frames (mean P "
                                   f"{float(paths.count.float().mean().item()):.1f}), {ITERS} iterations / sweeps, "
                                   "device time per call over 20 calls"},
            "ss_mrc_ms": ms_mrc, "ss_cga_ms": ms_cga, "ss_cga_frames_s": F / ms_cga * 1e3,
            "gpu_launches": launch_count()}
    print(json.dumps(line))
    return 0


def impl_ber(args):
    """BER against SNR on Veh-A frames (Sec. VI's BER study; Table vehAProf): the library's
    SS-CGA (Algorithm 1) and SS-MRC, 10 iterations each as in the paper (and SS-CGA at 20), and
    the FP64 oracle's direct LMMSE (dense Eq. Hdd, Cholesky) on the same estimated path lists,
    QPSK and 16-QAM, grids 32x32 and 128x32.  Also the equalisers' throughput on 1024 frames of
    64x32 16-QAM with given lists."""
    import torch
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    cores = host_cores()
    pool = OraclePool(cores)  # spawned workers for the LMMSE leg
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as ge
    ge.build()
    import synth
    from paper_2604_02266_gb300 import Plan
    rows = []
    t0 = time.time()
    try:
        for (m, n, frames) in ((32, 32, args.ber_frames), (128, 32, args.ber_frames_large)):
            for q in (4, 16):
                plan = Plan(m, n, 1, 1, q)
                for snr in range(0, 31, 5):
                    b = synth.veh_a_batch(frames, SEED + 7 * m + q + snr, M=m, N=n, Q=q, snr_db=(snr,))
                    yp, yd = torch.from_numpy(b["y_pilot_td"]).to(dev), torch.from_numpy(b["y_data_td"]).to(dev)
                    nv, th = torch.from_numpy(b["noise_var"]).to(dev), torch.from_numpy(b["theta"]).to(dev)
                    paths = plan.estimate(yp, th, frames)
                    res = {}
                    for name, it in (("cga", 10), ("cga20", 20)):
                        x = plan.equalize(yd, paths, nv, it, frames)
                        _, bits = plan.demap(x, nv, frames, llr=False)
                        res[name] = int(bit_errors(bits.cpu().numpy(), b["bits"], frames).sum())
                    x = plan.equalize_mrc(yd, paths, 10, frames)
                    _, bits = plan.demap(x, nv, frames, llr=False)
                    res["mrc"] = int(bit_errors(bits.cpu().numpy(), b["bits"], frames).sum())
                    lists = paths.to_host()
                    futs = [pool.ex.submit(_lmmse_bits, b["y_data_td"][f, 0], lists[f][0], lists[f][1], lists[f][2], m,
                                           n, q, float(b["noise_var"][f])) for f in range(frames)]
                    lm = np.stack([fu.result() for fu in futs])
                    res["lmmse"] = int((lm != b["bits"].reshape(frames, -1)).sum())
                    nbits = int(b["bits"].size)
                    rows.append({"M": m, "N": n, "qam": q, "snr_db": snr, "frames": frames, "bits": nbits,
                                 "paths_mean": float(paths.count.float().mean().item()),
                                 "ber_cga": res["cga"] / nbits, "ber_cga20": res["cga20"] / nbits,
                                 "ber_mrc": res["mrc"] / nbits, "ber_lmmse": res["lmmse"] / nbits})
    finally:
        pool.close()
    sweep_s = time.time() - t0

    # equaliser throughput with given lists: 1024 frames of 64x32 16-QAM, 10 iterations
    F = FRAMES
    b = synth.fractional_batch(F, seed=SEED + 5, M=M, N=N, Q=Q)
    plan = Plan(M, N, 1, 1, Q)
    yd, nv = torch.from_numpy(b["y_data_td"]).to(dev), torch.from_numpy(b["noise_var"]).to(dev)
    paths = plan.estimate(torch.from_numpy(b["y_pilot_td"]).to(dev), torch.from_numpy(b["theta"]).to(dev), F)
    x = torch.empty(F, 1, M * N, dtype=torch.complex64, device=dev)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_cga = timed(lambda: plan.equalize(yd, paths, nv, ITERS, F, x_hat=x))
    ms_mrc = timed(lambda: plan.equalize_mrc(yd, paths, ITERS, F, x_hat=x))
    claims = ber_claims(rows)
    line = {"metric": "BER vs SNR: SS-CGA, SS-MRC and LMMSE on Veh-A frames",
            "value": claims["worst_ratio_cga20_lmmse"], "unit": "worst BER ratio SS-CGA (20 iterations) / LMMSE",
            "n_gpus": 1, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (LMMSE: f64 oracle)", "data": "synthetic",
            "config": {"workload": "Veh-A frames (Table vehAProf delays and powers, nu_max 100 Hz, delta_f 30 kHz), "
                                   "separate pilot frame per frame, threshold 3 sigma, p_max 64, SNR 0..30 dB step 5, "
                                   "QPSK and 16-QAM; grids 32x32 and 128x32; 10 iterations (SS-CGA also 20); "
                                   "LMMSE = the FP64 oracle's dense Cholesky solve on the library's path lists",
                       "frames_32x32": args.ber_frames, "frames_128x32": args.ber_frames_large},
            "claims": claims, "rows": rows, "sweep_wall_s": sweep_s, "host_cores": cores,
            "equalizer_throughput": {"workload": f"{F} frames 64x32 16-QAM, given path lists (mean P "
                                                 f"{float(paths.count.float().mean().item()):.1f}), {ITERS} iterations",
                                     "ss_cga_frames_s": F / ms_cga * 1e3, "ss_mrc_frames_s": F / ms_mrc * 1e3,
                                     "ss_cga_ms": ms_cga, "ss_mrc_ms": ms_mrc}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------- paper-scale workload

PAPER_M, PAPER_N = 16384, 32


def impl_paper(args):
    """The paper's operating point (M, N) = (16384, 32), 16-QAM SISO: one pilot + data frame
    per call (524288 DD bins, 4 MB per FP32 vector) on the grid receiver, the whole GPU per
    frame.  Device time per call, p50 / p99 over the calls; the paper's own figure for the
    same packet on an H200 is 1.69 ms p99.9 (context only, other hardware)."""
    import torch
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as ge
    ge.build()
    import synth
    from paper_2604_02266_gb300 import Plan, launch_count
    M, N, pool = PAPER_M, PAPER_N, args.paper_pool
    b = synth.fractional_batch(pool, seed=SEED + 16384, M=M, N=N, Q=Q, snr_db=tuple(range(0, 31, 2)))
    plan = Plan(M, N, 1, 1, Q)
    if args.ctas:
        plan.set_tuning(ctas_per_sm=args.ctas)
    yp, yd = torch.from_numpy(b["y_pilot_td"]).to(dev), torch.from_numpy(b["y_data_td"]).to(dev)
    nv, th = torch.from_numpy(b["noise_var"]).to(dev), torch.from_numpy(b["theta"]).to(dev)
    outs = plan._rx_outputs(1, dev, True, False, False)

    def call(f):
        plan.rx(yp[f:f + 1], yd[f:f + 1], nv[f:f + 1], th[f:f + 1], ITERS, 1, out=outs)

    for i in range(max(args.warmup, 3)):
        call(i % pool)
    torch.cuda.synchronize()
    ts = []
    for i in range(args.paper_calls):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call(i % pool)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts = np.array(ts)
    launches = launch_count()
    P = outs[0].count.cpu().numpy()
    st = outs[4].cpu().numpy()
    # several frames in one call (the kernel takes them one after another)
    batch = plan._rx_outputs(pool, dev, False, False, False)
    plan.rx(yp, yd, nv, th, ITERS, pool, out=batch)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.rx(yp, yd, nv, th, ITERS, pool, out=batch)
    e1.record()
    torch.cuda.synchronize()
    ms_batch = e0.elapsed_time(e1)
    line = {"metric": "paper-scale one-packet receiver latency (p50/p99), 16384x32 16-QAM SISO", "value": float(np.percentile(ts, 50)),
            "unit": "ms", "n_gpus": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "one pilot frame + one data frame per call, M=16384, N=32, 16-QAM, 6-path fractional "
                                   "channel, SNR 0..30 dB, threshold 3 sigma, p_max 64, 10 CG iterations, device time "
                                   "per call", "calls": args.paper_calls, "pool": pool},
            "p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)), "max_ms": float(ts.max()),
            "frames_s_one_per_call": 1e3 / float(np.percentile(ts, 50)),
            "frames_s_in_one_call": pool / ms_batch * 1e3, "paths_per_frame": float(P.mean()),
            "status_ok_or_truncated": float(np.isin(st, (0, 6)).mean()), "gpu_launches_per_call": launches,
            "paper_context": {"p99_9_ms": 1.69, "hardware": "H200", "scope": "pilot + data frame, (16384, 32)"}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------- one-frame latency workload

LATENCY_SHAPES = ((64, 32), (128, 32), (64, 64), (128, 64), (256, 32))


def impl_latency(args):
    """Per-frame latency of the receiver called one frame at a time (the paper's real-time
    setting: each packet is processed as it arrives): p50 / p99 over a stream of frames, for
    one CTA per frame (or the large-frame kernel) and for the 2-CTA cluster receiver."""
    import torch
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import __graft_entry__ as ge
    ge.build()
    import synth
    from paper_2604_02266_gb300 import Plan
    rows = []
    for (m, n) in LATENCY_SHAPES:
        b = synth.fractional_batch(args.latency_frames, seed=SEED + m + n, M=m, N=n, Q=Q)
        yp, yd = torch.from_numpy(b["y_pilot_td"]).to(dev), torch.from_numpy(b["y_data_td"]).to(dev)
        nv, th = torch.from_numpy(b["noise_var"]).to(dev), torch.from_numpy(b["theta"]).to(dev)
        res = {"M": m, "N": n}
        for name, cl in (("one_cta", 1), ("cluster2", 2), ("cluster4", 4)):
            plan = Plan(m, n, 1, 1, Q)
            plan.set_tuning(cluster=cl)
            outs = plan._rx_outputs(1, dev, False, False, False)
            for f in range(3):
                plan.rx(yp[f:f + 1], yd[f:f + 1], nv[f:f + 1], th[f:f + 1], ITERS, 1, out=outs)
            torch.cuda.synchronize()
            ts = []
            for f in range(args.latency_frames):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                plan.rx(yp[f:f + 1], yd[f:f + 1], nv[f:f + 1], th[f:f + 1], ITERS, 1, out=outs)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ts = np.array(ts)
            res[name] = {"p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
                         "within_0_5ms": float((ts <= DEADLINE_MS).mean())}
        rows.append(res)
    head = rows[0]["one_cta"]
    line = {"metric": "one-frame Zak-OTFS receiver latency (p50/p99), SISO 16-QAM", "value": head["p50_ms"],
            "unit": "ms", "n_gpus": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "one frame per call: pilot + data frame in HBM, 6-path fractional channel, "
                                   "SNR 0..30 dB, 10 CG iterations, device time per call", "frames": args.latency_frames},
            "shapes": rows}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 2000; 20 with --impl reference)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="zotfs", choices=["zotfs", "reference"])
    ap.add_argument("--threads", type=int, default=0, help="threads per frame (tuning)")
    ap.add_argument("--radix", type=int, default=0, help="FFT radix (tuning)")
    ap.add_argument("--ctas", type=int, default=0, help="CTAs per SM (tuning)")
    ap.add_argument("--plain-frames", type=int, default=32)
    ap.add_argument("--oracle-frames", type=int, default=24, help="oracle sample per host core for cpu_baseline")
    ap.add_argument("--ref-frames", type=int, default=4, help="oracle frames per host core per step (--impl reference)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="batch", choices=["batch", "serve", "mixed", "mimo", "latency", "paper", "packets", "iterations", "ber",
                             "equalizers"],
                    help="batch: the 64x32 16-QAM batch (default line); serve: the Poisson serving loop; "
                         "mixed: the uneven FP16/BF16 batch under CUDA graphs; mimo: 4x4 128x64 64-QAM frames; "
                         "latency: one frame per call; paper: one 16384x32 packet per call on the grid receiver; "
                         "packets: one pilot frame per D data frames (pilot reuse); "
                         "iterations: the BER-driven CG iteration budget on Veh-A frames; "
                         "equalizers: SS-CGA and SS-MRC alone on given lists")
    ap.add_argument("--eq-frames", type=int, default=2048, help="equalizers: frames per call")
    ap.add_argument("--mimo-steps", type=int, default=5, help="mimo: timed steps")
    ap.add_argument("--latency-frames", type=int, default=200, help="latency: frames per shape")
    ap.add_argument("--paper-calls", type=int, default=200, help="paper: timed one-packet calls")
    ap.add_argument("--packet-data", type=int, default=8, help="packets: data frames per pilot frame")
    ap.add_argument("--iter-frames", type=int, default=32, help="iterations: Veh-A frames per (grid, SNR)")
    ap.add_argument("--iter-max", type=int, default=30, help="iterations: CG iterations profiled")
    ap.add_argument("--ber-frames", type=int, default=32, help="ber: Veh-A frames per 32x32 point")
    ap.add_argument("--ber-frames-large", type=int, default=8, help="ber: Veh-A frames per 128x32 point")
    ap.add_argument("--paper-pool", type=int, default=8, help="paper: synthetic packets cycled through")
    ap.add_argument("--mixed-steps", type=int, default=20, help="mixed: timed steps per storage type")
    ap.add_argument("--tune-frames", type=int, default=64, help="mixed: frames per shape group the autotuner times")
    ap.add_argument("--tuning-file", default="", help="mixed: write the autotuner's JSON here ({dtype} expands)")
    ap.add_argument("--rates", type=lambda v: [float(x) for x in v.split(",")], default=[200000.0, 20000.0],
                    help="serve: offered frames/s, one run each")
    ap.add_argument("--duration", type=float, default=1.0, help="serve: seconds of arrivals per rate")
    ap.add_argument("--pool", type=int, default=2, help="serve: synthetic frames per (M, N, antennas, QAM) class")
    ap.add_argument("--serve-mix", default="c5", choices=["c5", "c2"],
                    help="serve: c5 = mixed shapes/antennas/QAM, c2 = 64x32 SISO 16-QAM frames only")
    ap.add_argument("--wave-frames", type=int, default=512, help="serve: frames admitted per wave")
    ap.add_argument("--waves", type=int, default=16, help="serve: waves in flight")
    ap.add_argument("--light-work", type=int, default=8192,
                    help="serve (c5 mix): frames with M*N*n_rx*n_tx up to this run in their own waves")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 20 if args.impl == "reference" else 2000
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return impl_reference(args)
    if args.workload == "serve":
        return impl_serve(args)
    if args.workload == "mixed":
        return impl_mixed(args)
    if args.workload == "mimo":
        return impl_mimo(args)
    if args.workload == "paper":
        return impl_paper(args)
    if args.workload == "packets":
        return impl_packets(args)
    if args.workload == "iterations":
        return impl_iterations(args)
    if args.workload == "latency":
        return impl_latency(args)
    if args.workload == "ber":
        return impl_ber(args)
    if args.workload == "equalizers":
        return impl_equalizers(args)
    return impl_zotfs(args)


if __name__ == "__main__":
    sys.exit(main())
