"""GB300-native Zak-OTFS receiver hot path (SS-CGA), Python binding.

The library itself is ``libzotfs.so`` (hand-written CUDA for sm_103a, C ABI in
``include/zotfs.h``).  This package only marshals PyTorch tensors into that ABI: device
pointers, sizes and the current CUDA stream.  There is no CPU or PyTorch fallback; if the
library is missing, loading it raises.

Tensor conventions (see include/zotfs.h for the full contract):

* complex data is ``torch.complex64`` (ZOTFS_C64), or a ``[..., 2]`` float16 / bfloat16
  tensor for 16-bit storage;
* a DD grid is vectorised q = l*M + k; a TD frame is in sample order;
* frames are batched on the leading axis: pilots ``[F, n_tx, n_rx, M*N]``, data
  ``[F, n_rx, M*N]``, ``x_hat [F, n_tx, M*N]``, LLRs ``[F, n_tx, M*N, bps]``,
  bits ``[F, n_tx, M*N*bps/8]`` (uint8, LSB-first).
"""

import ctypes as C
import math

import torch

from . import _zotfs as Z
from ._zotfs import (ZotfsError, OK, EINVAL, ENOMEM, ECUDA, EUNSUPPORTED, ETIMEOUT, ETRUNCATED,  # noqa: F401
                     ENONFINITE, STATUS_NAMES, C64, C32_F16, C32_BF16, C128, COMPUTE_FP32, COMPUTE_FP64,
                     PILOT_SEPARATE, PILOT_EMBEDDED, PULSE_SINC, PULSE_RECT)

__all__ = ["Plan", "Paths", "Batch", "Graph", "Server", "ZotfsError", "autotune", "save_tuning", "load_tuning",
           "library_path", "launch_count"]

_DTYPES = {C64: torch.complex64, C32_F16: torch.float16, C32_BF16: torch.bfloat16, C128: torch.complex128}


def library_path():
    return Z.LIB_PATH


def launch_count():
    """Fused-kernel launches made by the most recent library call in this thread."""
    return int(Z.zotfs_last_launch_count())


def _p(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _s(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _need_cuda(*ts):
    for t in ts:
        if t is not None:
            if not t.is_cuda:
                raise ValueError("zotfs tensors must live on a CUDA device")
            if not t.is_contiguous():
                raise ValueError("zotfs tensors must be contiguous")


class Paths:
    """Device path lists for ``n_lists = n_frames * n_rx * n_tx`` antenna pairs."""

    def __init__(self, n_lists, p_max, tap_dtype=C64, device="cuda"):
        self.n_lists = n_lists
        self.p_max = p_max
        self.tap_dtype = tap_dtype
        self.count = torch.zeros(n_lists, dtype=torch.int32, device=device)
        self.status = torch.zeros(n_lists, dtype=torch.int32, device=device)
        self.dk = torch.zeros(n_lists * p_max, dtype=torch.int16, device=device)
        self.dl = torch.zeros(n_lists * p_max, dtype=torch.int16, device=device)
        if tap_dtype in (C64, C128):
            self.h = torch.zeros(n_lists * p_max, dtype=_DTYPES[tap_dtype], device=device)
        else:
            self.h = torch.zeros(n_lists * p_max, 2, dtype=_DTYPES[tap_dtype], device=device)
        self._c = Z.zotfs_paths(self.count.data_ptr(), self.status.data_ptr(), self.dk.data_ptr(),
                                self.dl.data_ptr(), self.h.data_ptr(), p_max, tap_dtype)

    @property
    def c(self):
        return C.byref(self._c)

    def to_host(self):
        """List of (dk, dl, h) numpy arrays per list (h as complex128)."""
        cnt = self.count.cpu().numpy()
        dk = self.dk.cpu().numpy().reshape(self.n_lists, self.p_max)
        dl = self.dl.cpu().numpy().reshape(self.n_lists, self.p_max)
        if self.tap_dtype in (C64, C128):
            h = self.h.cpu().numpy().reshape(self.n_lists, self.p_max)
        else:
            hh = self.h.float().cpu().numpy().reshape(self.n_lists, self.p_max, 2)
            h = hh[..., 0] + 1j * hh[..., 1]
        return [(dk[i, :cnt[i]].astype(int), dl[i, :cnt[i]].astype(int), h[i, :cnt[i]].astype(complex))
                for i in range(self.n_lists)]


class Plan:
    """A zotfs plan: one grid shape, antenna configuration and QAM order."""

    def __init__(self, M, N, n_rx=1, n_tx=1, qam=16, pulse=PULSE_SINC, **options):
        h = C.c_void_p()
        Z.check(Z.zotfs_plan_create(M, N, n_rx, n_tx, pulse, qam, C.byref(h)))
        self._h = h
        self.M, self.N, self.n_rx, self.n_tx, self.qam = M, N, n_rx, n_tx, qam
        self.MN = M * N
        self.bps = int(round(math.log2(qam)))
        if options:
            self.set_options(**options)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                Z.zotfs_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    # ----------------------------------------------------------------- configuration
    def options(self):
        o = Z.zotfs_options()
        Z.check(Z.zotfs_plan_get_options(self._h, C.byref(o)))
        return {f: getattr(o, f) for f, _ in o._fields_}

    def set_options(self, **kw):
        o = Z.zotfs_options()
        Z.check(Z.zotfs_plan_get_options(self._h, C.byref(o)))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        Z.check(Z.zotfs_plan_set_options(self._h, C.byref(o)))

    def set_tuning(self, threads_per_frame=0, fft_radix=0, ctas_per_sm=0, cluster=0, frames_per_cta=0):
        t = Z.zotfs_tuning(threads_per_frame, fft_radix, ctas_per_sm, cluster, frames_per_cta)
        Z.check(Z.zotfs_plan_set_tuning(self._h, C.byref(t)))

    def tuning(self):
        t = Z.zotfs_tuning()
        Z.check(Z.zotfs_plan_get_tuning(self._h, C.byref(t)))
        return {"threads_per_frame": t.threads_per_frame, "fft_radix": t.fft_radix, "ctas_per_sm": t.ctas_per_sm,
                "cluster": t.cluster, "frames_per_cta": t.frames_per_cta}

    @property
    def p_max(self):
        return self.options()["p_max"]

    @property
    def cdtype(self):
        """torch dtype of the plan's complex vectors (complex64, or complex128 for FP64 plans)."""
        return torch.complex128 if self.options()["compute"] == COMPUTE_FP64 else torch.complex64

    def new_paths(self, n_frames, device="cuda"):
        o = self.options()
        return Paths(n_frames * self.n_rx * self.n_tx, o["p_max"], o["tap_dtype"], device)

    # ---------------------------------------------------------------------- stages
    def dzt(self, y_td, out=None, stream=None):
        n = y_td.numel() // self.MN if y_td.is_complex() else y_td.numel() // (2 * self.MN)
        out = torch.empty(n, self.MN, dtype=self.cdtype, device=y_td.device) if out is None else out
        _need_cuda(y_td, out)
        Z.check(Z.zotfs_dzt(self._h, _p(y_td), _p(out), n, _s(stream)))
        return out

    def estimate(self, y_pilot_td, theta, n_frames, paths=None, stream=None):
        paths = self.new_paths(n_frames, y_pilot_td.device) if paths is None else paths
        _need_cuda(y_pilot_td, theta)
        Z.check(Z.zotfs_estimate(self._h, _p(y_pilot_td), _p(theta), n_frames, paths.c, _s(stream)))
        return paths

    def ss_apply(self, paths, v, n_frames, adjoint=False, out=None, status=None, stream=None):
        nout = self.n_tx if adjoint else self.n_rx
        out = torch.empty(n_frames, nout, self.MN, dtype=self.cdtype, device=v.device) if out is None else out
        _need_cuda(v, out, status)
        Z.check(Z.zotfs_ss_apply(self._h, paths.c, _p(v), _p(out), int(bool(adjoint)), n_frames, _p(status),
                                 _s(stream)))
        return out

    def equalize(self, y, paths, noise_var, iters, n_frames, y_is_dd=False, x_hat=None, status=None,
                 stream=None):
        x_hat = (torch.empty(n_frames, self.n_tx, self.MN, dtype=self.cdtype, device=y.device)
                 if x_hat is None else x_hat)
        _need_cuda(y, noise_var, x_hat, status)
        Z.check(Z.zotfs_equalize(self._h, _p(y), int(bool(y_is_dd)), paths.c, _p(noise_var), iters, _p(x_hat),
                                 n_frames, _p(status), _s(stream)))
        return x_hat

    def equalize_mrc(self, y, paths, iters, n_frames, y_is_dd=False, x_hat=None, status=None, stream=None):
        """SS-MRC (zotfs_equalize_mrc): decision-feedback maximal-ratio combining on the path
        lists; returns the soft estimate of the last sweep."""
        x_hat = (torch.empty(n_frames, 1, self.MN, dtype=torch.complex64, device=y.device)
                 if x_hat is None else x_hat)
        _need_cuda(y, x_hat, status)
        Z.check(Z.zotfs_equalize_mrc(self._h, _p(y), int(bool(y_is_dd)), paths.c, iters, _p(x_hat), _p(status),
                                     n_frames, _s(stream)))
        return x_hat

    def demap(self, x_hat, noise_var, n_frames, llr=True, bits=True, stream=None):
        dev = x_hat.device
        L = torch.empty(n_frames, self.n_tx, self.MN, self.bps, dtype=torch.float32, device=dev) if llr else None
        B = torch.empty(n_frames, self.n_tx, self.MN * self.bps // 8, dtype=torch.uint8, device=dev) if bits else None
        _need_cuda(x_hat, noise_var, L, B)
        Z.check(Z.zotfs_demap(self._h, _p(x_hat), _p(noise_var), _p(L), _p(B), n_frames, _s(stream)))
        return L, B

    def _rx_outputs(self, n_frames, device, want_paths, want_x, want_llr):
        paths = self.new_paths(n_frames, device) if want_paths else None
        x = torch.empty(n_frames, self.n_tx, self.MN, dtype=self.cdtype, device=device) if want_x else None
        L = torch.empty(n_frames, self.n_tx, self.MN, self.bps, dtype=torch.float32, device=device) if want_llr else None
        B = torch.empty(n_frames, self.n_tx, self.MN * self.bps // 8, dtype=torch.uint8, device=device)
        st = torch.empty(n_frames, dtype=torch.int32, device=device)
        return paths, x, L, B, st

    def rx(self, y_pilot_td, y_data_td, noise_var, theta, iters, n_frames, want_paths=False, want_x=False,
           want_llr=False, out=None, stream=None, plain=False):
        """Whole receiver per frame (fused persistent kernel, or the plain form)."""
        if out is None:
            out = self._rx_outputs(n_frames, y_data_td.device, want_paths, want_x, want_llr)
        paths, x, L, B, st = out
        _need_cuda(y_pilot_td, y_data_td, noise_var, theta, x, L, B, st)
        fn = Z.zotfs_rx_plain if plain else Z.zotfs_rx
        Z.check(fn(self._h, _p(y_pilot_td), _p(y_data_td), _p(noise_var), _p(theta), iters,
                   paths.c if paths is not None else None, _p(x), _p(L), _p(B), _p(st), n_frames, _s(stream)))
        return {"paths": paths, "x_hat": x, "llr": L, "bits": B, "status": st}

    def rx_lists(self, y_data_td, paths, noise_var, iters, n_frames, path_ids=None, n_sets=None, want_x=False,
                 want_llr=False, out=None, stream=None):
        """Data frames through Zak transform, CGA and demapping with lists estimated earlier
        (zotfs_rx_lists): frame f uses list set ``path_ids[f]`` of ``paths`` (pilot reuse)."""
        if out is None:
            _, x, L, B, st = self._rx_outputs(n_frames, y_data_td.device, False, want_x, want_llr)
        else:
            x, L, B, st = out
        if n_sets is None:
            n_sets = int(paths.count.numel() // (self.n_rx * self.n_tx))
        _need_cuda(y_data_td, noise_var, path_ids, x, L, B, st)
        Z.check(Z.zotfs_rx_lists(self._h, _p(y_data_td), paths.c, _p(path_ids), n_sets, _p(noise_var), iters, _p(x),
                                 _p(L), _p(B), _p(st), n_frames, _s(stream)))
        return {"x_hat": x, "llr": L, "bits": B, "status": st}


class Batch:
    """An uneven batch (zotfs_batch_create / zotfs_rx_batch).  ``frames`` is a list of dicts
    with the zotfs_frame_desc fields; tensor-valued fields are device tensors whose
    storage must stay alive while the batch is used (the Batch keeps references)."""

    _PTR_FIELDS = ("y_pilot", "y_data", "x_hat", "llr", "bits", "path_count", "path_dk", "path_dl", "path_h")

    @classmethod
    def descriptors(cls, frames):
        """zotfs_frame_desc array for a list of frame dicts, and the tensors it points into."""
        n = len(frames)
        arr = (Z.zotfs_frame_desc * max(n, 1))()
        keep = []
        for i, fr in enumerate(frames):
            d = arr[i]
            d.K0 = d.L0 = -1
            for key, val in fr.items():
                if key in cls._PTR_FIELDS:
                    if val is not None:
                        _need_cuda(val)
                        keep.append(val)
                        setattr(d, key, val.data_ptr())
                else:
                    setattr(d, key, val)
        return arr, keep

    def __init__(self, frames, threads_per_frame=0, ctas_per_sm=0, fft_radix=0, tuning=None, max_sms=0, cluster=0):
        n = len(frames)
        arr, self._keep = self.descriptors(frames)
        entries = tuning or []
        tarr = (Z.zotfs_tuning_entry * max(len(entries), 1))()
        for i, (shape, tun) in enumerate(entries):
            tarr[i].M, tarr[i].N, tarr[i].n_rx, tarr[i].n_tx = shape
            tarr[i].tuning = Z.zotfs_tuning(tun.get("threads_per_frame", 0), tun.get("fft_radix", 0),
                                            tun.get("ctas_per_sm", 0), tun.get("cluster", 0),
                                            tun.get("frames_per_cta", 0))
        opts = Z.zotfs_batch_opts(threads_per_frame, ctas_per_sm, fft_radix, len(entries), tarr, max_sms, cluster)
        h = C.c_void_p()
        Z.check(Z.zotfs_batch_create(arr, n, C.byref(opts), C.byref(h)))
        self._h = h
        self.n_frames = n

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                Z.zotfs_batch_destroy(h)
            except Exception:
                pass
            self._h = None

    def run(self, status, stream=None):
        _need_cuda(status)
        Z.check(Z.zotfs_rx_batch(self._h, _p(status), _s(stream)))
        return status

    def capture(self, status):
        """A CUDA graph of one run of this batch (zotfs_batch_capture)."""
        return Graph(self, status)


class Graph:
    """An instantiated CUDA graph of one batch run; ``launch`` replays it on a stream."""

    def __init__(self, batch, status):
        _need_cuda(status)
        h = C.c_void_p()
        Z.check(Z.zotfs_batch_capture(batch._h, _p(status), C.byref(h)))
        self._h = h
        self._keep = (batch, status)

    def launch(self, stream=None):
        Z.check(Z.zotfs_graph_launch(self._h, _s(stream)))

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            Z.zotfs_graph_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(frames, warmup=0, reps=0, max_frames=0, stream=None):
    """Time every launch shape per (M, N, n_rx, n_tx) group of ``frames`` (zotfs_autotune) and
    return one dict per group: the shape, the chosen tuning, its cost (SM-ms per frame) and
    the default and best times of the group's timing set.  The frames' outputs are not
    written (the tuner writes to its own scratch)."""
    arr, keep = Batch.descriptors(frames)
    groups = len({(f["M"], f["N"], f["n_rx"], f["n_tx"]) for f in frames})
    res = (Z.zotfs_tuning_result * max(groups, 1))()
    n = C.c_int(0)
    opts = Z.zotfs_autotune_opts(warmup, reps, max_frames)
    Z.check(Z.zotfs_autotune(arr, len(frames), C.byref(opts), res, groups, C.byref(n), _s(stream)))
    out = []
    for i in range(n.value):
        r = res[i]
        b = r.best
        out.append({"M": b.M, "N": b.N, "n_rx": b.n_rx, "n_tx": b.n_tx,
                    "threads_per_frame": b.tuning.threads_per_frame, "fft_radix": b.tuning.fft_radix,
                    "ctas_per_sm": b.tuning.ctas_per_sm, "cluster": b.tuning.cluster,
                    "frames_per_cta": b.tuning.frames_per_cta,
                    "sm_ms_per_frame": r.sm_ms_per_frame, "ms_best": r.ms_best,
                    "ms_default": r.ms_default,
                    "n_candidates": r.n_candidates, "n_frames": r.n_frames})
    del keep
    return out


def save_tuning(path, results, device_name=None):
    """Persist autotuner results as JSON (one entry per shape group)."""
    import json
    with open(path, "w") as fh:
        json.dump({"format": "zotfs-tuning-1", "device": device_name, "entries": list(results)}, fh, indent=1)


def load_tuning(path):
    """Read a JSON tuning file into the ``tuning=`` argument of Batch: [((M, N, n_rx, n_tx), dict)]."""
    import json
    with open(path) as fh:
        doc = json.load(fh)
    if doc.get("format") != "zotfs-tuning-1":
        raise ValueError(f"{path}: not a zotfs tuning file")
    out = []
    for e in doc["entries"]:
        shape = (int(e["M"]), int(e["N"]), int(e["n_rx"]), int(e["n_tx"]))
        out.append((shape, {k: int(e.get(k, 0)) for k in ("threads_per_frame", "fft_radix", "ctas_per_sm", "cluster",
                                                           "frames_per_cta")}))
    return out


class Server:
    """Continuous-batching request loop (zotfs_server_*).  Requests reference device tensors
    (pilot and data TD frames, complex64) that must stay alive until their completion."""

    def __init__(self, p_max=64, max_wave_frames=256, waves_in_flight=4, keep_llr=False, arena_bytes=1 << 30,
                 max_M=256, max_N=64, max_ant=4, light_work=0):
        o = Z.zotfs_server_opts(p_max, max_wave_frames, waves_in_flight, int(bool(keep_llr)), arena_bytes, max_M,
                                max_N, max_ant, light_work)
        h = C.c_void_p()
        Z.check(Z.zotfs_server_create(C.byref(o), C.byref(h)))
        self._h = h
        self.p_max = p_max
        self._keep = {}

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            Z.zotfs_server_destroy(h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def request(tag, y_pilot, y_data, M, N, n_rx, n_tx, qam, iters, noise_var, theta, a_pilot=0.0, cg_eps=0.0):
        _need_cuda(y_pilot, y_data)
        return Z.zotfs_request(M, N, n_rx, n_tx, qam, iters, noise_var, theta, a_pilot, cg_eps, y_pilot.data_ptr(),
                               y_data.data_ptr(), tag)

    def submit(self, reqs):
        arr = (Z.zotfs_request * len(reqs))(*reqs)
        Z.check(Z.zotfs_server_submit(self._h, arr, len(reqs)))

    def replay(self, reqs, arrival_s):
        arr = (Z.zotfs_request * len(reqs))(*reqs)
        ts = (C.c_double * len(reqs))(*[float(t) for t in arrival_s])
        Z.check(Z.zotfs_server_replay(self._h, arr, ts, len(reqs)))

    def poll(self, max_n=4096):
        buf = (Z.zotfs_completion * max_n)()
        k = Z.zotfs_server_poll(self._h, buf, max_n)
        return [buf[i] for i in range(k)]

    def release(self, tag):
        Z.check(Z.zotfs_server_release(self._h, tag))

    def stats(self):
        s = Z.zotfs_server_stats()
        Z.check(Z.zotfs_server_get_stats(self._h, C.byref(s)))
        return {n: getattr(s, n) for n, _ in s._fields_}

    def read(self, tag, n_tx, MN, bps, n_lists, llr=False):
        """Host copies of a completed frame's outputs: dict of numpy arrays."""
        import numpy as np
        bits = np.zeros(n_tx * MN * bps // 8, np.uint8)
        L = np.zeros(n_tx * MN * bps, np.float32) if llr else None
        pc = np.zeros(n_lists, np.int32)
        dk = np.zeros(n_lists * self.p_max, np.int16)
        dl = np.zeros(n_lists * self.p_max, np.int16)
        h = np.zeros(n_lists * self.p_max, np.complex64)
        ptr = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)
        Z.check(Z.zotfs_server_read(self._h, tag, ptr(bits), ptr(L), ptr(pc), ptr(dk), ptr(dl), ptr(h)))
        return {"bits": bits, "llr": L, "count": pc, "dk": dk, "dl": dl, "h": h}

from . import iterations  # noqa: E402,F401  (BER-driven iteration budget)
