"""ctypes binding of libzotfs.so: the C ABI of include/zotfs.h under the same names.

Argument marshalling only.  Every computation runs in the library's CUDA kernels; if the
library is missing this module raises instead of falling back to anything else.
"""

import ctypes as C
import os

from . import build as _build

LIB_PATH = _build.LIB


class ZotfsError(RuntimeError):
    """A zotfs call returned a status other than ZOTFS_OK."""

    def __init__(self, status, message):
        super().__init__(f"zotfs status {status}: {message}")
        self.status = status


# status codes (zotfs_status)
OK, EINVAL, ENOMEM, ECUDA, EUNSUPPORTED, ETIMEOUT, ETRUNCATED, ENONFINITE = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EUNSUPPORTED", "ETIMEOUT", "ETRUNCATED", "ENONFINITE"]
# enums
PULSE_SINC, PULSE_RECT = 0, 1
C64, C32_F16, C32_BF16, C128 = 0, 1, 2, 3
COMPUTE_FP32, COMPUTE_FP64 = 0, 1
PILOT_SEPARATE, PILOT_EMBEDDED = 0, 1


class zotfs_options(C.Structure):
    _fields_ = [("pilot_mode", C.c_int32), ("K0", C.c_int32), ("L0", C.c_int32), ("a_pilot", C.c_float),
                ("guard", C.c_int32), ("p_max", C.c_int32), ("in_dtype", C.c_int32), ("tap_dtype", C.c_int32),
                ("compute", C.c_int32), ("cg_eps", C.c_float)]


class zotfs_paths(C.Structure):
    _fields_ = [("count", C.c_void_p), ("status", C.c_void_p), ("dk", C.c_void_p), ("dl", C.c_void_p),
                ("h", C.c_void_p), ("p_max", C.c_int32), ("tap_dtype", C.c_int32)]


class zotfs_tuning(C.Structure):
    _fields_ = [("threads_per_frame", C.c_int32), ("fft_radix", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("cluster", C.c_int32), ("frames_per_cta", C.c_int32)]


class zotfs_frame_desc(C.Structure):
    _fields_ = [("M", C.c_int32), ("N", C.c_int32), ("n_rx", C.c_int32), ("n_tx", C.c_int32),
                ("qam", C.c_int32), ("iters", C.c_int32), ("pilot_mode", C.c_int32), ("guard", C.c_int32),
                ("p_max", C.c_int32), ("in_dtype", C.c_int32), ("K0", C.c_int32), ("L0", C.c_int32),
                ("noise_var", C.c_float), ("theta", C.c_float), ("a_pilot", C.c_float), ("cg_eps", C.c_float),
                ("y_pilot", C.c_void_p), ("y_data", C.c_void_p), ("x_hat", C.c_void_p), ("llr", C.c_void_p),
                ("bits", C.c_void_p), ("path_count", C.c_void_p), ("path_dk", C.c_void_p),
                ("path_dl", C.c_void_p), ("path_h", C.c_void_p)]


class zotfs_tuning_entry(C.Structure):
    _fields_ = [("M", C.c_int32), ("N", C.c_int32), ("n_rx", C.c_int32), ("n_tx", C.c_int32),
                ("tuning", zotfs_tuning)]


class zotfs_batch_opts(C.Structure):
    _fields_ = [("threads_per_frame", C.c_int32), ("ctas_per_sm", C.c_int32), ("fft_radix", C.c_int32),
                ("n_tuning", C.c_int32), ("tuning", C.POINTER(zotfs_tuning_entry)), ("max_sms", C.c_int32),
                ("cluster", C.c_int32)]


class zotfs_autotune_opts(C.Structure):
    _fields_ = [("warmup", C.c_int32), ("reps", C.c_int32), ("max_frames", C.c_int32)]


class zotfs_tuning_result(C.Structure):
    _fields_ = [("best", zotfs_tuning_entry), ("ms_best", C.c_float), ("ms_default", C.c_float),
                ("sm_ms_per_frame", C.c_float), ("n_candidates", C.c_int32), ("n_frames", C.c_int32)]


class zotfs_server_opts(C.Structure):
    _fields_ = [("p_max", C.c_int32), ("max_wave_frames", C.c_int32), ("waves_in_flight", C.c_int32),
                ("keep_llr", C.c_int32), ("arena_bytes", C.c_int64), ("max_M", C.c_int32), ("max_N", C.c_int32),
                ("max_ant", C.c_int32), ("light_work", C.c_int32)]


class zotfs_request(C.Structure):
    _fields_ = [("M", C.c_int32), ("N", C.c_int32), ("n_rx", C.c_int32), ("n_tx", C.c_int32), ("qam", C.c_int32),
                ("iters", C.c_int32), ("noise_var", C.c_float), ("theta", C.c_float), ("a_pilot", C.c_float),
                ("cg_eps", C.c_float), ("y_pilot", C.c_void_p), ("y_data", C.c_void_p), ("tag", C.c_uint64)]


class zotfs_completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("status", C.c_int32), ("n_lists", C.c_int32), ("arrival_ns", C.c_int64),
                ("admit_ns", C.c_int64), ("done_ns", C.c_int64), ("bits", C.c_void_p), ("llr", C.c_void_p),
                ("path_count", C.c_void_p), ("path_dk", C.c_void_p), ("path_dl", C.c_void_p), ("path_h", C.c_void_p)]


class zotfs_server_stats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("submitted", "admitted", "completed", "released", "pending", "waves",
                                         "arena_bytes", "arena_in_use", "arena_high_water", "rejected_too_large")]


_P = C.c_void_p
_I = C.c_int
# name -> (restype, argtypes); mirrors include/zotfs.h
SIGNATURES = {
    "zotfs_plan_create": (_I, [_I, _I, _I, _I, _I, _I, C.POINTER(_P)]),
    "zotfs_plan_set_options": (_I, [_P, C.POINTER(zotfs_options)]),
    "zotfs_plan_get_options": (_I, [_P, C.POINTER(zotfs_options)]),
    "zotfs_plan_destroy": (_I, [_P]),
    "zotfs_plan_set_tuning": (_I, [_P, C.POINTER(zotfs_tuning)]),
    "zotfs_plan_get_tuning": (_I, [_P, C.POINTER(zotfs_tuning)]),
    "zotfs_dzt": (_I, [_P, _P, _P, _I, _P]),
    "zotfs_estimate": (_I, [_P, _P, _P, _I, C.POINTER(zotfs_paths), _P]),
    "zotfs_ss_apply": (_I, [_P, C.POINTER(zotfs_paths), _P, _P, _I, _I, _P, _P]),
    "zotfs_equalize": (_I, [_P, _P, _I, C.POINTER(zotfs_paths), _P, _I, _P, _I, _P, _P]),
    "zotfs_equalize_mrc": (_I, [_P, _P, _I, C.POINTER(zotfs_paths), _I, _P, _P, _I, _P]),
    "zotfs_check_cg_ratio": (_I, [_P, _P, _P, _I, _P]),
    "zotfs_demap": (_I, [_P, _P, _P, _P, _P, _I, _P]),
    "zotfs_rx": (_I, [_P, _P, _P, _P, _P, _I, C.POINTER(zotfs_paths), _P, _P, _P, _P, _I, _P]),
    "zotfs_rx_plain": (_I, [_P, _P, _P, _P, _P, _I, C.POINTER(zotfs_paths), _P, _P, _P, _P, _I, _P]),
    "zotfs_rx_lists": (_I, [_P, _P, C.POINTER(zotfs_paths), _P, _I, _P, _I, _P, _P, _P, _P, _I, _P]),
    "zotfs_check_bounded_wait": (_I, [_I, C.c_uint32, _P, _P]),
    "zotfs_debug_fail_alloc": (_I, [_I]),
    "zotfs_equalize_static": (_I, [_I, _I, _I, _I, C.POINTER(zotfs_paths), _P, _P, _I, _P, _P, _I, _P]),
    "zotfs_batch_create": (_I, [C.POINTER(zotfs_frame_desc), _I, C.POINTER(zotfs_batch_opts), C.POINTER(_P)]),
    "zotfs_rx_batch": (_I, [_P, _P, _P]),
    "zotfs_batch_destroy": (_I, [_P]),
    "zotfs_batch_capture": (_I, [_P, _P, C.POINTER(_P)]),
    "zotfs_graph_launch": (_I, [_P, _P]),
    "zotfs_graph_destroy": (_I, [_P]),
    "zotfs_autotune": (_I, [C.POINTER(zotfs_frame_desc), _I, C.POINTER(zotfs_autotune_opts),
                            C.POINTER(zotfs_tuning_result), _I, C.POINTER(_I), _P]),
    "zotfs_server_create": (_I, [C.POINTER(zotfs_server_opts), C.POINTER(_P)]),
    "zotfs_server_submit": (_I, [_P, C.POINTER(zotfs_request), _I]),
    "zotfs_server_replay": (_I, [_P, C.POINTER(zotfs_request), C.POINTER(C.c_double), _I]),
    "zotfs_server_poll": (_I, [_P, C.POINTER(zotfs_completion), _I]),
    "zotfs_server_read": (_I, [_P, C.c_uint64, _P, _P, _P, _P, _P, _P]),
    "zotfs_server_release": (_I, [_P, C.c_uint64]),
    "zotfs_server_get_stats": (_I, [_P, C.POINTER(zotfs_server_stats)]),
    "zotfs_server_destroy": (_I, [_P]),
    "zotfs_last_error": (C.c_char_p, []),
    "zotfs_last_launch_count": (_I, []),
}

_lib = None


def lib():
    """Load libzotfs.so (built in-tree by paper_2604_02266_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status):
    """Raise ZotfsError for a non-OK status, with the library's thread-local message."""
    if status != OK:
        msg = lib().zotfs_last_error().decode(errors="replace")
        raise ZotfsError(status, msg)
    return status


def _mk(name):
    def call(*args):
        return getattr(lib(), name)(*args)
    call.__name__ = name
    call.__doc__ = f"Direct call of {name} (see include/zotfs.h)."
    return call


zotfs_plan_create = _mk("zotfs_plan_create")
zotfs_plan_set_options = _mk("zotfs_plan_set_options")
zotfs_plan_get_options = _mk("zotfs_plan_get_options")
zotfs_plan_destroy = _mk("zotfs_plan_destroy")
zotfs_plan_set_tuning = _mk("zotfs_plan_set_tuning")
zotfs_plan_get_tuning = _mk("zotfs_plan_get_tuning")
zotfs_dzt = _mk("zotfs_dzt")
zotfs_estimate = _mk("zotfs_estimate")
zotfs_ss_apply = _mk("zotfs_ss_apply")
zotfs_equalize = _mk("zotfs_equalize")
zotfs_equalize_mrc = _mk("zotfs_equalize_mrc")
zotfs_check_cg_ratio = _mk("zotfs_check_cg_ratio")
zotfs_demap = _mk("zotfs_demap")
zotfs_rx = _mk("zotfs_rx")
zotfs_rx_plain = _mk("zotfs_rx_plain")
zotfs_rx_lists = _mk("zotfs_rx_lists")
zotfs_check_bounded_wait = _mk("zotfs_check_bounded_wait")
zotfs_debug_fail_alloc = _mk("zotfs_debug_fail_alloc")
zotfs_equalize_static = _mk("zotfs_equalize_static")
zotfs_batch_create = _mk("zotfs_batch_create")
zotfs_rx_batch = _mk("zotfs_rx_batch")
zotfs_batch_destroy = _mk("zotfs_batch_destroy")
zotfs_batch_capture = _mk("zotfs_batch_capture")
zotfs_graph_launch = _mk("zotfs_graph_launch")
zotfs_graph_destroy = _mk("zotfs_graph_destroy")
zotfs_autotune = _mk("zotfs_autotune")
zotfs_server_create = _mk("zotfs_server_create")
zotfs_server_submit = _mk("zotfs_server_submit")
zotfs_server_replay = _mk("zotfs_server_replay")
zotfs_server_poll = _mk("zotfs_server_poll")
zotfs_server_read = _mk("zotfs_server_read")
zotfs_server_release = _mk("zotfs_server_release")
zotfs_server_get_stats = _mk("zotfs_server_get_stats")
zotfs_server_destroy = _mk("zotfs_server_destroy")
zotfs_last_error = _mk("zotfs_last_error")
zotfs_last_launch_count = _mk("zotfs_last_launch_count")
