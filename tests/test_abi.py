"""The C ABI library builds, loads and exports every function include/zotfs.h declares, and
the Python binding covers each of them (no GPU needed: nothing here calls into CUDA)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "zotfs.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(zotfs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2604_02266_gb300 import build
    try:
        return build.build()
    except RuntimeError as e:  # no nvcc on this machine
        if "nvcc not found" in str(e):
            pytest.skip(str(e))
        raise


def test_header_declares_the_pipeline():
    names = _declared_functions()
    for required in ("zotfs_plan_create", "zotfs_plan_destroy", "zotfs_dzt", "zotfs_estimate", "zotfs_ss_apply",
                     "zotfs_equalize", "zotfs_demap", "zotfs_rx", "zotfs_rx_plain", "zotfs_batch_create",
                     "zotfs_rx_batch", "zotfs_batch_destroy", "zotfs_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_header(libpath):
    from paper_2604_02266_gb300 import _zotfs
    assert set(_zotfs.SIGNATURES) == set(_declared_functions())
    _zotfs.lib()  # loads and binds every signature


def test_struct_layouts_match_header_sizes(libpath):
    """The ctypes mirrors have the sizes the C compiler gives the header's structs."""
    from paper_2604_02266_gb300 import _zotfs as Z
    # all fields are 4-byte ints/floats or 8-byte pointers in declaration order
    assert ctypes.sizeof(Z.zotfs_options) == 40
    assert ctypes.sizeof(Z.zotfs_paths) == 5 * 8 + 8
    assert ctypes.sizeof(Z.zotfs_tuning) == 20
    assert ctypes.sizeof(Z.zotfs_frame_desc) == 16 * 4 + 9 * 8  # 16 scalars, 9 pointers
    assert ctypes.sizeof(Z.zotfs_request) == 10 * 4 + 3 * 8  # 10 scalars, 2 pointers, the tag
    assert ctypes.sizeof(Z.zotfs_batch_opts) == 4 * 4 + 8 + 4 + 4  # ..., max_sms, cluster
    assert ctypes.sizeof(Z.zotfs_autotune_opts) == 12
    assert ctypes.sizeof(Z.zotfs_tuning_entry) == 4 * 4 + 20
    assert ctypes.sizeof(Z.zotfs_tuning_result) == 4 * 4 + 20 + 5 * 4


def test_argument_errors_without_gpu(libpath):
    """Argument validation happens before any CUDA call."""
    from paper_2604_02266_gb300 import _zotfs as Z
    h = ctypes.c_void_p()
    assert Z.zotfs_plan_create(48, 32, 1, 1, 0, 16, ctypes.byref(h)) == Z.EINVAL  # M not a power of two
    assert b"power of two" in Z.zotfs_last_error()
    assert Z.zotfs_plan_create(64, 32, 1, 1, 0, 8, ctypes.byref(h)) == Z.EINVAL   # qam
    assert Z.zotfs_plan_create(64, 32, 5, 1, 0, 16, ctypes.byref(h)) == Z.EINVAL  # antennas
    assert Z.zotfs_plan_create(256, 128, 1, 1, 0, 16, ctypes.byref(h)) == Z.EINVAL  # N too large
    assert h.value is None
    assert Z.zotfs_dzt(None, None, None, 1, None) == Z.EINVAL
    assert Z.zotfs_rx_batch(None, None, None) == Z.EINVAL
    d = (Z.zotfs_frame_desc * 1)()
    d[0].M, d[0].N, d[0].n_rx, d[0].n_tx, d[0].qam = 64, 32, 1, 1, 5
    out = ctypes.c_void_p()
    assert Z.zotfs_batch_create(d, 1, None, ctypes.byref(out)) == Z.EINVAL
    assert b"qam" in Z.zotfs_last_error()
    assert Z.zotfs_batch_capture(None, None, ctypes.byref(out)) == Z.EINVAL
    assert Z.zotfs_graph_launch(None, None) == Z.EINVAL
    assert Z.zotfs_graph_destroy(None) == Z.OK
    n = ctypes.c_int(7)
    assert Z.zotfs_autotune(d, 1, None, None, 0, None, None) == Z.EINVAL  # n_out NULL
    assert Z.zotfs_autotune(d, 1, None, None, 1, ctypes.byref(n), None) == Z.EINVAL  # out NULL
    assert n.value == 0
    bad = Z.zotfs_autotune_opts(-1, 0, 0)
    res = (Z.zotfs_tuning_result * 1)()
    assert Z.zotfs_autotune(d, 1, ctypes.byref(bad), res, 1, ctypes.byref(n), None) == Z.EINVAL


def _declared_arity():
    """Number of parameters of each function declared in the header."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(zotfs_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_arity_matches_header():
    """Each ctypes signature has as many arguments as the header's prototype."""
    from paper_2604_02266_gb300 import _zotfs
    arity = _declared_arity()
    assert set(arity) == set(_zotfs.SIGNATURES)
    wrong = {n: (len(args), arity[n]) for n, (_, args) in _zotfs.SIGNATURES.items() if len(args) != arity[n]}
    assert not wrong, wrong


def test_newer_entry_points_validate_without_gpu(libpath):
    """zotfs_rx_lists, zotfs_check_bounded_wait and zotfs_server_create reject bad arguments
    with ZOTFS_EINVAL before any CUDA call."""
    from paper_2604_02266_gb300 import _zotfs as Z
    st = ctypes.c_int32(-99)
    assert Z.zotfs_check_bounded_wait(2, 100, ctypes.byref(st), None) == Z.EINVAL
    assert b"which" in Z.zotfs_last_error()
    assert Z.zotfs_check_bounded_wait(-1, 100, ctypes.byref(st), None) == Z.EINVAL
    assert Z.zotfs_check_bounded_wait(0, 0, ctypes.byref(st), None) == Z.EINVAL
    assert Z.zotfs_check_bounded_wait(1, (1 << 24) + 1, ctypes.byref(st), None) == Z.EINVAL
    assert b"max_polls" in Z.zotfs_last_error()
    assert Z.zotfs_check_bounded_wait(0, 100, None, None) == Z.EINVAL
    assert st.value == -99  # nothing was written
    assert Z.zotfs_debug_fail_alloc(-2) == Z.EINVAL
    assert Z.zotfs_debug_fail_alloc(3) == Z.OK and Z.zotfs_debug_fail_alloc(-1) == Z.OK
    assert Z.zotfs_rx_lists(None, None, None, None, 1, None, 10, None, None, None, None, 1, None) == Z.EINVAL
    assert b"plan" in Z.zotfs_last_error()
    out = ctypes.c_void_p(1)
    assert Z.zotfs_server_create(None, ctypes.byref(out)) == Z.EINVAL
    good = dict(p_max=64, max_wave_frames=256, waves_in_flight=4, keep_llr=0, arena_bytes=1 << 20, max_M=64,
                max_N=32, max_ant=1, light_work=0)
    for key, bad in (("p_max", 0), ("p_max", 257), ("max_wave_frames", 4097), ("waves_in_flight", 17),
                     ("arena_bytes", 1024), ("max_M", 48), ("max_M", 512), ("max_N", 128), ("max_ant", 5),
                     ("light_work", -1)):
        o = Z.zotfs_server_opts(**{**good, key: bad})
        assert Z.zotfs_server_create(ctypes.byref(o), ctypes.byref(out)) == Z.EINVAL, key
        assert b"out of range" in Z.zotfs_last_error(), key
        assert out.value is None, key


def test_tuning_file_round_trip(tmp_path, libpath):
    """Autotuner results persist as JSON and load back as Batch(tuning=...) entries; a file of
    another format is refused."""
    import json
    from paper_2604_02266_gb300 import load_tuning, save_tuning
    res = [{"M": 64, "N": 32, "n_rx": 1, "n_tx": 1, "threads_per_frame": 256, "fft_radix": 4, "ctas_per_sm": 2,
            "cluster": 0, "frames_per_cta": 2, "sm_ms_per_frame": 0.08, "ms_best": 0.5, "ms_default": 0.6,
            "n_candidates": 9, "n_frames": 1024},
           {"M": 128, "N": 64, "n_rx": 4, "n_tx": 4, "threads_per_frame": 512, "fft_radix": 2, "ctas_per_sm": 1,
            "cluster": 4, "sm_ms_per_frame": 9.5, "ms_best": 17.0, "ms_default": 17.7, "n_candidates": 6,
            "n_frames": 256}]
    path = tmp_path / "tuning.json"
    save_tuning(str(path), res, "GB300")
    doc = json.loads(path.read_text())
    assert doc["format"] == "zotfs-tuning-1" and doc["device"] == "GB300" and len(doc["entries"]) == 2
    assert load_tuning(str(path)) == [
        ((64, 32, 1, 1), {"threads_per_frame": 256, "fft_radix": 4, "ctas_per_sm": 2, "cluster": 0, "frames_per_cta": 2}),
        ((128, 64, 4, 4), {"threads_per_frame": 512, "fft_radix": 2, "ctas_per_sm": 1, "cluster": 4,
                           "frames_per_cta": 0})]  # files written before the field existed read as 0
    other = tmp_path / "other.json"
    other.write_text(json.dumps({"format": "something-else", "entries": []}))
    with pytest.raises(ValueError):
        load_tuning(str(other))
