"""The C-ABI library builds, loads and exports every function include/fsmi.h declares (CPU only: no
compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fsmi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"^\s*typedef\b.*$", "", src, flags=re.M)  # function-pointer types are not exports
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w \*]*?\b(fsmi_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1905_02238_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for fn in ("fsmi_eval_2d", "fsmi_eval_2d_sets", "fsmi_eval_beams", "fsmi_trace_2d", "fsmi_rle_encode_3d",
               "fsmi_eval_rle", "fsmi_eval_3d", "fsmi_workspace_size", "fsmi_device_status", "fsmi_status_str",
               "fsmi_version", "fsmi_set_schedule", "fsmi_get_schedule", "fsmi_autotune", "fsmi_schedule_candidates",
               "fsmi_prepare", "fsmi_capture_begin", "fsmi_capture_end", "fsmi_graph_launch", "fsmi_graph_destroy"):
        assert fn in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib_path):
    # functions that need no device: status strings, version, workspace sizing
    lib = ctypes.CDLL(lib_path)
    lib.fsmi_status_str.restype = ctypes.c_char_p
    assert lib.fsmi_status_str(0) == b"ok"
    assert lib.fsmi_status_str(5) == b"workspace too small"
    assert lib.fsmi_version() >= 100
    b = ctypes.c_size_t(0)
    lib.fsmi_workspace_size.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]
    assert lib.fsmi_workspace_size(2, 4096 * 3 + 1, None, ctypes.byref(b)) == 0
    assert b.value == 4 * 4
    # eval workspaces: the 256-byte work-queue counter, then (2D) 16 bytes of gains per map cell
    assert lib.fsmi_workspace_size(0, 100, None, ctypes.byref(b)) == 0 and b.value == 256 + 1600
    for fn in (1, 3, 4):
        assert lib.fsmi_workspace_size(fn, 100, None, ctypes.byref(b)) == 0 and b.value == 256
    assert lib.fsmi_workspace_size(9, 100, None, ctypes.byref(b)) == 1


def test_range_argument_is_checked_before_any_launch(lib_path):
    # a NaN range is an argument error, found on the host (no pointer is touched, nothing launched)
    lib = ctypes.CDLL(lib_path)
    p, i, f, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_longlong
    lib.fsmi_profiles_2d.argtypes = [p, i, i, p, i, p, i, f, p, ll, p, p]
    lib.fsmi_surrogate_predict.argtypes = [p, p, p, i, i, p, i, p, i, f, p, ll, p, p, ctypes.c_size_t, p]
    nan = float("nan")
    # with nothing to do these return ok for a finite range, so only the range check can fail them
    assert lib.fsmi_profiles_2d(None, 16, 16, None, 0, None, 1, 5.0, None, 0, None, None) == 0
    assert lib.fsmi_profiles_2d(None, 16, 16, None, 0, None, 1, nan, None, 0, None, None) == 1
    dummy = ctypes.c_void_p(16)  # never dereferenced: no beams
    assert lib.fsmi_surrogate_predict(dummy, dummy, None, 0, 0, None, 0, None, 0, 5.0, None, 0, dummy, None, 0,
                                      None) == 0
    assert lib.fsmi_surrogate_predict(dummy, dummy, None, 0, 0, None, 0, None, 0, nan, None, 0, dummy, None, 0,
                                      None) == 1


class _Sched(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("warps_per_block", "blocks_per_sm", "queue_chunk", "cell_runlen")]


def test_schedule_is_checked_per_family_and_thread_local(lib_path):
    import threading

    lib = ctypes.CDLL(lib_path)
    S = ctypes.POINTER(_Sched)
    lib.fsmi_set_schedule.argtypes = [ctypes.c_int, S]
    lib.fsmi_get_schedule.argtypes = [ctypes.c_int, S]

    def get(kind):
        s = _Sched()
        assert lib.fsmi_get_schedule(kind, ctypes.byref(s)) == 0
        return (s.warps_per_block, s.blocks_per_sm, s.queue_chunk, s.cell_runlen)

    for k in (0, 1):
        assert lib.fsmi_set_schedule(k, None) == 0
    assert get(0) == (4, 0, 1, 32) and get(1) == (2, 0, 4, 32)  # family defaults
    assert lib.fsmi_set_schedule(0, ctypes.byref(_Sched(8, 2, -1, 0))) == 0
    assert get(0) == (8, 2, -1, 32) and get(1) == (2, 0, 4, 32)  # the other family is untouched
    assert lib.fsmi_set_schedule(1, ctypes.byref(_Sched(0, 0, 0, 7))) == 0
    assert get(1) == (2, 0, 4, 7)
    for bad in (_Sched(9, 0, 0, 0), _Sched(-1, 0, 0, 0), _Sched(4, -1, 0, 0), _Sched(4, 0, -2, 0),
                _Sched(4, 0, 0, -3)):
        assert lib.fsmi_set_schedule(0, ctypes.byref(bad)) == 1
    assert lib.fsmi_set_schedule(2, None) == 1
    assert lib.fsmi_get_schedule(-1, ctypes.byref(_Sched())) == 1
    other = {}

    def peek():
        other["2d"] = get(0)

    t = threading.Thread(target=peek)
    t.start()
    t.join()
    assert other["2d"] == (4, 0, 1, 32)  # another thread still has the defaults
    assert get(0) == (8, 2, -1, 32)
    for k in (0, 1):
        assert lib.fsmi_set_schedule(k, None) == 0


def test_schedule_candidates(lib_path):
    lib = ctypes.CDLL(lib_path)
    arr = (_Sched * 64)()
    n = ctypes.c_int(0)
    lib.fsmi_schedule_candidates.argtypes = [ctypes.c_int, ctypes.POINTER(_Sched), ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_int)]
    assert lib.fsmi_schedule_candidates(0, arr, 64, ctypes.byref(n)) == 0 and n.value == 9
    assert {arr[i].warps_per_block for i in range(n.value)} == {2, 4, 8}
    assert {arr[i].queue_chunk for i in range(n.value)} == {1, 4, -1}
    assert lib.fsmi_schedule_candidates(1, arr, 64, ctypes.byref(n)) == 0 and n.value == 24
    assert {arr[i].cell_runlen for i in range(n.value)} == {16, 32}
    assert lib.fsmi_schedule_candidates(1, arr, 5, ctypes.byref(n)) == 0 and n.value == 5
    assert lib.fsmi_schedule_candidates(2, arr, 64, ctypes.byref(n)) == 1
