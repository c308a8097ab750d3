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
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w \*]*?\b(fsmi_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1905_02238_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for fn in ("fsmi_eval_2d", "fsmi_eval_beams", "fsmi_trace_2d", "fsmi_rle_encode_3d", "fsmi_eval_rle",
               "fsmi_eval_3d", "fsmi_workspace_size", "fsmi_device_status", "fsmi_status_str", "fsmi_version"):
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
    assert lib.fsmi_workspace_size(0, 100, None, ctypes.byref(b)) == 0 and b.value == 1600
    assert lib.fsmi_workspace_size(3, 100, None, ctypes.byref(b)) == 0 and b.value == 0
    assert lib.fsmi_workspace_size(9, 100, None, ctypes.byref(b)) == 1


def test_binding_fails_loudly_without_gpu():
    import torch

    from paper_1905_02238_gb300 import fsmi

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(fsmi.FsmiError):
        fsmi.load()
