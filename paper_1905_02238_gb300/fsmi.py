"""Thin Python binding of libfsmi (include/fsmi.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module checks tensor
types, passes device pointers and the current torch stream, and raises on a non-OK status. There
is no CPU fallback: without a CUDA device or without the built library every call raises.

Inputs may be CUDA tensors (the device path) or CPU tensors, in which case they are copied to
the current device on the current stream (from pinned memory when the caller pinned them) and the
result is copied back; that is the end-to-end form of the same call.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

from . import build as _build

EXACT, APPROX, UNIFORM = 0, 1, 2
G_PDF, G_ERF = 0, 1
FLAG_FULL_SWEEP = 0x1
FN_EVAL_2D, FN_EVAL_BEAMS, FN_RLE_ENCODE_3D, FN_EVAL_RLE, FN_EVAL_3D = 0, 1, 2, 3, 4
STATUS_BEAM_OVERFLOW, STATUS_RUN_OVERFLOW, STATUS_BAD_BEAM = 0x1, 0x2, 0x4
MAX_RANGE_2D, MAX_CELLS, MAX_SAMPLES_3D = 1024.0, 2048, 1024

_lock = threading.Lock()
_lib = None


class FsmiError(RuntimeError):
    pass


class _CParams(ctypes.Structure):
    _fields_ = [
        ("variant", ctypes.c_int),
        ("sigma", ctypes.c_float),
        ("delta_occ", ctypes.c_float),
        ("delta_emp", ctypes.c_float),
        ("trunc_delta", ctypes.c_int),
        ("uniform_h", ctypes.c_int),
        ("max_range", ctypes.c_float),
        ("run_cap", ctypes.c_int),
        ("g_kernel", ctypes.c_int),
        ("e0_mode", ctypes.c_int),
        ("approx_reading", ctypes.c_int),
        ("flags", ctypes.c_int),
    ]


@dataclass
class Params:
    """fsmi_params: method parameters in cell units."""

    variant: int = EXACT
    sigma: float = 1.5
    delta_occ: float = 1.5
    delta_emp: float = 0.67
    trunc_delta: int = 3
    uniform_h: int = 2
    max_range: float = 64.0
    run_cap: int = 64
    g_kernel: int = G_PDF
    e0_mode: int = 0
    approx_reading: int = 0
    flags: int = 0

    def c(self) -> _CParams:
        return _CParams(int(self.variant), float(self.sigma), float(self.delta_occ), float(self.delta_emp),
                        int(self.trunc_delta), int(self.uniform_h), float(self.max_range), int(self.run_cap),
                        int(self.g_kernel), int(self.e0_mode), int(self.approx_reading), int(self.flags))


def library_path() -> str:
    return _build.LIB


def load():
    """Load libfsmi.so (built by __graft_entry__.build() or paper_1905_02238_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not torch.cuda.is_available():
            raise FsmiError("no CUDA device: libfsmi runs only on the GPU (there is no CPU fallback)")
        path = os.environ.get("FSMI_LIBRARY", _build.LIB)
        if not os.path.exists(path):
            raise FsmiError(f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(path)
        i, p, ll = ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong
        P = ctypes.POINTER(_CParams)
        sig = {
            "fsmi_eval_2d": [p, i, i, p, i, p, i, P, p, p, ctypes.c_size_t, p],
            "fsmi_eval_beams": [p, p, p, p, i, P, p, p],
            "fsmi_trace_2d": [i, i, p, i, p, i, ctypes.c_float, i, p, p, p, p],
            "fsmi_rle_encode_3d": [p, i, i, i, p, i, p, i, P, p, p, p, i, p, ctypes.c_size_t, p],
            "fsmi_eval_rle": [p, p, p, i, P, p, p],
            "fsmi_eval_3d": [p, i, i, i, p, i, p, i, P, p, p, p],
            "fsmi_workspace_size": [i, ll, P, ctypes.POINTER(ctypes.c_size_t)],
            "fsmi_device_status": [p, ctypes.POINTER(ctypes.c_int)],
            "fsmi_gauss_tail": [p, p, ll, p],
            "fsmi_rle_encode_3d_noalloc": [p, i, i, i, p, i, p, i, P, p, p, p, i, p],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.fsmi_status_str.restype = ctypes.c_char_p
        lib.fsmi_status_str.argtypes = [ctypes.c_int]
        lib.fsmi_last_cuda_error.restype = ctypes.c_int
        lib.fsmi_version.restype = ctypes.c_int
        _lib = lib
        return lib


def _raise(code: int, what: str):
    if code != 0:
        lib = load()
        msg = lib.fsmi_status_str(code).decode()
        if code == 3:
            msg += f" (cudaError {lib.fsmi_last_cuda_error()})"
        raise FsmiError(f"{what}: {msg}")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class _Marshal:
    """Moves CPU inputs to the device (non-blocking) and remembers to bring results back."""

    def __init__(self, *tensors):
        self.host = any(t is not None and not t.is_cuda for t in tensors)
        self.dev = torch.device("cuda", torch.cuda.current_device())

    def arg(self, t, dtype, name, ndim=None, last=None):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch.Tensor")
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        if ndim is not None and t.dim() != ndim:
            raise ValueError(f"{name} must have {ndim} dims, got shape {tuple(t.shape)}")
        if last is not None and t.shape[-1] != last:
            raise ValueError(f"{name} must have last dim {last}, got shape {tuple(t.shape)}")
        if not t.is_cuda:
            t = t.to(self.dev, non_blocking=True)
        elif t.device != self.dev:
            raise ValueError(f"{name} is on {t.device}, the current device is {self.dev}")
        return t.contiguous()

    def out(self, t):
        return t.to("cpu", non_blocking=False) if self.host else t


def eval_2d(grid: torch.Tensor, poses: torch.Tensor, dirs: torch.Tensor, prm: Params,
            out: torch.Tensor | None = None, ws: torch.Tensor | None = None) -> torch.Tensor:
    """fsmi_eval_2d: grid float32 [H, W]; poses int32 [P, 4]; dirs int32 [B, 2] -> float32 [P, B].
    ws: optional device workspace (uint8, >= workspace_size(FN_EVAL_2D, H*W) bytes) for per-cell
    gains; by default one is taken from torch's allocator. Pass an empty tensor to use none."""
    lib = load()
    m = _Marshal(grid, poses, dirs)
    g = m.arg(grid, torch.float32, "grid", 2)
    ps = m.arg(poses, torch.int32, "poses", 2, 4)
    ds = m.arg(dirs, torch.int32, "dirs", 2, 2)
    P, B = ps.shape[0], ds.shape[0]
    if out is None or m.host:
        out = torch.empty((P, B), dtype=torch.float32, device=m.dev)
    if ws is None:
        ws = torch.empty(16 * g.numel(), dtype=torch.uint8, device=m.dev)
    cp = prm.c()
    _raise(lib.fsmi_eval_2d(_ptr(g), g.shape[1], g.shape[0], _ptr(ps), P, _ptr(ds), B, ctypes.byref(cp),
                            _ptr(out), _ptr(ws) if ws.numel() else None, ws.numel() * ws.element_size(),
                            _stream()), "fsmi_eval_2d")
    return m.out(out)


def eval_beams(off, o, l, lend, prm: Params, out=None) -> torch.Tensor:
    """fsmi_eval_beams on CSR beams -> float32 [nbeams]."""
    lib = load()
    m = _Marshal(off, o, l, lend)
    off = m.arg(off, torch.int32, "off", 1)
    o = m.arg(o, torch.float32, "o", 1)
    l = m.arg(l, torch.float32, "l", 1)
    lend = m.arg(lend, torch.float32, "lend", 1)
    nb = off.shape[0] - 1
    if out is None or m.host:
        out = torch.empty(nb, dtype=torch.float32, device=m.dev)
    cp = prm.c()
    _raise(lib.fsmi_eval_beams(_ptr(off), _ptr(o), _ptr(l), _ptr(lend), nb, ctypes.byref(cp), _ptr(out), _stream()),
           "fsmi_eval_beams")
    return m.out(out)


def trace_2d(W: int, H: int, poses, dirs, max_range: float, cap: int):
    """fsmi_trace_2d -> (cells int32 [P*B, cap], l float32 [P*B, cap+1], n int32 [P*B])."""
    lib = load()
    m = _Marshal(poses, dirs)
    ps = m.arg(poses, torch.int32, "poses", 2, 4)
    ds = m.arg(dirs, torch.int32, "dirs", 2, 2)
    nb = ps.shape[0] * ds.shape[0]
    cells = torch.empty((nb, cap), dtype=torch.int32, device=m.dev)
    l = torch.empty((nb, cap + 1), dtype=torch.float32, device=m.dev)
    n = torch.empty(nb, dtype=torch.int32, device=m.dev)
    _raise(lib.fsmi_trace_2d(W, H, _ptr(ps), ps.shape[0], _ptr(ds), ds.shape[0], ctypes.c_float(max_range), cap,
                             _ptr(cells), _ptr(l), _ptr(n), _stream()), "fsmi_trace_2d")
    return m.out(cells), m.out(l), m.out(n)


def workspace_size(fn: int, nitems: int, prm: Params | None = None) -> int:
    lib = load()
    b = ctypes.c_size_t(0)
    cp = (prm or Params()).c()
    _raise(lib.fsmi_workspace_size(fn, nitems, ctypes.byref(cp), ctypes.byref(b)), "fsmi_workspace_size")
    return int(b.value)


def rle_encode_3d(vox, poses, dirs, prm: Params, capacity: int, ws: torch.Tensor | None = None):
    """fsmi_rle_encode_3d -> (run_off int32 [P*R+1], run_o float32 [capacity], run_len uint8 [capacity])."""
    lib = load()
    m = _Marshal(vox, poses, dirs)
    v = m.arg(vox, torch.float32, "vox", 3)
    ps = m.arg(poses, torch.int32, "poses", 2, 12)
    ds = m.arg(dirs, torch.int32, "dirs", 2, 3)
    Z, Y, X = v.shape
    P, R = ps.shape[0], ds.shape[0]
    off = torch.empty(P * R + 1, dtype=torch.int32, device=m.dev)
    ro = torch.empty(max(capacity, 1), dtype=torch.float32, device=m.dev)
    rl = torch.empty(max(capacity, 1), dtype=torch.uint8, device=m.dev)
    need = workspace_size(FN_RLE_ENCODE_3D, P * R, prm)
    if ws is None:
        ws = torch.empty(max(need, 4), dtype=torch.uint8, device=m.dev)
    cp = prm.c()
    _raise(lib.fsmi_rle_encode_3d(_ptr(v), X, Y, Z, _ptr(ps), P, _ptr(ds), R, ctypes.byref(cp), _ptr(off), _ptr(ro),
                                  _ptr(rl), capacity, _ptr(ws), ws.numel() * ws.element_size(), _stream()),
           "fsmi_rle_encode_3d")
    return m.out(off), m.out(ro[:capacity]), m.out(rl[:capacity])


NOALLOC_MAX_RAYS = 4096 * 4096


def rle_encode_3d_noalloc(vox, poses, dirs, prm: Params, capacity: int):
    """fsmi_rle_encode_3d_noalloc: the encoder for callers that cannot allocate device memory; the
    offset scan uses a library-owned array instead of a workspace. Calls that overlap on the GPU
    race; the first call on a device should precede any stream capture."""
    lib = load()
    m = _Marshal(vox, poses, dirs)
    v = m.arg(vox, torch.float32, "vox", 3)
    ps = m.arg(poses, torch.int32, "poses", 2, 12)
    ds = m.arg(dirs, torch.int32, "dirs", 2, 3)
    Z, Y, X = v.shape
    P, R = ps.shape[0], ds.shape[0]
    off = torch.empty(P * R + 1, dtype=torch.int32, device=m.dev)
    ro = torch.empty(max(capacity, 1), dtype=torch.float32, device=m.dev)
    rl = torch.empty(max(capacity, 1), dtype=torch.uint8, device=m.dev)
    cp = prm.c()
    _raise(lib.fsmi_rle_encode_3d_noalloc(_ptr(v), X, Y, Z, _ptr(ps), P, _ptr(ds), R, ctypes.byref(cp), _ptr(off),
                                          _ptr(ro), _ptr(rl), capacity, _stream()), "fsmi_rle_encode_3d_noalloc")
    return m.out(off), m.out(ro[:capacity]), m.out(rl[:capacity])


def eval_rle(off, run_o, run_len, prm: Params, out=None) -> torch.Tensor:
    """fsmi_eval_rle on CSR runs -> float32 [nrays]."""
    lib = load()
    m = _Marshal(off, run_o, run_len)
    off = m.arg(off, torch.int32, "run_off", 1)
    ro = m.arg(run_o, torch.float32, "run_o", 1)
    rl = m.arg(run_len, torch.uint8, "run_len", 1)
    nr = off.shape[0] - 1
    if out is None or m.host:
        out = torch.empty(nr, dtype=torch.float32, device=m.dev)
    cp = prm.c()
    _raise(lib.fsmi_eval_rle(_ptr(off), _ptr(ro), _ptr(rl), nr, ctypes.byref(cp), _ptr(out), _stream()), "fsmi_eval_rle")
    return m.out(out)


def eval_3d(vox, poses, dirs, prm: Params, out=None, with_runs: bool = False):
    """fsmi_eval_3d (fused sample + encode + RLE variant) -> float32 [P, R] (and run counts)."""
    lib = load()
    m = _Marshal(vox, poses, dirs)
    v = m.arg(vox, torch.float32, "vox", 3)
    ps = m.arg(poses, torch.int32, "poses", 2, 12)
    ds = m.arg(dirs, torch.int32, "dirs", 2, 3)
    Z, Y, X = v.shape
    P, R = ps.shape[0], ds.shape[0]
    if out is None or m.host:
        out = torch.empty((P, R), dtype=torch.float32, device=m.dev)
    nr = torch.empty((P, R), dtype=torch.int32, device=m.dev) if with_runs else None
    cp = prm.c()
    _raise(lib.fsmi_eval_3d(_ptr(v), X, Y, Z, _ptr(ps), P, _ptr(ds), R, ctypes.byref(cp), _ptr(out), _ptr(nr),
                            _stream()), "fsmi_eval_3d")
    if with_runs:
        return m.out(out), m.out(nr)
    return m.out(out)


def gauss_tail(s: torch.Tensor) -> torch.Tensor:
    """fsmi_gauss_tail: 0.5 * erfc(s / sqrt(log2 e)) elementwise (float32 CUDA tensor)."""
    lib = load()
    m = _Marshal(s)
    s = m.arg(s, torch.float32, "s")
    out = torch.empty_like(s)
    _raise(lib.fsmi_gauss_tail(_ptr(s), _ptr(out), s.numel(), _stream()), "fsmi_gauss_tail")
    return m.out(out)


def device_status() -> int:
    """Reads and clears the current device's status word (waits for the current stream)."""
    lib = load()
    v = ctypes.c_int(0)
    _raise(lib.fsmi_device_status(_stream(), ctypes.byref(v)), "fsmi_device_status")
    return int(v.value)
