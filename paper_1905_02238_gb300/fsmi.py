"""Thin Python binding of libfsmi (include/fsmi.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module checks tensor
types, passes device pointers and the current torch stream, and raises on a non-OK status. There
is no CPU fallback: without a CUDA device or without the built library every call raises.

Inputs may be CUDA tensors (the device path) or CPU tensors, in which case they are copied to
the current device on the current stream (from pinned memory when the caller pinned them) and the
result is copied back; that is the end-to-end form of the same call.

Inside a CUDA graph capture (torch's or the library's own, `Graph`) nothing may be allocated:
pass device inputs and a preallocated `out`; a call without `ws` then runs without a workspace.
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
FLAG_FULL_WINDOW = 0x2
FN_EVAL_2D, FN_EVAL_BEAMS, FN_RLE_ENCODE_3D, FN_EVAL_RLE, FN_EVAL_3D, FN_UPDATE_MAP_2D = 0, 1, 2, 3, 4, 5
QUEUE_BYTES = 256
SURR_L, SURR_NPARAMS = 256, 269089
KIND_2D, KIND_RLE = 0, 1
STATUS_BEAM_OVERFLOW, STATUS_RUN_OVERFLOW, STATUS_BAD_BEAM, STATUS_TIMEOUT = 0x1, 0x2, 0x4, 0x10
MAX_RANGE_2D, MAX_CELLS, MAX_SAMPLES_3D = 1024.0, 2048, 1024

_lock = threading.Lock()
_lib = None
_TUNE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)


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


class _CSchedule(ctypes.Structure):
    _fields_ = [
        ("warps_per_block", ctypes.c_int),
        ("blocks_per_sm", ctypes.c_int),
        ("queue_chunk", ctypes.c_int),
        ("cell_runlen", ctypes.c_int),
    ]


@dataclass(frozen=True)
class Schedule:
    """fsmi_schedule: warps per block, resident-block cap, work-queue chunk (-1 = static), RLE
    cell-form threshold. Zeros select the family's defaults."""

    warps_per_block: int = 0
    blocks_per_sm: int = 0
    queue_chunk: int = 0
    cell_runlen: int = 0

    def c(self) -> _CSchedule:
        return _CSchedule(self.warps_per_block, self.blocks_per_sm, self.queue_chunk, self.cell_runlen)

    @staticmethod
    def of(c: _CSchedule) -> "Schedule":
        return Schedule(c.warps_per_block, c.blocks_per_sm, c.queue_chunk, c.cell_runlen)


SET_2D, SET_3D = 0, 1
# fsmi_set as 10 int32 words: kind, pose_offset, npose, dir_offset, ndir, max_range (float bits),
# volume, reserved, out_offset (int64, low word first); fsmi_volume as 6: pointer (2), X, Y, Z, 0
SET_WORDS, VOLUME_WORDS = 10, 6

# fsmi_set_2d as 8 int32 words: pose_offset, npose, dir_offset, nbeam, max_range (float bits),
# reserved, beam_offset (int64, little-endian low word first)
SET_2D_WORDS = 8


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
        sz = ctypes.c_size_t
        S = ctypes.POINTER(_CSchedule)
        sig = {
            "fsmi_eval_2d": [p, i, i, p, i, p, i, P, p, p, sz, p],
            "fsmi_eval_2d_sets": [p, i, i, p, i, p, i, p, i, ll, P, p, p, sz, p],
            "fsmi_eval_beams": [p, p, p, p, i, P, p, p, sz, p],
            "fsmi_trace_2d": [i, i, p, i, p, i, ctypes.c_float, i, p, p, p, p],
            "fsmi_rle_encode_3d": [p, i, i, i, p, i, p, i, P, p, p, p, i, p, ctypes.c_size_t, p],
            "fsmi_eval_rle": [p, p, p, i, P, p, p, sz, p],
            "fsmi_eval_3d": [p, i, i, i, p, i, p, i, P, p, p, p, sz, p],
            "fsmi_set_schedule": [i, S],
            "fsmi_get_schedule": [i, S],
            "fsmi_schedule_candidates": [i, S, i, ctypes.POINTER(ctypes.c_int)],
            "fsmi_autotune": [i, _TUNE_FN, p, S, i, i, p, S, ctypes.POINTER(ctypes.c_float)],
            "fsmi_prepare": [],
            "fsmi_capture_begin": [p],
            "fsmi_capture_end": [p, ctypes.POINTER(p)],
            "fsmi_graph_launch": [p, p],
            "fsmi_graph_destroy": [p],
            "fsmi_workspace_size": [i, ll, P, ctypes.POINTER(ctypes.c_size_t)],
            "fsmi_trajectory_workspace_size": [i, i, i, ctypes.POINTER(ctypes.c_size_t)],
            "fsmi_eval_trajectories_2d": [p, i, i, p, i, p, i, p, i, P, p, p, p, p, sz, p],
            "fsmi_best_trajectory": [p, p, i, p, i, p, p, p],
            "fsmi_scan_sums": [p, ll, i, p, p],
            "fsmi_update_map_2d": [p, i, i, p, i, p, i, p, P, p, sz, p],
            "fsmi_profiles_2d": [p, i, i, p, i, p, i, ctypes.c_float, p, ll, p, p],
            "fsmi_eval_mixed": [p, i, i, p, i, p, i, P, p, i, p, i, p, i, P, p, i, ll, p, p, p, sz, p],
            "fsmi_surrogate_workspace_size": [i, ll, ctypes.POINTER(ctypes.c_size_t)],
            "fsmi_surrogate_loss_grad": [p, p, p, p, i, p, p, p, p, sz, p],
            "fsmi_surrogate_adam": [p, p, p, p, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, i, p,
                                    p],
            "fsmi_surrogate_cast": [p, p, p],
            "fsmi_surrogate_predict": [p, p, p, i, i, p, i, p, i, ctypes.c_float, p, ll, p, p, sz, p],
            "fsmi_topk": [p, i, i, p, p],
            "fsmi_gather_rows": [p, ll, i, p, i, p, p],
            "fsmi_device_status": [p, ctypes.POINTER(ctypes.c_int)],
            "fsmi_gauss_tail": [p, p, ll, p],
            "fsmi_rle_encode_3d_noalloc": [p, i, i, i, p, i, p, i, P, p, p, p, i, p],
            "fsmi_probe": [i, ll, p, sz, p],
            "fsmi_probe_threads": [i],
            "fsmi_set_wait_limit": [ll],
            "fsmi_mixed_workspace_size": [ll, i, ctypes.POINTER(ctypes.c_size_t)],
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


def _capturing() -> bool:
    return torch.cuda.is_current_stream_capturing()


def _ws_args(ws):
    """(pointer, bytes) of an optional workspace tensor (None or empty = none)."""
    if ws is None or ws.numel() == 0:
        return None, 0
    if not ws.is_cuda:
        raise ValueError("ws must be a CUDA tensor")
    return _ptr(ws), ws.numel() * ws.element_size()


def _default_ws(nbytes: int, dev):
    """A fresh workspace from torch's allocator, or none inside a graph capture."""
    if _capturing():
        return None
    return torch.empty(nbytes, dtype=torch.uint8, device=dev)


def _out(out, shape, m):
    if out is None or m.host:
        if _capturing():
            raise FsmiError("inside a graph capture pass a preallocated device `out`")
        out = torch.empty(shape, dtype=torch.float32, device=m.dev)
    return out


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
    ws: optional device workspace (uint8, 16-byte aligned; workspace_size(FN_EVAL_2D, H*W) bytes
    hold the work-queue counter and the per-cell gains); by default one is taken from torch's
    allocator. Pass an empty tensor to use none."""
    lib = load()
    m = _Marshal(grid, poses, dirs)
    g = m.arg(grid, torch.float32, "grid", 2)
    ps = m.arg(poses, torch.int32, "poses", 2, 4)
    ds = m.arg(dirs, torch.int32, "dirs", 2, 2)
    P, B = ps.shape[0], ds.shape[0]
    out = _out(out, (P, B), m)
    if ws is None:
        ws = _default_ws(workspace_size(FN_EVAL_2D, g.numel()), m.dev)
    wp, wb = _ws_args(ws)
    cp = prm.c()
    _raise(lib.fsmi_eval_2d(_ptr(g), g.shape[1], g.shape[0], _ptr(ps), P, _ptr(ds), B, ctypes.byref(cp),
                            _ptr(out), wp, wb, _stream()), "fsmi_eval_2d")
    return m.out(out)


class Pipeline2D:
    """Consecutive fsmi_eval_2d calls on host data with their copies overlapped: submit() copies its
    host inputs (pinned, for the copies to be asynchronous) into one of two device buffer sets on a
    copy stream, evaluates them on a compute stream once they have landed, and copies the result
    into the given host tensor (pinned as well); the next submit's input copies then run while this
    evaluation does. The host tensors must stay alive and unchanged until wait(). The results are
    the floats eval_2d returns. wait() returns when every submitted result is on the host. Shapes
    are fixed at construction: grid [H, W], poses [P, 4], dirs [B, 2]."""

    def __init__(self, prm: Params, W: int, H: int, P: int, B: int):
        load()
        dev = torch.device("cuda", torch.cuda.current_device())
        self.prm = prm
        self.copy = torch.cuda.Stream(dev)
        self.comp = torch.cuda.Stream(dev)
        self.bufs = [(torch.empty((H, W), dtype=torch.float32, device=dev),
                      torch.empty((P, 4), dtype=torch.int32, device=dev),
                      torch.empty((B, 2), dtype=torch.int32, device=dev),
                      torch.empty((P, B), dtype=torch.float32, device=dev)) for _ in range(2)]
        self.ws = torch.empty(workspace_size(FN_EVAL_2D, W * H), dtype=torch.uint8, device=dev)
        self.free = [None, None]  # per buffer set: the event after which its last evaluation is done
        self.k = 0

    def submit(self, grid: torch.Tensor, poses: torch.Tensor, dirs: torch.Tensor, out: torch.Tensor) -> torch.Tensor:
        for t, name in ((grid, "grid"), (poses, "poses"), (dirs, "dirs"), (out, "out")):
            if t.is_cuda:
                raise ValueError(f"{name} must be a host tensor")
        g, ps, ds, o = self.bufs[self.k]
        if out.shape != o.shape or out.dtype != torch.float32:
            raise ValueError(f"out must be float32 {tuple(o.shape)}")
        with torch.cuda.stream(self.copy):
            if self.free[self.k] is not None:
                self.copy.wait_event(self.free[self.k])  # the evaluation that last read these buffers
            g.copy_(grid, non_blocking=True)
            ps.copy_(poses, non_blocking=True)
            ds.copy_(dirs, non_blocking=True)
            landed = torch.cuda.Event()
            landed.record(self.copy)
        with torch.cuda.stream(self.comp):
            self.comp.wait_event(landed)
            eval_2d(g, ps, ds, self.prm, out=o, ws=self.ws)
            out.copy_(o, non_blocking=True)
            done = torch.cuda.Event()
            done.record(self.comp)
        self.free[self.k] = done
        self.k ^= 1
        return out

    def wait(self) -> None:
        self.comp.synchronize()


def make_sets_2d(sets, device=None):
    """Packs candidate-set descriptors [(pose_offset, npose, dir_offset, nbeam, max_range), ...]
    into the fsmi_set_2d layout (int32 [nsets, 8] on `device`, consecutive output blocks in list
    order). Returns (tensor, total beams)."""
    import struct
    words, off = [], 0
    for po, npose, do, nbeam, rng in sets:
        fbits = struct.unpack("<i", struct.pack("<f", float(rng)))[0]
        lo, hi = struct.unpack("<ii", struct.pack("<q", off))
        words.append([int(po), int(npose), int(do), int(nbeam), fbits, 0, lo, hi])
        off += int(npose) * int(nbeam)
    t = torch.tensor(words, dtype=torch.int32).reshape(len(words), SET_2D_WORDS)
    return (t.to(device) if device is not None else t), off


def eval_2d_sets(grid, poses, dirs, sets, nbeams: int, prm: Params, out=None, ws=None) -> torch.Tensor:
    """fsmi_eval_2d_sets: several candidate sets (own poses, beams and range each) in one launch.
    sets: int32 [nsets, 8] from make_sets_2d; nbeams its total -> float32 [nbeams]."""
    lib = load()
    m = _Marshal(grid, poses, dirs, sets)
    g = m.arg(grid, torch.float32, "grid", 2)
    ps = m.arg(poses, torch.int32, "poses", 2, 4)
    ds = m.arg(dirs, torch.int32, "dirs", 2, 2)
    st = m.arg(sets, torch.int32, "sets", 2, SET_2D_WORDS)
    out = _out(out, (nbeams,), m)
    if ws is None:
        ws = _default_ws(workspace_size(FN_EVAL_2D, g.numel()), m.dev)
    wp, wb = _ws_args(ws)
    cp = prm.c()
    _raise(lib.fsmi_eval_2d_sets(_ptr(g), g.shape[1], g.shape[0], _ptr(ps), ps.shape[0], _ptr(ds), ds.shape[0],
                                 _ptr(st), st.shape[0], nbeams, ctypes.byref(cp), _ptr(out), wp, wb, _stream()),
           "fsmi_eval_2d_sets")
    return m.out(out)


def trajectory_workspace_size(W: int, H: int, T: int) -> int:
    lib = load()
    b = ctypes.c_size_t(0)
    _raise(lib.fsmi_trajectory_workspace_size(W, H, T, ctypes.byref(b)), "fsmi_trajectory_workspace_size")
    return int(b.value)


def eval_trajectories_2d(grid, poses, traj_off, dirs, prm: Params, ws=None, out=None):
    """fsmi_eval_trajectories_2d: MI along T trajectories (states = poses in CSR order traj_off
    int32 [T+1]); cells counted at an earlier state add nothing later (Section 2.4).
    Returns (beam_mi [P, B], state_mi [P], traj_mi [T]); `out` may pass those three tensors."""
    lib = load()
    m = _Marshal(grid, poses, traj_off, dirs)
    g = m.arg(grid, torch.float32, "grid", 2)
    ps = m.arg(poses, torch.int32, "poses", 2, 4)
    to = m.arg(traj_off, torch.int32, "traj_off", 1)
    ds = m.arg(dirs, torch.int32, "dirs", 2, 2)
    P, B, T = ps.shape[0], ds.shape[0], to.shape[0] - 1
    if out is None or m.host:
        if _capturing():
            raise FsmiError("inside a graph capture pass preallocated outputs")
        out = (torch.empty((P, B), dtype=torch.float32, device=m.dev), torch.empty(P, dtype=torch.float32, device=m.dev),
               torch.empty(T, dtype=torch.float32, device=m.dev))
    beam, state, traj = out
    if ws is None:
        if _capturing():
            raise FsmiError("inside a graph capture pass a preallocated workspace")
        ws = torch.empty(trajectory_workspace_size(g.shape[1], g.shape[0], T), dtype=torch.uint8, device=m.dev)
    wp, wb = _ws_args(ws)
    cp = prm.c()
    _raise(lib.fsmi_eval_trajectories_2d(_ptr(g), g.shape[1], g.shape[0], _ptr(ps), P, _ptr(to), T, _ptr(ds), B,
                                         ctypes.byref(cp), _ptr(beam), _ptr(state), _ptr(traj), wp, wb, _stream()),
           "fsmi_eval_trajectories_2d")
    return m.out(beam), m.out(state), m.out(traj)


def best_trajectory(traj_mi, poses, traj_off):
    """fsmi_best_trajectory -> (ratio float32 [T] = MI per travel distance, best index int)."""
    lib = load()
    m = _Marshal(traj_mi, poses, traj_off)
    tm = m.arg(traj_mi, torch.float32, "traj_mi", 1)
    ps = m.arg(poses, torch.int32, "poses", 2, 4)
    to = m.arg(traj_off, torch.int32, "traj_off", 1)
    T = tm.shape[0]
    ratio = torch.empty(T, dtype=torch.float32, device=m.dev)
    best = torch.empty(1, dtype=torch.int32, device=m.dev)
    _raise(lib.fsmi_best_trajectory(_ptr(tm), _ptr(ps), ps.shape[0], _ptr(to), T, _ptr(ratio), _ptr(best), _stream()),
           "fsmi_best_trajectory")
    return m.out(ratio), int(best.item())


def scan_sums_into(beam_mi, out) -> torch.Tensor:
    """fsmi_scan_sums into a preallocated device tensor out [P]."""
    return scan_sums(beam_mi, out=out)


def scan_sums(beam_mi, out=None) -> torch.Tensor:
    """fsmi_scan_sums: float32 [P, B] beam MI -> [P] scan MI per pose."""
    lib = load()
    m = _Marshal(beam_mi)
    b = m.arg(beam_mi, torch.float32, "beam_mi", 2)
    out = _out(out, (b.shape[0],), m)
    _raise(lib.fsmi_scan_sums(_ptr(b), b.shape[0], b.shape[1], _ptr(out), _stream()), "fsmi_scan_sums")
    return m.out(out)


def update_map_2d(grid: torch.Tensor, poses, dirs, ranges, prm: Params, ws=None) -> torch.Tensor:
    """fsmi_update_map_2d: Bayesian update (eq. 1) of `grid` (float32 CUDA tensor, in place) by
    measured ranges float32 [P, B]. Returns grid."""
    lib = load()
    if not (isinstance(grid, torch.Tensor) and grid.is_cuda and grid.dtype == torch.float32 and grid.dim() == 2
            and grid.is_contiguous()):
        raise TypeError("grid must be a contiguous float32 CUDA tensor [H, W] (updated in place)")
    m = _Marshal(poses, dirs, ranges)
    ps = m.arg(poses, torch.int32, "poses", 2, 4)
    ds = m.arg(dirs, torch.int32, "dirs", 2, 2)
    rg = m.arg(ranges, torch.float32, "ranges", 2)
    if tuple(rg.shape) != (ps.shape[0], ds.shape[0]):
        raise ValueError(f"ranges must be [P, B] = [{ps.shape[0]}, {ds.shape[0]}], got {tuple(rg.shape)}")
    if ws is None:
        if _capturing():
            raise FsmiError("inside a graph capture pass a preallocated workspace")
        ws = torch.empty(workspace_size(FN_UPDATE_MAP_2D, grid.numel()), dtype=torch.uint8, device=grid.device)
    wp, wb = _ws_args(ws)
    cp = prm.c()
    _raise(lib.fsmi_update_map_2d(_ptr(grid), grid.shape[1], grid.shape[0], _ptr(ps), ps.shape[0], _ptr(ds),
                                  ds.shape[0], _ptr(rg), ctypes.byref(cp), wp, wb, _stream()), "fsmi_update_map_2d")
    return grid


def eval_beams(off, o, l, lend, prm: Params, out=None, ws=None) -> torch.Tensor:
    """fsmi_eval_beams on CSR beams -> float32 [nbeams]. ws: optional work-queue workspace."""
    lib = load()
    m = _Marshal(off, o, l, lend)
    off = m.arg(off, torch.int32, "off", 1)
    o = m.arg(o, torch.float32, "o", 1)
    l = m.arg(l, torch.float32, "l", 1)
    lend = m.arg(lend, torch.float32, "lend", 1)
    nb = off.shape[0] - 1
    out = _out(out, (nb,), m)
    if ws is None:
        ws = _default_ws(QUEUE_BYTES, m.dev)
    wp, wb = _ws_args(ws)
    cp = prm.c()
    _raise(lib.fsmi_eval_beams(_ptr(off), _ptr(o), _ptr(l), _ptr(lend), nb, ctypes.byref(cp), _ptr(out), wp, wb,
                               _stream()), "fsmi_eval_beams")
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


def eval_rle(off, run_o, run_len, prm: Params, out=None, ws=None) -> torch.Tensor:
    """fsmi_eval_rle on CSR runs -> float32 [nrays]. ws: optional work-queue workspace."""
    lib = load()
    m = _Marshal(off, run_o, run_len)
    off = m.arg(off, torch.int32, "run_off", 1)
    ro = m.arg(run_o, torch.float32, "run_o", 1)
    rl = m.arg(run_len, torch.uint8, "run_len", 1)
    nr = off.shape[0] - 1
    out = _out(out, (nr,), m)
    if ws is None:
        ws = _default_ws(QUEUE_BYTES, m.dev)
    wp, wb = _ws_args(ws)
    cp = prm.c()
    _raise(lib.fsmi_eval_rle(_ptr(off), _ptr(ro), _ptr(rl), nr, ctypes.byref(cp), _ptr(out), wp, wb, _stream()),
           "fsmi_eval_rle")
    return m.out(out)


def eval_3d(vox, poses, dirs, prm: Params, out=None, with_runs: bool = False, ws=None):
    """fsmi_eval_3d (fused sample + encode + RLE variant) -> float32 [P, R] (and run counts).
    ws: optional work-queue workspace."""
    lib = load()
    m = _Marshal(vox, poses, dirs)
    v = m.arg(vox, torch.float32, "vox", 3)
    ps = m.arg(poses, torch.int32, "poses", 2, 12)
    ds = m.arg(dirs, torch.int32, "dirs", 2, 3)
    Z, Y, X = v.shape
    P, R = ps.shape[0], ds.shape[0]
    out = _out(out, (P, R), m)
    nr = torch.empty((P, R), dtype=torch.int32, device=m.dev) if with_runs else None
    if ws is None:
        ws = _default_ws(QUEUE_BYTES, m.dev)
    wp, wb = _ws_args(ws)
    cp = prm.c()
    _raise(lib.fsmi_eval_3d(_ptr(v), X, Y, Z, _ptr(ps), P, _ptr(ds), R, ctypes.byref(cp), _ptr(out), _ptr(nr),
                            wp, wb, _stream()), "fsmi_eval_3d")
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


PROBE_EX2, PROBE_RCP, PROBE_FMA, PROBE_FMA2, PROBE_READ, PROBE_SPIN = range(6)


def probe(kind: int, iters: int, buf: torch.Tensor) -> None:
    """fsmi_probe: one launch of a measurement kernel (PROBE_*) on the current stream; buf is the
    sink (ALU probes), the buffer read (PROBE_READ) or the int64 cycle count (PROBE_SPIN)."""
    lib = load()
    if not buf.is_cuda or not buf.is_contiguous():
        raise FsmiError("probe: buf must be a contiguous CUDA tensor")
    _raise(lib.fsmi_probe(kind, iters, _ptr(buf), buf.numel() * buf.element_size(), _stream()), "fsmi_probe")


def probe_threads(kind: int) -> int:
    """Threads of one fsmi_probe launch of `kind` on the current device."""
    return int(load().fsmi_probe_threads(kind))


def set_wait_limit(polls: int) -> None:
    """fsmi_set_wait_limit: poll limit of the surrogate inference epilogue's wait for its
    accumulator on this host thread (polls < 0 restores the default)."""
    _raise(load().fsmi_set_wait_limit(polls), "fsmi_set_wait_limit")


def device_status() -> int:
    """Reads and clears the current device's status word (waits for the current stream)."""
    lib = load()
    v = ctypes.c_int(0)
    _raise(lib.fsmi_device_status(_stream(), ctypes.byref(v)), "fsmi_device_status")
    return int(v.value)


def set_schedule(kind: int, sched: Schedule | None) -> None:
    """fsmi_set_schedule of family `kind` (KIND_2D / KIND_RLE) for the calling thread (None
    restores the defaults)."""
    lib = load()
    c = sched.c() if sched is not None else None
    _raise(lib.fsmi_set_schedule(kind, ctypes.byref(c) if c is not None else None), "fsmi_set_schedule")


def get_schedule(kind: int) -> Schedule:
    lib = load()
    c = _CSchedule()
    _raise(lib.fsmi_get_schedule(kind, ctypes.byref(c)), "fsmi_get_schedule")
    return Schedule.of(c)


def schedule_candidates(kind: int) -> list[Schedule]:
    """The library's default candidate schedules of family `kind`."""
    lib = load()
    arr = (_CSchedule * 64)()
    n = ctypes.c_int(0)
    _raise(lib.fsmi_schedule_candidates(kind, arr, 64, ctypes.byref(n)), "fsmi_schedule_candidates")
    return [Schedule.of(arr[i]) for i in range(n.value)]


def autotune(kind: int, fn, candidates: list[Schedule] | None = None, reps: int = 3):
    """fsmi_autotune: times fn() (fsmi calls of family `kind` on the current stream) under each
    candidate (default: the library's list); leaves the fastest schedule set for this thread.
    Returns (best, candidates, [ms per candidate or -1])."""
    lib = load()
    if candidates is None:
        candidates = schedule_candidates(kind)

    def cb(ctx, stream):
        try:
            fn()
            return 0
        except FsmiError:  # a schedule the launch cannot take: the candidate is skipped
            return 1

    cfn = _TUNE_FN(cb)
    arr = (_CSchedule * len(candidates))(*[c.c() for c in candidates])
    ms = (ctypes.c_float * len(candidates))()
    best = _CSchedule()
    _raise(lib.fsmi_autotune(kind, cfn, None, arr, len(candidates), reps, _stream(), ctypes.byref(best), ms),
           "fsmi_autotune")
    return Schedule.of(best), list(candidates), [float(v) for v in ms]


def prepare() -> None:
    """fsmi_prepare: per-device lookups and kernel loads, ahead of a graph capture."""
    _raise(load().fsmi_prepare(), "fsmi_prepare")


class Graph:
    """fsmi_* calls captured by the library's own stream-capture helpers and replayed as one CUDA
    graph. fn must make only asynchronous fsmi calls on device tensors with preallocated outputs
    and workspaces."""

    def __init__(self, fn, stream: torch.cuda.Stream | None = None):
        lib = load()
        prepare()
        self.stream = stream or torch.cuda.Stream()
        self._g = ctypes.c_void_p()
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            _raise(lib.fsmi_capture_begin(_stream()), "fsmi_capture_begin")
            try:
                fn()
            finally:
                code = lib.fsmi_capture_end(_stream(), ctypes.byref(self._g))
            _raise(code, "fsmi_capture_end")
        torch.cuda.current_stream().wait_stream(self.stream)

    def replay(self) -> None:
        """Launches the graph on the current stream."""
        _raise(load().fsmi_graph_launch(self._g, _stream()), "fsmi_graph_launch")

    def close(self) -> None:
        if self._g:
            load().fsmi_graph_destroy(self._g)
            self._g = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- learned surrogate ------------------------------------------------------------------------------

def profiles_2d(grid, poses, dirs, beam_ids=None, out=None, max_range: float = 0.0) -> torch.Tensor:
    """fsmi_profiles_2d -> bfloat16 [N][256][2] beam profiles (all P*B beams, or beam_ids); samples
    at distance i + 1/2 >= max_range read as outside the map (max_range <= 0: all 256)."""
    lib = load()
    m = _Marshal(grid, poses, dirs, beam_ids)
    g = m.arg(grid, torch.float32, "grid", 2)
    ps = m.arg(poses, torch.int32, "poses", 2, 4)
    ds = m.arg(dirs, torch.int32, "dirs", 2, 2)
    ids = m.arg(beam_ids, torch.int32, "beam_ids", 1) if beam_ids is not None else None
    N = ids.shape[0] if ids is not None else ps.shape[0] * ds.shape[0]
    if out is None or m.host:
        out = torch.empty((N, SURR_L, 2), dtype=torch.bfloat16, device=m.dev)
    _raise(lib.fsmi_profiles_2d(_ptr(g), g.shape[1], g.shape[0], _ptr(ps), ps.shape[0], _ptr(ds), ds.shape[0],
                                float(max_range), _ptr(ids), N, _ptr(out), _stream()), "fsmi_profiles_2d")
    return m.out(out)


def surrogate_workspace_size(mode: int, N: int) -> int:
    lib = load()
    b = ctypes.c_size_t(0)
    _raise(lib.fsmi_surrogate_workspace_size(mode, N, ctypes.byref(b)), "fsmi_surrogate_workspace_size")
    return int(b.value)


def _dev_tensor(t, dtype, name, numel=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t


def surrogate_loss_grad(params, wbf16, x, y, grad, loss, pred=None, ws=None):
    """fsmi_surrogate_loss_grad: MSE loss (device float32 [1]) and its gradient into grad; with
    y=None only the predictions (pred) are computed. All tensors on the device."""
    lib = load()
    _dev_tensor(params, torch.float32, "params", SURR_NPARAMS)
    _dev_tensor(wbf16, torch.bfloat16, "wbf16", SURR_NPARAMS)
    _dev_tensor(x, torch.bfloat16, "x")
    N = x.shape[0]
    if y is not None:
        _dev_tensor(y, torch.float32, "y", N)
        _dev_tensor(grad, torch.float32, "grad", SURR_NPARAMS)
        _dev_tensor(loss, torch.float32, "loss", 1)
    if pred is not None:
        _dev_tensor(pred, torch.float32, "pred", N)
    if ws is None:
        ws = torch.empty(surrogate_workspace_size(0, N), dtype=torch.uint8, device=x.device)
    wp, wb = _ws_args(ws)
    _raise(lib.fsmi_surrogate_loss_grad(_ptr(params), _ptr(wbf16), _ptr(x), _ptr(y), N, _ptr(grad), _ptr(loss),
                                        _ptr(pred), wp, wb, _stream()), "fsmi_surrogate_loss_grad")


def surrogate_adam(params, m, v, grad, lr: float, t: int, wbf16, beta1=0.9, beta2=0.999, eps=1e-8):
    lib = load()
    for name, tt in (("params", params), ("m", m), ("v", v), ("grad", grad)):
        _dev_tensor(tt, torch.float32, name, SURR_NPARAMS)
    _dev_tensor(wbf16, torch.bfloat16, "wbf16", SURR_NPARAMS)
    _raise(lib.fsmi_surrogate_adam(_ptr(params), _ptr(m), _ptr(v), _ptr(grad), float(lr), float(beta1), float(beta2),
                                   float(eps), int(t), _ptr(wbf16), _stream()), "fsmi_surrogate_adam")


def surrogate_cast(params, wbf16):
    lib = load()
    _dev_tensor(params, torch.float32, "params", SURR_NPARAMS)
    _dev_tensor(wbf16, torch.bfloat16, "wbf16", SURR_NPARAMS)
    _raise(lib.fsmi_surrogate_cast(_ptr(params), _ptr(wbf16), _stream()), "fsmi_surrogate_cast")


def surrogate_predict(params, wbf16, grid=None, poses=None, dirs=None, x=None, out=None, ws=None,
                      max_range: float = 0.0) -> torch.Tensor:
    """fsmi_surrogate_predict on the tensor cores: every beam of every pose on `grid` (profiles sampled
    in the kernel, cut at max_range) -> float32 [P*B], or given profiles x [N][256][2] -> [N]."""
    lib = load()
    _dev_tensor(params, torch.float32, "params", SURR_NPARAMS)
    _dev_tensor(wbf16, torch.bfloat16, "wbf16", SURR_NPARAMS)
    dev = params.device
    if grid is not None:
        g = _dev_tensor(grid, torch.float32, "grid")
        ps = _dev_tensor(poses, torch.int32, "poses")
        ds = _dev_tensor(dirs, torch.int32, "dirs")
        N = ps.shape[0] * ds.shape[0]
        args = (_ptr(g), g.shape[1], g.shape[0], _ptr(ps), ps.shape[0], _ptr(ds), ds.shape[0], float(max_range), None, 0)
    else:
        xx = _dev_tensor(x, torch.bfloat16, "x")
        N = xx.shape[0]
        args = (None, 0, 0, None, 0, None, 0, 0.0, _ptr(xx), N)
    if out is None:
        if _capturing():
            raise FsmiError("inside a graph capture pass a preallocated `out`")
        out = torch.empty(N, dtype=torch.float32, device=dev)
    if ws is None:
        if _capturing():
            raise FsmiError("inside a graph capture pass a preallocated workspace")
        ws = torch.empty(surrogate_workspace_size(1, N), dtype=torch.uint8, device=dev)
    wp, wb = _ws_args(ws)
    _raise(lib.fsmi_surrogate_predict(_ptr(params), _ptr(wbf16), *args, _ptr(out), wp, wb, _stream()),
           "fsmi_surrogate_predict")
    return out


def topk(v, k: int, out=None) -> torch.Tensor:
    """fsmi_topk: int32 indices of the k largest values, descending, lower index first on ties."""
    lib = load()
    vv = _dev_tensor(v, torch.float32, "v")
    if out is None:
        out = torch.empty(k, dtype=torch.int32, device=vv.device)
    _raise(lib.fsmi_topk(_ptr(vv), vv.numel(), k, _ptr(out), _stream()), "fsmi_topk")
    return out


def gather_rows(src, idx, out=None) -> torch.Tensor:
    """fsmi_gather_rows: src int32 [R][w], idx int32 [k] -> [k][w]."""
    lib = load()
    s_ = _dev_tensor(src, torch.int32, "src")
    ii = _dev_tensor(idx, torch.int32, "idx")
    w = s_.shape[1]
    if out is None:
        out = torch.empty((ii.numel(), w), dtype=torch.int32, device=s_.device)
    _raise(lib.fsmi_gather_rows(_ptr(s_), s_.shape[0], w, _ptr(ii), ii.numel(), _ptr(out), _stream()),
           "fsmi_gather_rows")
    return out


# ---- mixed 2D / 3D candidate sets -------------------------------------------------------------------

def make_sets(sets, device=None):
    """Packs [(kind, pose_offset, npose, dir_offset, ndir, max_range[, volume]), ...] into the fsmi_set
    layout (int32 [nsets, 10]), outputs consecutive in list order. Returns (tensor, total items)."""
    import struct
    words, off = [], 0
    for st in sets:
        kind, po, npose, do, ndir, rng = st[:6]
        vol = st[6] if len(st) > 6 else 0
        fbits = struct.unpack("<i", struct.pack("<f", float(rng)))[0]
        lo, hi = struct.unpack("<ii", struct.pack("<q", off))
        words.append([int(kind), int(po), int(npose), int(do), int(ndir), fbits, int(vol), 0, lo, hi])
        off += int(npose) * int(ndir)
    t = torch.tensor(words, dtype=torch.int32).reshape(len(words), SET_WORDS)
    return (t.to(device) if device is not None else t), off


def make_volumes(volumes, device=None):
    """fsmi_volume descriptors (int32 [nvol, 6]) of float32 CUDA tensors [Z][Y][X]."""
    import struct
    words = []
    for v in volumes:
        if not (v.is_cuda and v.dtype == torch.float32 and v.dim() == 3 and v.is_contiguous()):
            raise TypeError("volumes must be contiguous float32 CUDA tensors [Z][Y][X]")
        lo, hi = struct.unpack("<ii", struct.pack("<Q", v.data_ptr()))
        Z, Y, X = v.shape
        words.append([lo, hi, X, Y, Z, 0])
    t = torch.tensor(words, dtype=torch.int32).reshape(len(words), VOLUME_WORDS)
    return t.to(device) if device is not None else t


def mixed_workspace_size(map_cells: int, nsets: int) -> int:
    """fsmi_mixed_workspace_size: bytes of fsmi_eval_mixed's workspace with the range-class plan."""
    b = ctypes.c_size_t(0)
    _raise(load().fsmi_mixed_workspace_size(map_cells, nsets, ctypes.byref(b)), "fsmi_mixed_workspace_size")
    return int(b.value)


def eval_mixed(sets, nitems: int, out=None, times=None, ws=None, grid=None, poses2=None, dirs2=None,
               prm2: Params | None = None, volumes=None, poses3=None, dirs3=None, prm3: Params | None = None):
    """fsmi_eval_mixed: 2D and 3D candidate sets (make_sets) in one call -> float32 [nitems]
    (without `ws`, a workspace with the range-class plan is allocated). volumes: int32 [nvol, 6] from make_volumes (the tensors must stay alive). times
    (optional) uint64-as-int64 [nitems + 1] receives the block start and per-item completion times."""
    lib = load()
    st = _dev_tensor(sets, torch.int32, "sets")
    dev = st.device
    if out is None:
        if _capturing():
            raise FsmiError("inside a graph capture pass a preallocated `out`")
        out = torch.empty(nitems, dtype=torch.float32, device=dev)
    if times is not None:
        _dev_tensor(times, torch.int64, "times", nitems + 1)
    if ws is None:
        if _capturing():
            raise FsmiError("inside a graph capture pass a preallocated workspace")
        nb = mixed_workspace_size(grid.numel() if prm2 is not None and grid is not None else 0, st.shape[0])
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    wp, wb = _ws_args(ws)
    c2 = prm2.c() if prm2 is not None else None
    c3 = prm3.c() if prm3 is not None else None
    g = grid
    args2 = (_ptr(g), g.shape[1], g.shape[0], _ptr(poses2), poses2.shape[0], _ptr(dirs2), dirs2.shape[0],
             ctypes.byref(c2)) if prm2 is not None else (None, 1, 1, None, 0, None, 0, None)
    args3 = (_ptr(volumes), volumes.shape[0], _ptr(poses3), poses3.shape[0], _ptr(dirs3), dirs3.shape[0],
             ctypes.byref(c3)) if prm3 is not None else (None, 0, None, 0, None, 0, None)
    _raise(lib.fsmi_eval_mixed(*args2, *args3, _ptr(st), st.shape[0], nitems, _ptr(out), _ptr(times), wp, wb,
                               _stream()), "fsmi_eval_mixed")
    return out
