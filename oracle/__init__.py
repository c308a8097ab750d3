"""FP64 CPU oracle for FSMI (Zhang, Henderson, Karaman, Sze, IJRR 2019).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA library in
``paper_1905_02238_gb300``; the two meet only at the seeded input arrays.

The arithmetic lives in ``fsmi_oracle.c`` (plain C, double precision, one function per equation or
algorithm of the paper). This module compiles it with gcc on first use and wraps it with ctypes.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against something other
than itself (closed forms, brute-force integration of the mutual-information definition, exact
rational geometry, enumeration, identities proved in the paper); see ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsmi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle_fsmi.so")
_lock = threading.Lock()
_lib = None

EXACT, APPROX, UNIFORM = 0, 1, 2
G_PDF, G_ERF = 0, 1


class _Params(ctypes.Structure):
    _fields_ = [
        ("variant", ctypes.c_int),
        ("sigma", ctypes.c_double),
        ("delta_occ", ctypes.c_double),
        ("delta_emp", ctypes.c_double),
        ("trunc_delta", ctypes.c_int),
        ("uniform_h", ctypes.c_int),
        ("max_range", ctypes.c_double),
        ("run_cap", ctypes.c_int),
        ("g_kernel", ctypes.c_int),
        ("e0_mode", ctypes.c_int),
        ("approx_reading", ctypes.c_int),
    ]


@dataclass
class Params:
    """Method parameters, in cell units (w = 1)."""

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

    def c(self) -> _Params:
        return _Params(int(self.variant), float(self.sigma), float(self.delta_occ), float(self.delta_emp),
                       int(self.trunc_delta), int(self.uniform_h), float(self.max_range), int(self.run_cap),
                       int(self.g_kernel), int(self.e0_mode), int(self.approx_reading))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP over beams). Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            P = ctypes.POINTER(_Params)
            lib.oracle_f_odds.restype = d
            lib.oracle_f_odds.argtypes = [d, d]
            lib.oracle_f_prob.restype = d
            lib.oracle_f_prob.argtypes = [d, d]
            lib.oracle_first_hit.argtypes = [p, i, p]
            lib.oracle_c_k.argtypes = [p, i, d, d, p]
            lib.oracle_fsmi_beam.restype = d
            lib.oracle_fsmi_beam.argtypes = [p, p, i, P]
            lib.oracle_fsmi_beam_skip.restype = d
            lib.oracle_fsmi_beam_skip.argtypes = [p, p, p, i, P]
            lib.oracle_eval_trajectories_2d.argtypes = [p, i, i, p, p, i, p, i, P, p, p, p]
            lib.oracle_update_map_2d.argtypes = [p, i, i, p, i, p, i, p, P]
            lib.oracle_uniform_pairsum.restype = d
            lib.oracle_uniform_pairsum.argtypes = [p, p, i, P]
            lib.oracle_beam_dir_2d.argtypes = [p, p, p]
            lib.oracle_trace_2d.restype = i
            lib.oracle_trace_2d.argtypes = [i, i, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int64, i, p, p]
            lib.oracle_eval_2d.argtypes = [p, i, i, p, i, p, i, P, p, i]
            lib.oracle_eval_beams.argtypes = [p, p, p, p, i, P, p, i]
            lib.oracle_sample_3d.restype = i
            lib.oracle_sample_3d.argtypes = [p, i, i, i, p, p, i, p]
            lib.oracle_rle_encode.restype = i
            lib.oracle_rle_encode.argtypes = [p, i, i, p, p]
            lib.oracle_rle_A.restype = d
            lib.oracle_rle_A.argtypes = [i, d, i, i, d, i, i, i]
            lib.oracle_rle_B.restype = d
            lib.oracle_rle_B.argtypes = [i, d, i, i, d, i, i, i]
            lib.oracle_rle_beam.restype = d
            lib.oracle_rle_beam.argtypes = [p, p, i, P]
            lib.oracle_eval_rle.argtypes = [p, p, p, i, P, p, i]
            lib.oracle_eval_3d.argtypes = [p, i, i, i, p, i, p, i, P, p, p, i]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def default_threads() -> int:
    return os.cpu_count() or 1


# ---- Section 2.2 -------------------------------------------------------------------------------

def f_odds(delta: float, r: float) -> float:
    """f(delta, r) as printed in Section 2.2 (odds form)."""
    return _load().oracle_f_odds(float(delta), float(r))


def f_prob(delta: float, o: float) -> float:
    """f(delta, r) rewritten in o = r/(1+r)."""
    return _load().oracle_f_prob(float(delta), float(o))


def first_hit(o) -> np.ndarray:
    """Algorithm 2: [P(e_0), P(e_1), ..., P(e_n)]."""
    o = _c(o, np.float64)
    pe = np.zeros(len(o) + 1)
    _load().oracle_first_hit(_ptr(o), len(o), _ptr(pe))
    return pe


def c_k(o, delta_occ: float, delta_emp: float) -> np.ndarray:
    """Algorithm 3: [C_1, ..., C_n]."""
    o = _c(o, np.float64)
    C = np.zeros(len(o))
    _load().oracle_c_k(_ptr(o), len(o), float(delta_occ), float(delta_emp), _ptr(C))
    return C


# ---- 2D variants ---------------------------------------------------------------------------------

def fsmi_beam(o, l, prm: Params) -> float:
    """FSMI / Approx-FSMI / Uniform-FSMI of one explicit beam; o has n entries, l has n+1."""
    o = _c(o, np.float64)
    l = _c(l, np.float64)
    assert len(l) == len(o) + 1
    cp = prm.c()
    return _load().oracle_fsmi_beam(_ptr(o), _ptr(l), len(o), ctypes.byref(cp))


def fsmi_beam_skip(o, l, skip, prm: Params) -> float:
    """fsmi_beam summing only the cells with skip[i] == 0 (Section 2.4: already-counted cells keep
    their occupancy but add no gain)."""
    o = _c(o, np.float64)
    l = _c(l, np.float64)
    sk = _c(np.asarray(skip, bool), np.uint8)
    assert len(l) == len(o) + 1 and len(sk) == len(o)
    cp = prm.c()
    return _load().oracle_fsmi_beam_skip(_ptr(o), _ptr(l), _ptr(sk), len(o), ctypes.byref(cp))


def uniform_pairsum(o, l, prm: Params) -> float:
    """Uniform-FSMI as the generic pair sum of eq. (uniform) (overlap of the uniform density)."""
    o = _c(o, np.float64)
    l = _c(l, np.float64)
    cp = prm.c()
    return _load().oracle_uniform_pairsum(_ptr(o), _ptr(l), len(o), ctypes.byref(cp))


def beam_dir_2d(pose, u) -> np.ndarray:
    pose = _c(pose, np.int32)
    u = _c(u, np.int32)
    d = np.zeros(2, np.int32)
    _load().oracle_beam_dir_2d(_ptr(pose), _ptr(u), _ptr(d))
    return d


def range_fix(max_range: float) -> int:
    return int(np.rint(np.float64(np.float32(max_range)) * 65536.0))


def trace_2d(W: int, H: int, ox: int, oy: int, dx: int, dy: int, max_range: float, cap: int | None = None):
    """Integer DDA of one beam. Returns (cell_ids int32[n], l float64[n+1])."""
    if cap is None:
        cap = int(max_range * 1.5) + 4
    cells = np.zeros(cap, np.int32)
    l = np.zeros(cap + 1, np.float64)
    n = _load().oracle_trace_2d(W, H, int(ox), int(oy), int(dx), int(dy), range_fix(max_range), cap,
                                _ptr(cells), _ptr(l))
    if n < 0:
        raise OverflowError("beam longer than cap")
    return cells[:n].copy(), l[: n + 1].copy()


def eval_2d(grid, poses, dirs, prm: Params, nthreads: int | None = None) -> np.ndarray:
    """Batched 2D path: grid float32 [H, W]; poses int32 [P, 4]; dirs int32 [B, 2]. Returns [P, B]."""
    grid = _c(grid, np.float32)
    poses = _c(poses, np.int32)
    dirs = _c(dirs, np.int32)
    Hh, W = grid.shape
    P, B = poses.shape[0], dirs.shape[0]
    out = np.zeros((P, B), np.float64)
    cp = prm.c()
    cp.max_range = float(np.float32(prm.max_range))
    _load().oracle_eval_2d(_ptr(grid), W, Hh, _ptr(poses), P, _ptr(dirs), B, ctypes.byref(cp), _ptr(out),
                           nthreads or default_threads())
    return out


def eval_trajectories_2d(grid, poses, traj_off, dirs, prm: Params):
    """Section 2.4: MI along trajectories with already-counted cells dropped at later states.
    Returns (beam [P, B], state [P], traj [T]) in float64."""
    grid = _c(grid, np.float32)
    poses = _c(poses, np.int32)
    traj_off = _c(traj_off, np.int32)
    dirs = _c(dirs, np.int32)
    Hh, W = grid.shape
    P, B, T = poses.shape[0], dirs.shape[0], len(traj_off) - 1
    beam = np.zeros((P, B), np.float64)
    state = np.zeros(P, np.float64)
    traj = np.zeros(T, np.float64)
    cp = prm.c()
    cp.max_range = float(np.float32(prm.max_range))
    _load().oracle_eval_trajectories_2d(_ptr(grid), W, Hh, _ptr(poses), _ptr(traj_off), T, _ptr(dirs), B,
                                        ctypes.byref(cp), _ptr(beam), _ptr(state), _ptr(traj))
    return beam, state, traj


def path_lengths(poses, traj_off) -> np.ndarray:
    """Travel distance of each trajectory: the straight distances between consecutive states
    (cells), at least 1."""
    xy = np.asarray(poses, np.float64)[:, :2] / 65536.0
    out = []
    for a, b in zip(traj_off[:-1], traj_off[1:]):
        seg = np.diff(xy[a:b], axis=0)
        out.append(max(1.0, float(np.sqrt((seg ** 2).sum(axis=1)).sum())))
    return np.array(out)


def update_map_2d(grid, poses, dirs, ranges, prm: Params) -> np.ndarray:
    """Eq. (bayesian_filter) applied beam by beam; returns the updated map in float64."""
    m = np.array(grid, np.float64, copy=True, order="C")
    poses = _c(poses, np.int32)
    dirs = _c(dirs, np.int32)
    ranges = _c(ranges, np.float32)
    Hh, W = m.shape
    P, B = poses.shape[0], dirs.shape[0]
    assert ranges.size == P * B
    cp = prm.c()
    cp.max_range = float(np.float32(prm.max_range))
    _load().oracle_update_map_2d(_ptr(m), W, Hh, _ptr(poses), P, _ptr(dirs), B, _ptr(ranges), ctypes.byref(cp))
    return m


def eval_beams(off, o, l, lend, prm: Params, nthreads: int | None = None) -> np.ndarray:
    """Batched explicit beams (CSR): off int32 [nb+1], o/l float32 [total], lend float32 [nb]."""
    off = _c(off, np.int32)
    o = _c(o, np.float32)
    l = _c(l, np.float32)
    lend = _c(lend, np.float32)
    nb = len(off) - 1
    out = np.zeros(nb, np.float64)
    cp = prm.c()
    _load().oracle_eval_beams(_ptr(off), _ptr(o), _ptr(l), _ptr(lend), nb, ctypes.byref(cp), _ptr(out),
                              nthreads or default_threads())
    return out


# ---- Section 4 (RLE) ---------------------------------------------------------------------------

def sample_3d(vox, pose, u, nsamp: int) -> np.ndarray:
    """Virtual-cell samples of one 3D ray; vox float32 [Z, Y, X]; pose int32[12]; u int32[3]."""
    vox = _c(vox, np.float32)
    Z, Y, X = vox.shape
    out = np.zeros(nsamp, np.float32)
    n = _load().oracle_sample_3d(_ptr(vox), X, Y, Z, _ptr(_c(pose, np.int32)), _ptr(_c(u, np.int32)), nsamp,
                                 _ptr(out))
    return out[:n].copy()


def rle_encode(samples, cap: int):
    """Runs (o_u float32[nr], L_u int32[nr]) of a sample sequence."""
    s = _c(samples, np.float32)
    ro = np.zeros(max(len(s), 1), np.float32)
    rl = np.zeros(max(len(s), 1), np.int32)
    nr = _load().oracle_rle_encode(_ptr(s), len(s), int(cap), _ptr(ro), _ptr(rl))
    return ro[:nr].copy(), rl[:nr].copy()


def rle_A(kind: int, sigma: float, H: int, trunc: int, x: float, Lu: int, Lv: int, t: int) -> float:
    return _load().oracle_rle_A(kind, sigma, H, trunc, x, Lu, Lv, t)


def rle_B(kind: int, sigma: float, H: int, trunc: int, x: float, Lu: int, Lv: int, t: int) -> float:
    return _load().oracle_rle_B(kind, sigma, H, trunc, x, Lu, Lv, t)


def rle_beam(run_o, run_len, prm: Params) -> float:
    """FSMI-RLE / Approx-FSMI-RLE / Uniform-FSMI-RLE of one encoded ray."""
    ro = _c(run_o, np.float32)
    rl = _c(run_len, np.int32)
    cp = prm.c()
    return _load().oracle_rle_beam(_ptr(ro), _ptr(rl), len(ro), ctypes.byref(cp))


def eval_rle(off, run_o, run_len, prm: Params, nthreads: int | None = None) -> np.ndarray:
    off = _c(off, np.int32)
    ro = _c(run_o, np.float32)
    rl = _c(run_len, np.uint8)
    nr = len(off) - 1
    out = np.zeros(nr, np.float64)
    cp = prm.c()
    _load().oracle_eval_rle(_ptr(off), _ptr(ro), _ptr(rl), nr, ctypes.byref(cp), _ptr(out),
                            nthreads or default_threads())
    return out


def eval_3d(vox, poses, dirs, prm: Params, nthreads: int | None = None):
    """Batched 3D path. vox float32 [Z, Y, X]; poses int32 [P, 12]; dirs int32 [R, 3].
    Returns (mi float64 [P, R], run counts int32 [P, R])."""
    vox = _c(vox, np.float32)
    poses = _c(poses, np.int32)
    dirs = _c(dirs, np.int32)
    Z, Y, X = vox.shape
    P, R = poses.shape[0], dirs.shape[0]
    out = np.zeros((P, R), np.float64)
    nr = np.zeros((P, R), np.int32)
    cp = prm.c()
    _load().oracle_eval_3d(_ptr(vox), X, Y, Z, _ptr(poses), P, _ptr(dirs), R, ctypes.byref(cp), _ptr(out),
                           _ptr(nr), nthreads or default_threads())
    return out, nr
