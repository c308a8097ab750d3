"""Seeded synthetic inputs shaped like the paper's 2D and 3D workloads.

This module only draws random numbers and lays them out; it holds none of the method's
arithmetic. Both the CUDA path and the CPU oracle consume the arrays it returns, bit for bit.

Fixed-point conventions shared by every input:
  * positions are int32 in units of 2^-16 cell (Q16);
  * unit vectors and rotation entries are int32 in units of 2^-30 (Q30), rounded from float64;
  * a 2D pose is [x, y, cos(yaw), sin(yaw)] (Q16, Q16, Q30, Q30);
  * a 3D pose is [x, y, z, R00, R01, R02, R10, ..., R22] (Q16 x3, Q30 x9), R = Rz(yaw) Ry(pitch).

Workloads (sizes from the benchmark configurations; the paper's own timing experiments use random
occupancies, Section 5.1 and Section 5.4, and private robot logs that are not reproduced here):
  * ``random_grid_200``: 200x200 grid, o ~ U(0.05, 0.95) iid, one pose at the centre of cell (100, 100),
    360 beams at 1 degree, range 64 cells.
  * ``office_scene``: 2048x2048 grid, background 0.1, 400 rectangles (sides 8..64) at 0.9, then
    unknown (0.5) rectangles (sides 64..512) painted until they cover >= 40%; poses at centres of
    free (0.1) cells, yaw 0, 360 beams, range 256.
  * ``voxel_scene``: 512x512x128 voxels, background 0.1, 200 boxes (sides 8..64) at 0.9, half-space
    x >= 256 at 0.5, then 10% of voxels replaced by U(0.3, 0.7); 64 poses in free voxels with
    z in [32, 96), random yaw, pitch 0; 128x128 pinhole rays over a 90x90 degree field of view;
    range 384 virtual cells.
  * ``e5_runs``: the Section 5.4 micro-workload, n = 256 virtual cells in groups of L equal cells.
"""
from __future__ import annotations

import math

import numpy as np

Q16 = 1 << 16
Q30 = 1 << 30


def q30(v) -> np.ndarray:
    return np.rint(np.asarray(v, np.float64) * Q30).astype(np.int64).clip(-(2**31) + 1, 2**31 - 1).astype(np.int32)


def beam_dirs_2d(nbeams: int = 360) -> np.ndarray:
    """Unit vectors of nbeams beams at b * 360/nbeams degrees, int32 [B, 2] (Q30)."""
    a = np.arange(nbeams, dtype=np.float64) * (2.0 * math.pi / nbeams)
    return np.stack([q30(np.cos(a)), q30(np.sin(a))], axis=1)


def pose_2d(x: float, y: float, yaw: float = 0.0) -> np.ndarray:
    return np.array([int(round(x * Q16)), int(round(y * Q16)), q30(math.cos(yaw)), q30(math.sin(yaw))],
                    dtype=np.int32)


def random_dirs_2d(n: int, rng: np.random.Generator) -> np.ndarray:
    a = rng.uniform(0.0, 2.0 * math.pi, n)
    return np.stack([q30(np.cos(a)), q30(np.sin(a))], axis=1)


def random_grid_200(seed: int = 0):
    """Returns (grid float32 [200, 200], poses int32 [1, 4], dirs int32 [360, 2])."""
    rng = np.random.default_rng(seed)
    grid = rng.uniform(0.05, 0.95, size=(200, 200)).astype(np.float32)
    poses = pose_2d(100.5, 100.5, 0.0)[None, :]
    return grid, poses, beam_dirs_2d(360)


def office_grid(size: int = 2048, n_obst: int = 400, unknown_cover: float = 0.40, seed: int = 0) -> np.ndarray:
    """Background 0.1, n_obst axis-aligned rectangles (sides 8..64) at 0.9, then unknown 0.5
    rectangles (sides 64..512, clipped to the grid) until they cover >= unknown_cover."""
    rng = np.random.default_rng(seed)
    g = np.full((size, size), 0.1, np.float32)
    for _ in range(n_obst):
        w, h = rng.integers(8, 65, size=2)
        x0, y0 = rng.integers(0, size - w + 1), rng.integers(0, size - h + 1)
        g[y0:y0 + h, x0:x0 + w] = 0.9
    unknown = np.zeros((size, size), bool)
    smax = min(512, size)
    smin = min(64, smax)
    while unknown.mean() < unknown_cover:
        w, h = rng.integers(smin, smax + 1, size=2)
        x0, y0 = rng.integers(0, size - w + 1), rng.integers(0, size - h + 1)
        unknown[y0:y0 + h, x0:x0 + w] = True
    g[unknown] = 0.5
    return g


def free_cell_poses_2d(grid: np.ndarray, n: int, seed: int = 1, margin: int = 0) -> np.ndarray:
    """n poses at centres of cells with o == 0.1, yaw 0. int32 [n, 4]."""
    rng = np.random.default_rng(seed)
    Hh, W = grid.shape
    ys, xs = np.nonzero(grid == np.float32(0.1))
    keep = (xs >= margin) & (xs < W - margin) & (ys >= margin) & (ys < Hh - margin)
    xs, ys = xs[keep], ys[keep]
    idx = rng.choice(len(xs), size=n, replace=len(xs) < n)
    poses = np.zeros((n, 4), np.int32)
    poses[:, 0] = xs[idx] * Q16 + Q16 // 2
    poses[:, 1] = ys[idx] * Q16 + Q16 // 2
    poses[:, 2] = Q30
    poses[:, 3] = 0
    return poses


def frontier_poses_2d(grid: np.ndarray, n: int, seed: int = 1, rmin: float = 2.0, rmax: float = 24.0) -> np.ndarray:
    """n poses at centres of free cells (o == 0.1) whose Euclidean distance to the nearest unknown
    cell (o == 0.5) lies in [rmin, rmax] cells: candidate sensing positions at the map's frontiers,
    where the information a pose sees varies far more than deep in explored space. int32 [n, 4]."""
    from scipy.ndimage import distance_transform_edt

    rng = np.random.default_rng(seed)
    dist = distance_transform_edt(grid != np.float32(0.5))
    ys, xs = np.nonzero((grid == np.float32(0.1)) & (dist >= rmin) & (dist <= rmax))
    if len(xs) == 0:
        raise ValueError("no free cell at the requested distance from unknown space")
    idx = rng.choice(len(xs), size=n, replace=len(xs) < n)
    poses = np.zeros((n, 4), np.int32)
    poses[:, 0] = xs[idx] * Q16 + Q16 // 2
    poses[:, 1] = ys[idx] * Q16 + Q16 // 2
    poses[:, 2] = Q30
    poses[:, 3] = 0
    return poses


def office_scene(n_poses: int = 1024, size: int = 2048, seed: int = 0, pose_seed: int = 1):
    """Returns (grid float32 [size, size], poses int32 [P, 4], dirs int32 [360, 2])."""
    grid = office_grid(size, 400 if size >= 1024 else max(8, 400 * size * size // (2048 * 2048)), 0.40, seed)
    poses = free_cell_poses_2d(grid, n_poses, pose_seed)
    return grid, poses, beam_dirs_2d(360)


def rot3(yaw: float, pitch: float) -> np.ndarray:
    cy, sy, cp, sp = math.cos(yaw), math.sin(yaw), math.cos(pitch), math.sin(pitch)
    rz = np.array([[cy, -sy, 0.0], [sy, cy, 0.0], [0.0, 0.0, 1.0]])
    ry = np.array([[cp, 0.0, sp], [0.0, 1.0, 0.0], [-sp, 0.0, cp]])
    return rz @ ry


def pose_3d(x: float, y: float, z: float, yaw: float = 0.0, pitch: float = 0.0) -> np.ndarray:
    out = np.zeros(12, np.int32)
    out[:3] = [int(round(x * Q16)), int(round(y * Q16)), int(round(z * Q16))]
    out[3:] = q30(rot3(yaw, pitch).reshape(-1))
    return out


def pinhole_dirs(w: int = 128, h: int = 128, fov_deg: float = 90.0) -> np.ndarray:
    """Unit vectors of a w x h pinhole grid looking along +x, int32 [w*h, 3] (Q30)."""
    t = math.tan(math.radians(fov_deg) / 2.0)
    u = (-1.0 + (np.arange(w) + 0.5) * 2.0 / w) * t
    v = (-1.0 + (np.arange(h) + 0.5) * 2.0 / h) * t
    uu, vv = np.meshgrid(u, v)
    d = np.stack([np.ones_like(uu), uu, vv], axis=-1).reshape(-1, 3)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return q30(d)


def voxel_world(X: int = 512, Y: int = 512, Z: int = 128, n_boxes: int = 200, seed: int = 0,
                noise_seed: int = 2, noise_frac: float = 0.10) -> np.ndarray:
    """float32 [Z, Y, X] occupancy volume of the 3D workload."""
    rng = np.random.default_rng(seed)
    v = np.full((Z, Y, X), 0.1, np.float32)
    for _ in range(n_boxes):
        sx, sy, sz = (int(min(s, dim)) for s, dim in zip(rng.integers(8, 65, size=3), (X, Y, Z)))
        x0 = rng.integers(0, X - sx + 1)
        y0 = rng.integers(0, Y - sy + 1)
        z0 = rng.integers(0, Z - sz + 1)
        v[z0:z0 + sz, y0:y0 + sy, x0:x0 + sx] = 0.9
    v[:, :, X // 2:] = 0.5
    nrng = np.random.default_rng(noise_seed)
    flat = v.reshape(-1)
    mask = nrng.random(flat.shape[0], dtype=np.float32) < noise_frac
    flat[mask] = nrng.uniform(0.3, 0.7, int(mask.sum())).astype(np.float32)
    return v


def free_voxel_poses(vox: np.ndarray, n: int, seed: int = 3, zlo: int = 32, zhi: int = 96) -> np.ndarray:
    """n poses at centres of voxels with o == 0.1 and z in [zlo, zhi), random yaw, pitch 0."""
    rng = np.random.default_rng(seed)
    Z, Y, X = vox.shape
    zlo, zhi = min(zlo, Z - 1), min(zhi, Z)
    sub = vox[zlo:zhi]
    zs, ys, xs = np.nonzero(sub == np.float32(0.1))
    if len(xs) == 0:
        raise ValueError("no free (o == 0.1) voxel in the requested height band")
    idx = rng.choice(len(xs), size=n, replace=len(xs) < n)
    yaws = rng.uniform(0.0, 2.0 * math.pi, n)
    return np.stack([pose_3d(xs[i] + 0.5, ys[i] + 0.5, zs[i] + zlo + 0.5, yaws[k], 0.0)
                     for k, i in enumerate(idx)])


def voxel_scene(n_poses: int = 64, X: int = 512, Y: int = 512, Z: int = 128, rays: int = 128):
    """Returns (vox float32 [Z, Y, X], poses int32 [P, 12], dirs int32 [rays*rays, 3])."""
    scale = (X * Y * Z) / (512 * 512 * 128)
    vox = voxel_world(X, Y, Z, n_boxes=max(4, int(round(200 * scale))))
    poses = free_voxel_poses(vox, n_poses)
    return vox, poses, pinhole_dirs(rays, rays, 90.0)


# ---- explicit beams and runs (tests, Section 5.1 / 5.4 shapes) -------------------------------------

def random_beams(nbeams: int, nmin: int, nmax: int, seed: int, o_lo: float = 0.0, o_hi: float = 1.0,
                 w_lo: float = 0.05, w_hi: float = 1.4142, unit: bool = False):
    """CSR beams: off int32 [nb+1], o float32 [total], l float32 [total] (entry distances, the
    first of each beam 0), lend float32 [nb] (end distances). Cell widths U(w_lo, w_hi), or all
    1 when unit=True."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=nbeams)
    off = np.zeros(nbeams + 1, np.int32)
    off[1:] = np.cumsum(ns)
    o = rng.uniform(o_lo, o_hi, size=int(off[-1])).astype(np.float32)
    l = np.zeros(int(off[-1]), np.float32)
    lend = np.zeros(nbeams, np.float32)
    for b in range(nbeams):
        n = int(ns[b])
        w = np.ones(n) if unit else rng.uniform(w_lo, w_hi, size=n)
        edges = np.concatenate([[0.0], np.cumsum(w)]).astype(np.float32)
        l[off[b]:off[b + 1]] = edges[:n]
        lend[b] = edges[n]
    return off, o, l, lend


def random_runs(nrays: int, nr_min: int, nr_max: int, lmax: int, seed: int, o_lo: float = 0.0,
                o_hi: float = 1.0, lmin: int = 1):
    """CSR runs: off int32 [nr+1], run_o float32 [total], run_len uint8 [total]."""
    rng = np.random.default_rng(seed)
    counts = rng.integers(nr_min, nr_max + 1, size=nrays)
    off = np.zeros(nrays + 1, np.int32)
    off[1:] = np.cumsum(counts)
    ro = rng.uniform(o_lo, o_hi, size=int(off[-1])).astype(np.float32)
    rl = rng.integers(lmin, lmax + 1, size=int(off[-1])).astype(np.uint8)
    return off, ro, rl


def e5_runs(L: int, nbeams: int = 1000, n: int = 256, seed: int = 0):
    """Section 5.4 workload: n virtual cells in groups of L with o ~ U(0, 1) per group."""
    rng = np.random.default_rng(seed)
    per = n // L
    off = (np.arange(nbeams + 1) * per).astype(np.int32)
    ro = rng.uniform(0.0, 1.0, size=nbeams * per).astype(np.float32)
    rl = np.full(nbeams * per, L, np.uint8)
    return off, ro, rl
