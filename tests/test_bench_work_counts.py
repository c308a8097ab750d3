"""The bench's algorithmic work counts of the fused 3D launch (bench.rle_work_counts), on CPU: the
runs come from the oracle's sampler and encoder in place of the library's encoder, and the counts
are checked against loops over every ray, run and cell written out directly from their
definitions (Theorem 5's kept pairs as the oracle's pinned sub-block mask)."""
import types

import numpy as np
import pytest
import torch

import bench
import oracle
from paper_1905_02238_gb300 import synth


@pytest.fixture(scope="module", autouse=True)
def orc():
    oracle.build()
    return oracle


def _world():
    vox = synth.voxel_world(64, 48, 32, n_boxes=12, seed=0, noise_seed=1, noise_frac=0.3)
    poses = synth.free_voxel_poses(vox, 3, seed=2, zlo=4, zhi=28)
    dirs = synth.pinhole_dirs(6, 5, 100.0)
    return vox, poses, dirs


def _runs(vox, poses, dirs, nsamp, cap):
    per_ray = []
    for p in range(poses.shape[0]):
        for r in range(dirs.shape[0]):
            per_ray.append(oracle.rle_encode(oracle.sample_3d(vox, poses[p], dirs[r], nsamp), cap))
    return per_ray


def _fake_fsmi(vox, dirs, nsamp, cap):
    def rle_encode_3d(v, pp, vd, prm, capacity):
        off, ros, rls = [0], [], []
        for ro, rl in _runs(vox, pp.numpy(), dirs, nsamp, cap):
            ros.append(ro)
            rls.append(rl)
            off.append(off[-1] + len(rl))
        rl = np.concatenate(rls).astype(np.uint8)
        return (torch.tensor(off, dtype=torch.int32), torch.from_numpy(np.concatenate(ros)),
                torch.from_numpy(rl))

    return types.SimpleNamespace(APPROX=1, rle_encode_3d=rle_encode_3d)


def _keep(rl, D):
    """Theorem 5's kept pairs (j, k) of one ray: the diagonal blocks and the sub-blocks (su')-(Lv')."""
    s = np.concatenate([[0], np.cumsum(rl)])
    run_of = np.repeat(np.arange(len(rl)), rl)
    n = int(s[-1])
    keep = np.zeros((n, n), bool)
    for j in range(n):
        for k in range(n):
            u, v = run_of[j], run_of[k]
            if u == v:
                keep[j, k] = True
            elif u < v:
                keep[j, k] = (s[v] < s[u] + rl[u] + D and j >= max(s[u], s[v] - D)
                              and k < s[v] + min(rl[v], s[u] + rl[u] + D - s[v]))
            else:
                keep[j, k] = (s[u] < s[v] + rl[v] + D and j < s[u] + min(rl[u], s[v] + rl[v] + D - s[u])
                              and k >= max(s[v], s[u] - D))
    return keep


@pytest.mark.parametrize("D,cell_runlen", [(2, 8), (6, 32), (0, 4)])
def test_theorem5_window_taps_match_the_sub_block_mask(D, cell_runlen):
    vox, poses, dirs = _world()
    nsamp, cap, K = 48, 8, 5
    prm = types.SimpleNamespace(variant=1, approx_reading=0, trunc_delta=D, max_range=float(nsamp))
    tot = bench.rle_work_counts(_fake_fsmi(vox, dirs, nsamp, cap), torch.from_numpy(vox), torch.from_numpy(poses),
                                torch.from_numpy(dirs), prm, cell_runlen, K, poses_per_chunk=2)
    samples = runs = cell_rays = cell_cells = pair_rays = taps = 0
    for ro, rl in _runs(vox, poses, dirs, nsamp, cap):
        n, nr = int(rl.sum()), len(rl)
        samples += n
        runs += nr
        if n < cell_runlen * nr:
            cell_rays += 1
            cell_cells += n
            keep = _keep(rl, D)
            idx = np.arange(n)
            taps += int((keep & (np.abs(idx[None, :] - idx[:, None]) <= K)).sum())
        elif nr > 0:
            pair_rays += 1
    assert (tot["samples"], tot["runs"], tot["cell_rays"], tot["cell_cells"], tot["pair_rays"]) == \
        (samples, runs, cell_rays, cell_cells, pair_rays)
    assert tot["window_taps"] == taps
    assert tot["fp32_ops"] == taps + cell_cells + 6 * tot["pair_terms"]
