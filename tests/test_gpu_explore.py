"""GPU parity of the exploration loop (fsmi_eval_trajectories_2d, fsmi_best_trajectory,
fsmi_scan_sums, fsmi_update_map_2d) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
from paper_1905_02238_gb300 import fsmi, synth
from tests.parity import assert_mi_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1905_02238_gb300 import build

    build.build()
    oracle.build()
    return fsmi.load()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _prms(variant, R, **kw):
    base = dict(variant=variant, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=R, trunc_delta=6, uniform_h=4)
    base.update(kw)
    return fsmi.Params(**base), oracle.Params(**base)


def _trajectories(grid, T=7, seed=3, step=6.0):
    """T random walks through free cells: 0 .. 5 states each, steps of about `step` cells."""
    rng = np.random.default_rng(seed)
    free = synth.free_cell_poses_2d(grid, 200, seed=seed + 1)
    poses, off = [], [0]
    for t in range(T):
        ns = t % 6
        p = free[rng.integers(len(free))].copy()
        for _ in range(ns):
            poses.append(p.copy())
            ang = rng.uniform(0, 2 * np.pi)
            p[0] = int(np.clip(p[0] + step * np.cos(ang) * 65536, 0, (grid.shape[1] - 1) * 65536))
            p[1] = int(np.clip(p[1] + step * np.sin(ang) * 65536, 0, (grid.shape[0] - 1) * 65536))
        off.append(len(poses))
    return np.array(poses, np.int32).reshape(-1, 4), np.array(off, np.int32)


@pytest.mark.parametrize("variant", [fsmi.EXACT, fsmi.APPROX, fsmi.UNIFORM])
def test_trajectories_match_oracle(variant):
    grid = synth.office_grid(160, n_obst=25, seed=21)
    poses, off = _trajectories(grid)
    dirs = synth.beam_dirs_2d(72)
    gp, op = _prms(variant, 48.0)
    beam, state, traj = fsmi.eval_trajectories_2d(_cuda(grid), _cuda(poses), _cuda(off), _cuda(dirs), gp)
    rb, rs, rt = oracle.eval_trajectories_2d(grid, poses, off, dirs, op)
    assert_mi_close(beam.cpu().numpy(), rb, f"traj beams {variant}")
    assert_mi_close(state.cpu().numpy(), rs, f"traj states {variant}")
    assert_mi_close(traj.cpu().numpy(), rt, f"traj sums {variant}")
    assert traj.cpu().numpy()[0] == 0.0  # trajectory 0 has no state
    # the marks matter: a later state of a trajectory gets less than its scan alone
    alone = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp).sum(dim=1).cpu().numpy()
    first = np.zeros(len(poses), bool)
    first[off[:-1][off[:-1] < off[1:]]] = True
    assert np.all(state.cpu().numpy()[first] == pytest.approx(alone[first], rel=1e-5))
    assert np.all(state.cpu().numpy()[~first] < alone[~first])
    assert fsmi.device_status() == 0


def test_trajectories_repeat_and_determinism():
    grid = synth.office_grid(128, n_obst=20, seed=22)
    p = synth.free_cell_poses_2d(grid, 1, seed=23)
    poses = np.concatenate([p, p, p])
    dirs = synth.beam_dirs_2d(90)
    gp, op = _prms(fsmi.EXACT, 40.0)
    args = (_cuda(grid), _cuda(poses), _cuda(np.array([0, 3], np.int32)), _cuda(dirs), gp)
    beam, state, traj = fsmi.eval_trajectories_2d(*args)
    assert torch.all(beam[1:] == 0) and float(state[0]) > 0
    for s in (fsmi.Schedule(2, 0, -1, 0), fsmi.Schedule(8, 0, 3, 0)):
        fsmi.set_schedule(fsmi.KIND_2D, s)
        b2, s2, t2 = fsmi.eval_trajectories_2d(*args)
        assert torch.equal(b2, beam) and torch.equal(s2, state) and torch.equal(t2, traj)
    fsmi.set_schedule(fsmi.KIND_2D, None)


def test_uncovered_poses_are_flagged():
    grid = synth.office_grid(128, n_obst=20, seed=24)
    poses = synth.free_cell_poses_2d(grid, 5, seed=25)
    dirs = synth.beam_dirs_2d(16)
    gp, _ = _prms(fsmi.EXACT, 30.0)
    fsmi.device_status()
    beam, state, traj = fsmi.eval_trajectories_2d(_cuda(grid), _cuda(poses), _cuda(np.array([0, 2, 3], np.int32)),
                                                  _cuda(dirs), gp)
    beam = beam.cpu().numpy()
    assert np.isfinite(beam[:3]).all() and np.isnan(beam[3:]).all()
    assert np.isfinite(traj.cpu().numpy()).all()
    assert fsmi.device_status() & fsmi.STATUS_BAD_BEAM


def test_best_trajectory_and_scan_sums():
    grid = synth.office_grid(160, n_obst=25, seed=26)
    poses, off = _trajectories(grid, T=12, seed=27, step=9.0)
    dirs = synth.beam_dirs_2d(60)
    gp, op = _prms(fsmi.APPROX, 48.0)
    _, _, traj = fsmi.eval_trajectories_2d(_cuda(grid), _cuda(poses), _cuda(off), _cuda(dirs), gp)
    ratio, best = fsmi.best_trajectory(traj, _cuda(poses), _cuda(off))
    ratio = ratio.cpu().numpy()
    _, _, rt = oracle.eval_trajectories_2d(grid, poses, off, dirs, op)
    assert_mi_close(ratio, rt / oracle.path_lengths(poses, off), "MI per distance")
    # the argmax is taken on the GPU's own ratios: lowest index among the largest
    assert best == int(np.flatnonzero(ratio == ratio.max())[0])
    # scan sums
    out = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp)
    sums = fsmi.scan_sums(out).cpu().numpy()
    np.testing.assert_allclose(sums, out.cpu().numpy().astype(np.float64).sum(axis=1), rtol=2e-6, atol=1e-7)


# ---- eq. (1) --------------------------------------------------------------------------------------

def _measured_ranges(truth, poses, dirs, R, rng, noise=0.3):
    """Ranges a sensor would report on a binary map: the first occupied cell's middle plus noise;
    no return (inf) when nothing is hit within R; a few missing (NaN) readings."""
    H, W = truth.shape
    z = np.full((poses.shape[0], dirs.shape[0]), np.inf, np.float32)
    for p in range(poses.shape[0]):
        for b in range(dirs.shape[0]):
            d = oracle.beam_dir_2d(poses[p], dirs[b])
            cells, l = oracle.trace_2d(W, H, int(poses[p, 0]), int(poses[p, 1]), int(d[0]), int(d[1]), R)
            hit = np.flatnonzero(truth.reshape(-1)[cells])
            if len(hit):
                k = hit[0]
                z[p, b] = 0.5 * (l[k] + l[k + 1]) + rng.normal(0, noise)
    z[rng.random(z.shape) < 0.03] = np.nan
    return z


def test_update_map_matches_oracle():
    truth_src = synth.office_grid(192, n_obst=40, seed=31)
    truth = truth_src == np.float32(0.9)
    grid = np.full_like(truth_src, 0.5)
    grid[truth_src == np.float32(0.1)] = 0.4
    grid[:3, :3] = 0.0  # known cells stay put
    grid[-2:, -2:] = 1.0
    poses = synth.free_cell_poses_2d(truth_src, 6, seed=32)
    dirs = synth.beam_dirs_2d(180)
    rng = np.random.default_rng(33)
    R = 60.0
    z = _measured_ranges(truth, poses, dirs, R, rng)
    gp, op = _prms(fsmi.EXACT, R)
    g = _cuda(grid)
    fsmi.device_status()
    fsmi.update_map_2d(g, _cuda(poses), _cuda(dirs), _cuda(z), gp)
    got = g.cpu().numpy().astype(np.float64)
    ref = oracle.update_map_2d(grid, poses, dirs, z, op)
    # which cells moved, and in which direction, is decided by exact integer traversal
    np.testing.assert_array_equal(np.sign(got - grid), np.sign(ref - grid))
    # values: FP32 log-odds update against the FP64 beam-by-beam product
    tol = 1e-4 * ref * (1 - ref) + 3e-7
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (np.flatnonzero(bad)[:5], got.reshape(-1)[np.flatnonzero(bad)[:5]],
                           ref.reshape(-1)[np.flatnonzero(bad)[:5]])
    assert (got != grid).sum() > 1000
    assert fsmi.device_status() == 0


def test_update_then_information_drops():
    # closing the loop: after the robot scans from a pose and updates the map with what it
    # measured, the MI of scanning there again is lower
    truth_src = synth.office_grid(160, n_obst=30, seed=34)
    truth = truth_src == np.float32(0.9)
    grid = np.full_like(truth_src, 0.5)
    poses = synth.free_cell_poses_2d(truth_src, 1, seed=35)
    dirs = synth.beam_dirs_2d(360)
    z = _measured_ranges(truth, poses, dirs, 50.0, np.random.default_rng(36), noise=0.1)
    gp, _ = _prms(fsmi.EXACT, 50.0)
    g = _cuda(grid)
    before = float(fsmi.eval_2d(g, _cuda(poses), _cuda(dirs), gp).sum())
    for _ in range(3):
        fsmi.update_map_2d(g, _cuda(poses), _cuda(dirs), _cuda(z), gp)
    after = float(fsmi.eval_2d(g, _cuda(poses), _cuda(dirs), gp).sum())
    assert after < 0.5 * before


def test_update_invalid_arguments():
    g = torch.full((32, 32), 0.5, device="cuda")
    poses = _cuda(synth.pose_2d(3.5, 3.5)[None])
    dirs = _cuda(synth.beam_dirs_2d(4))
    gp, _ = _prms(fsmi.EXACT, 10.0)
    with pytest.raises(ValueError):
        fsmi.update_map_2d(g, poses, dirs, torch.ones(2, 4, device="cuda"), gp)
    with pytest.raises(fsmi.FsmiError):
        fsmi.update_map_2d(g, poses, dirs, torch.ones(1, 4, device="cuda"), gp,
                           ws=torch.empty(16, dtype=torch.uint8, device="cuda"))
