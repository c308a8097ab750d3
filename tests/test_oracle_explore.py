"""Pins of the oracle's exploration-loop functions (CPU): the skip mask of already-counted cells
(Section 2.4), trajectory aggregation, and the Bayesian map update of eq. (1) with the inverse
sensor model of Section 2.2."""
import math

import numpy as np
import pytest

import oracle
from paper_1905_02238_gb300 import synth
from tests.bruteforce import smi_integral


def _beam(rng, n):
    o = rng.uniform(0.02, 0.98, n)
    w = rng.uniform(0.3, 1.4, n)
    l = np.concatenate([[0.0], np.cumsum(w)])
    return o, l


VARS = [dict(variant=oracle.EXACT, sigma=0.8), dict(variant=oracle.APPROX, sigma=0.8, trunc_delta=2),
        dict(variant=oracle.UNIFORM, uniform_h=1)]


@pytest.mark.parametrize("kw", VARS)
def test_skip_is_additive_over_cells(orc, kw):
    # eq. (mi_sum): the beam MI is a sum over cells, so leaving out S and leaving out its
    # complement must add up to leaving out nothing
    rng = np.random.default_rng(3)
    prm = oracle.Params(delta_occ=1.5, delta_emp=0.67, **kw)
    for n in (1, 2, 5, 17, 40):
        o, l = _beam(rng, n)
        full = oracle.fsmi_beam(o, l, prm)
        S = rng.random(n) < 0.4
        a = oracle.fsmi_beam_skip(o, l, S, prm)
        b = oracle.fsmi_beam_skip(o, l, ~S, prm)
        assert abs(a + b - full) <= 1e-12 * max(1.0, abs(full))
        assert oracle.fsmi_beam_skip(o, l, np.zeros(n, bool), prm) == full
        assert oracle.fsmi_beam_skip(o, l, np.ones(n, bool), prm) == 0.0


@pytest.mark.parametrize("sigma", [0.4, 1.1])
def test_skip_matches_numerical_integral(orc, sigma):
    # the integral of eq. (mi_sum) with the skipped cells' f(delta, r) left out of F(z)
    rng = np.random.default_rng(5)
    prm = oracle.Params(variant=oracle.EXACT, sigma=sigma, delta_occ=1.5, delta_emp=0.67)
    for n in (3, 6, 8):
        o, l = _beam(rng, n)
        S = rng.random(n) < 0.5
        ref = smi_integral(o, l, sigma, 1.5, 0.67, skip=S)
        got = oracle.fsmi_beam_skip(o, l, S, prm)
        assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref)), (got, ref)


def _small_map(seed=2):
    g = synth.office_grid(96, n_obst=12, unknown_cover=0.3, seed=seed)
    return g


def _prm(**kw):
    base = dict(variant=oracle.EXACT, sigma=1.5, delta_occ=1.5, delta_emp=0.67, max_range=30.0, trunc_delta=4,
                uniform_h=2)
    base.update(kw)
    return oracle.Params(**base)


def test_single_state_trajectory_is_the_scan(orc):
    g = _small_map()
    poses = synth.free_cell_poses_2d(g, 3, seed=4)
    dirs = synth.beam_dirs_2d(24)
    prm = _prm()
    beam, state, traj = oracle.eval_trajectories_2d(g, poses, np.array([0, 1, 2, 3]), dirs, prm)
    ref = oracle.eval_2d(g, poses, dirs, prm)
    np.testing.assert_array_equal(beam, ref)
    np.testing.assert_allclose(state, ref.sum(axis=1), rtol=1e-14)
    np.testing.assert_allclose(traj, state, rtol=0)


def test_repeated_state_adds_nothing(orc):
    g = _small_map()
    p = synth.free_cell_poses_2d(g, 1, seed=6)
    poses = np.concatenate([p, p, p])
    dirs = synth.beam_dirs_2d(36)
    for kw in VARS:
        prm = _prm(**kw)
        beam, state, traj = oracle.eval_trajectories_2d(g, poses, np.array([0, 3]), dirs, prm)
        assert state[0] > 0 and np.all(beam[1:] == 0.0)
        assert traj[0] == state[0]


def test_disjoint_states_add_and_marks_follow_travel_order(orc):
    g = _small_map(7)
    poses = synth.free_cell_poses_2d(g, 40, seed=8)
    # two states farther apart than twice the range: no cell in common
    far = [(i, j) for i in range(40) for j in range(40)
           if np.hypot(*((poses[i, :2] - poses[j, :2]) / 65536.0)) > 2 * 12 + 3]
    i, j = far[0]
    dirs = synth.beam_dirs_2d(30)
    prm = _prm(max_range=12.0)
    pp = poses[[i, j]]
    _, state, traj = oracle.eval_trajectories_2d(g, pp, np.array([0, 2]), dirs, prm)
    ref = oracle.eval_2d(g, pp, dirs, prm).sum(axis=1)
    np.testing.assert_allclose(state, ref, rtol=1e-14)
    # an overlapping pair: the later state loses exactly the cells the earlier one crossed,
    # restated here with the traversal and the skip mask beam by beam
    near = [(a, b) for a in range(40) for b in range(40)
            if a != b and 2 < np.hypot(*((poses[a, :2] - poses[b, :2]) / 65536.0)) < 8]
    a, b = near[0]
    pp = poses[[a, b]]
    beam, state, _ = oracle.eval_trajectories_2d(g, pp, np.array([0, 2]), dirs, prm)
    seen = set()
    for s in range(2):
        for k in range(dirs.shape[0]):
            d = oracle.beam_dir_2d(pp[s], dirs[k])
            cells, l = oracle.trace_2d(g.shape[1], g.shape[0], int(pp[s, 0]), int(pp[s, 1]), int(d[0]), int(d[1]), 12.0)
            skip = np.array([c in seen for c in cells], bool)
            ref = oracle.fsmi_beam_skip(g.reshape(-1)[cells].astype(np.float64), l, skip, prm)
            assert beam[s, k] == ref
        for k in range(dirs.shape[0]):
            d = oracle.beam_dir_2d(pp[s], dirs[k])
            cells, _ = oracle.trace_2d(g.shape[1], g.shape[0], int(pp[s, 0]), int(pp[s, 1]), int(d[0]), int(d[1]), 12.0)
            seen.update(cells.tolist())
    assert state[1] < oracle.eval_2d(g, pp[1:], dirs, prm).sum()


def test_path_lengths(orc):
    poses = np.zeros((5, 4), np.int32)
    poses[:, 0] = np.array([0, 3, 3, 10, 10]) * 65536
    poses[:, 1] = np.array([0, 4, 4, 0, 0]) * 65536
    np.testing.assert_allclose(oracle.path_lengths(poses, [0, 3, 3, 4, 5]), [5.0, 1.0, 1.0, 1.0])


# ---- eq. (1) --------------------------------------------------------------------------------------

def _axis_case(W=40, H=20):
    g = np.full((H, W), 0.5, np.float32)
    pose = synth.pose_2d(5.5, 10.5, 0.0)[None]
    dirs = synth.q30(np.array([[1.0, 0.0]]))
    return g, pose, dirs


def test_update_single_beam_closed_form(orc):
    g, pose, dirs = _axis_case()
    prm = _prm(max_range=30.0)
    # cell 5 + k is entered at k - 1/2 (k >= 1); a range of 10.25 ends in cell 15
    m = oracle.update_map_2d(g, pose, dirs, np.array([[10.25]], np.float32), prm)
    row = m[10]
    emp = 0.5 * 0.67 / (1 + 0.5 * (0.67 - 1))
    occ = 0.5 * 1.5 / (1 + 0.5 * 0.5)
    np.testing.assert_allclose(row[5:15], emp, rtol=1e-15)
    assert abs(row[15] - occ) < 1e-15 and abs(occ - 0.6) < 1e-15
    assert np.all(row[16:] == 0.5) and np.all(row[:5] == 0.5)
    assert np.all(np.delete(m, 10, axis=0) == 0.5)


def test_update_no_return_outside_and_invalid(orc):
    g, pose, dirs = _axis_case()
    prm = _prm(max_range=30.0)
    emp = 0.5 * 0.67 / (1 + 0.5 * (0.67 - 1))
    for z in (30.0, 31.0, np.inf):  # no return: every cell entered below the range is crossed
        row = oracle.update_map_2d(g, pose, dirs, np.array([[z]], np.float32), prm)[10]
        np.testing.assert_allclose(row[5:36], emp, rtol=1e-15)  # cell 35 is entered at 29.5
        assert np.all(row[36:] == 0.5)
    # a range ending beyond the grid (x = 40 is 34.5 cells away): crossed cells only, no hit
    prm = _prm(max_range=60.0)
    row = oracle.update_map_2d(g, pose, dirs, np.array([[50.0]], np.float32), prm)[10]
    np.testing.assert_allclose(row[5:], emp, rtol=1e-15)
    for z in (np.nan, 0.0, -3.0):
        np.testing.assert_array_equal(oracle.update_map_2d(g, pose, dirs, np.array([[z]], np.float32), prm), g)


def test_update_repeated_and_commuting(orc):
    g = _small_map(9)
    g[g == np.float32(0.1)] = 0.0  # known-free cells must not move
    g[0, 0] = 1.0
    poses = synth.free_cell_poses_2d(synth.office_grid(96, n_obst=12, unknown_cover=0.3, seed=9), 4, seed=10)
    dirs = synth.beam_dirs_2d(45)
    rng = np.random.default_rng(11)
    ranges = rng.uniform(0.5, 25.0, (4, 45)).astype(np.float32)
    prm = _prm(max_range=20.0)
    m = oracle.update_map_2d(g, poses, dirs, ranges, prm)
    assert np.all(m[g == 0.0] == 0.0) and m[0, 0] == 1.0
    # the same beams in another order (poses and beams permuted) give the same map
    pi, bi = rng.permutation(4), rng.permutation(45)
    m2 = oracle.update_map_2d(g, poses[pi], dirs[bi], ranges[pi][:, bi], prm)
    np.testing.assert_allclose(m2, m, rtol=1e-13, atol=1e-15)
    # k identical hits on one cell: odds times delta_occ^k
    gg, pose, d1 = _axis_case()
    k = 7
    mk = oracle.update_map_2d(gg, np.repeat(pose, k, 0), d1, np.full((k, 1), 10.25, np.float32), prm)
    r = 1.0 * 1.5 ** k
    assert abs(mk[10, 15] - r / (1 + r)) < 1e-14
