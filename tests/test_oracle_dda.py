"""Pins of the oracle's fixed-point 2D ray traversal (the cells a beam intersects, ordered by
distance, Section 2.2; boundaries l_i with l_1 = 0, Section 3.1) against exact rational geometry
and closed-form cell lists."""
import numpy as np
import pytest

from paper_1905_02238_gb300 import synth
from tests.bruteforce import exact_cells


def _check(orc, W, H, ox, oy, dx, dy, R):
    cells, l = orc.trace_2d(W, H, ox, oy, dx, dy, R)
    ref_cells, ref_l, ref_end = exact_cells(W, H, ox, oy, dx, dy, orc.range_fix(R) / 65536.0)
    assert list(cells) == ref_cells
    np.testing.assert_allclose(l[:-1], ref_l, rtol=0, atol=1e-12)
    assert l[-1] == pytest.approx(ref_end, abs=1e-12)


def test_random_rays_match_exact_geometry(orc):
    rng = np.random.default_rng(11)
    W, H = 9, 7
    for _ in range(300):
        ox = int(rng.integers(0, W * 65536))
        oy = int(rng.integers(0, H * 65536))
        d = synth.random_dirs_2d(1, rng)[0]
        R = float(rng.choice([0.5, 2.0, 4.75, 20.0]))
        _check(orc, W, H, ox, oy, int(d[0]), int(d[1]), R)


def test_rays_from_cell_corners_and_edges(orc):
    # origins on grid lines and corners, directions with exact ties (45 degrees, axis-aligned)
    rng = np.random.default_rng(12)
    W, H = 8, 8
    dirs = [(1 << 30, 0), (-(1 << 30), 0), (0, 1 << 30), (0, -(1 << 30)), (759250125, 759250125),
            (-759250125, 759250125), (759250125, -759250125), (-759250125, -759250125),
            (1 << 29, 1 << 30), (-(1 << 30), 1 << 29)]
    for _ in range(60):
        ox = int(rng.integers(0, W + 1)) * 65536 if rng.random() < 0.5 else int(rng.integers(0, W * 65536))
        oy = int(rng.integers(0, H + 1)) * 65536 if rng.random() < 0.5 else int(rng.integers(0, H * 65536))
        ox, oy = min(ox, W * 65536 - 1), min(oy, H * 65536 - 1)
        for dx, dy in dirs:
            _check(orc, W, H, ox, oy, dx, dy, 6.0)


def test_axis_aligned_closed_form(orc):
    # +x beam from (2.25, 3.5): cells (2,3), (3,3), ... with entries 0, 0.75, 1.75, ...
    W, H = 10, 6
    cells, l = orc.trace_2d(W, H, int(2.25 * 65536), int(3.5 * 65536), 1 << 30, 0, 5.0)
    assert list(cells) == [3 * W + x for x in range(2, 8)]
    np.testing.assert_allclose(l, [0, 0.75, 1.75, 2.75, 3.75, 4.75, 5.0])
    # exits the grid before the range ends
    cells, l = orc.trace_2d(W, H, int(2.25 * 65536), int(3.5 * 65536), 1 << 30, 0, 50.0)
    assert list(cells) == [3 * W + x for x in range(2, 10)]
    assert l[-1] == pytest.approx(7.75)


def test_diagonal_ties_step_both_axes(orc):
    # 45 degrees from a cell centre: every crossing is a tie, so the beam steps diagonally and
    # never visits the two cells that touch it only at a corner.
    d = 759250125  # round(2^30 / sqrt(2))
    cells, l = orc.trace_2d(20, 20, int(5.5 * 65536), int(5.5 * 65536), d, d, 6.0)
    assert list(cells) == [(5 + i) * 20 + (5 + i) for i in range(len(cells))]
    assert len(cells) == 5


def test_zero_direction_and_outside_origin(orc):
    cells, l = orc.trace_2d(5, 5, 65536 * 2, 65536 * 2, 0, 0, 4.0)
    assert len(cells) == 0
    # on the left edge moving left: the first cell is outside the grid
    cells, l = orc.trace_2d(5, 5, 0, 65536 * 2 + 5, -(1 << 30), 0, 4.0)
    assert len(cells) == 0


def test_beam_direction_rotation(orc):
    # yaw 0 leaves the unit vector unchanged; yaw 90 degrees maps (1, 0) to (0, 1)
    dirs = synth.beam_dirs_2d(360)
    p0 = synth.pose_2d(1.0, 1.0, 0.0)
    for b in range(0, 360, 7):
        np.testing.assert_array_equal(orc.beam_dir_2d(p0, dirs[b]), dirs[b])
    p90 = synth.pose_2d(1.0, 1.0, np.pi / 2)
    assert list(orc.beam_dir_2d(p90, dirs[0])) == [0, 1 << 30]
