"""Pins of the surrogate's CPU oracle (oracle/surrogate.py): the convolution against its
definition written as loops, gradients against central differences, the profile sampler against
exact rational geometry, BF16 rounding against torch, one Adam step against its closed form."""
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import surrogate as S
from paper_1905_02238_gb300 import synth


def test_layout():
    assert S.n_params() == 192 + 32 + 3072 + 32 + 3072 + 32 + 262144 + 256 + 256 + 1
    th = np.arange(S.n_params(), dtype=np.float64)
    p = S.unflatten(th)
    assert p["W4"].shape == (256, 1024) and p["b5"][0] == S.n_params() - 1


def test_conv_is_the_definition():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 10, 3))
    W = rng.normal(size=(4, 3, 3))
    b = rng.normal(size=4)
    got = S.conv(x, W, b)
    ref = np.zeros((2, 5, 4))
    for n in range(2):
        for t in range(5):
            for c in range(4):
                acc = b[c]
                for k in range(3):
                    s = 2 * t + k - 1
                    if 0 <= s < 10:
                        for ci in range(3):
                            acc += W[c, k, ci] * x[n, s, ci]
                ref[n, t, c] = acc
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    theta = S.init_params(3).astype(np.float64)
    theta += rng.normal(0, 0.01, theta.shape)  # non-zero biases
    x = np.stack([np.stack([rng.uniform(0, 1, 256), (rng.random(256) < 0.9).astype(float)], 1) for _ in range(3)])
    y = rng.uniform(0, 2, 3)

    def loss(th):
        pred, _ = S.forward(th, x, bf16_weights=False)
        return S.mse(pred, y)[0]

    pred, cache = S.forward(theta, x, bf16_weights=False)
    g = S.backward(cache, S.mse(pred, y)[1])
    off = S.offsets()
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4", "W5", "b5"):
        o, shape = off[name]
        n = int(np.prod(shape))
        for i in rng.choice(n, min(n, 6), replace=False):
            e = np.zeros_like(theta)
            e[o + i] = h
            fd = (loss(theta + e) - loss(theta - e)) / (2 * h)
            assert abs(fd - g[o + i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (name, i, fd, g[o + i])


def test_profile_is_exact_geometry():
    grid = synth.office_grid(96, n_obst=10, seed=2)
    rng = np.random.default_rng(4)
    poses = synth.free_cell_poses_2d(grid, 4, seed=5)
    dirs = synth.random_dirs_2d(6, rng)
    for p in poses:
        for u in dirs:
            prof = S.profile_2d(grid, p, u, 150)
            c, s = int(p[2]), int(p[3])
            d = [(c * int(u[0]) - s * int(u[1]) + (1 << 29)) >> 30, (s * int(u[0]) + c * int(u[1]) + (1 << 29)) >> 30]
            for i in range(0, 150, 7):
                px = Fraction(int(p[0]), 1 << 16) + Fraction(2 * i + 1, 2) * Fraction(d[0], 1 << 30)
                py = Fraction(int(p[1]), 1 << 16) + Fraction(2 * i + 1, 2) * Fraction(d[1], 1 << 30)
                cx, cy = px.__floor__(), py.__floor__()
                inside = 0 <= cx < 96 and 0 <= cy < 96
                assert prof[i, 1] == float(inside)
                assert prof[i, 0] == (float(grid[cy, cx]) if inside else 0.0)
    # axis-aligned: from the centre of cell (x0, y0) along +x, sample i lies in cell x0 + i + 1
    g = np.arange(20 * 20, dtype=np.float32).reshape(20, 20) / 400.0
    prof = S.profile_2d(g, synth.pose_2d(3.5, 7.5, 0.0), synth.q30(np.array([1.0, 0.0])), 20)
    np.testing.assert_array_equal(prof[:16, 0], g[7, 4:20])
    assert np.all(prof[16:] == 0)


def test_profile_range_cut_is_a_map_that_ends_there():
    # a beam cut at range R sees the cells of a map cropped just past R: along +x from (3.5, 7.5)
    # sample i lies at x = 4 + i, inside the range when i + 1/2 < R
    g = np.arange(30 * 30, dtype=np.float32).reshape(30, 30) / 900.0 + 0.01
    pose, u = synth.pose_2d(3.5, 7.5, 0.0), synth.q30(np.array([1.0, 0.0]))
    for R in (0.4, 0.5, 0.6, 7.0, 7.5, 7.51, 12.25, 25.5):
        cut = S.profile_2d(g, pose, u, 40, max_range=R)
        keep = int(np.ceil(R - 0.5))  # samples i with i + 1/2 < R
        cropped = S.profile_2d(g[:, :4 + keep], pose, u, 40)
        np.testing.assert_array_equal(cut, cropped)
        full = S.profile_2d(g, pose, u, 40)
        np.testing.assert_array_equal(cut[:keep], full[:keep])
        assert np.all(cut[keep:] == 0)
    np.testing.assert_array_equal(S.profile_2d(g, pose, u, 40, max_range=0.0), S.profile_2d(g, pose, u, 40))


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(6)
    a = np.concatenate([rng.normal(0, 10, 1000), rng.normal(0, 1e-3, 1000), [0.0, -0.0, 1.0, 3.0e38, -3.4e38]])
    a = a.astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(S.bf16_round(a), ref)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(7)
    th, g = rng.normal(size=50), rng.normal(size=50)
    new, m, v = S.adam(th, np.zeros(50), np.zeros(50), g, 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(new, th - 0.01 * np.sign(g), rtol=1e-14)
    np.testing.assert_allclose(m, 0.1 * g) and np.testing.assert_allclose(v, 0.001 * g * g)
