"""GPU parity of the 3D / RLE path (fsmi_rle_encode_3d, fsmi_eval_rle, fsmi_eval_3d) against the
FP64 oracle, through the C ABI. Run decompositions bit for bit; MI within tests/parity.py."""
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


def _prms(**kw):
    base = dict(sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=384.0, run_cap=64, trunc_delta=6, uniform_h=4)
    base.update(kw)
    return fsmi.Params(**base), oracle.Params(**base)


def _rle_variants():
    return [
        dict(variant=fsmi.EXACT, g_kernel=fsmi.G_PDF),
        dict(variant=fsmi.EXACT, g_kernel=fsmi.G_ERF),
        dict(variant=fsmi.APPROX, approx_reading=0, trunc_delta=0),
        dict(variant=fsmi.APPROX, approx_reading=0, trunc_delta=3),
        dict(variant=fsmi.APPROX, approx_reading=0, trunc_delta=6),
        dict(variant=fsmi.APPROX, approx_reading=1, trunc_delta=3),
        dict(variant=fsmi.APPROX, approx_reading=0, trunc_delta=6, g_kernel=fsmi.G_ERF),
        dict(variant=fsmi.UNIFORM, uniform_h=0),
        dict(variant=fsmi.UNIFORM, uniform_h=2),
        dict(variant=fsmi.UNIFORM, uniform_h=4),
        dict(variant=fsmi.APPROX, approx_reading=1, trunc_delta=6),  # kernel radius 6 (register taps)
    ]


def _small_world(seed=0):
    vox = synth.voxel_world(64, 48, 32, n_boxes=12, seed=seed, noise_seed=seed + 1, noise_frac=0.05)
    poses = synth.free_voxel_poses(vox, 6, seed=seed + 2, zlo=4, zhi=28)
    dirs = synth.pinhole_dirs(12, 10, 100.0)
    return vox, poses, dirs


def _oracle_runs(vox, poses, dirs, nsamp, cap):
    offs, ros, rls = [0], [], []
    for p in range(poses.shape[0]):
        for r in range(dirs.shape[0]):
            s = oracle.sample_3d(vox, poses[p], dirs[r], nsamp)
            ro, rl = oracle.rle_encode(s, cap)
            ros.append(ro)
            rls.append(rl)
            offs.append(offs[-1] + len(ro))
    return np.array(offs, np.int32), np.concatenate(ros), np.concatenate(rls)


@pytest.mark.parametrize("cap", [64, 5, 1])
def test_encode_bit_exact(cap):
    vox, poses, dirs = _small_world()
    gp, _ = _prms(max_range=80.0, run_cap=cap)
    roff, ro_ref, rl_ref = _oracle_runs(vox, poses, dirs, 80, cap)
    off, ro, rl = fsmi.rle_encode_3d(_cuda(vox), _cuda(poses), _cuda(dirs), gp, capacity=int(roff[-1]) + 7)
    off, ro, rl = off.cpu().numpy(), ro.cpu().numpy(), rl.cpu().numpy()
    np.testing.assert_array_equal(off, roff)
    n = int(roff[-1])
    np.testing.assert_array_equal(ro[:n].view(np.uint32), ro_ref.view(np.uint32))
    np.testing.assert_array_equal(rl[:n], rl_ref)
    assert fsmi.device_status() == 0


def test_encode_capacity_overflow_is_flagged_and_bounded():
    vox, poses, dirs = _small_world(1)
    gp, _ = _prms(max_range=80.0, run_cap=8)
    roff, ro_ref, rl_ref = _oracle_runs(vox, poses, dirs, 80, 8)
    cap = int(roff[-1]) // 2
    fsmi.device_status()
    # place the run buffers inside larger guard buffers and check the guards stay untouched
    off, ro, rl = fsmi.rle_encode_3d(_cuda(vox), _cuda(poses), _cuda(dirs), gp, capacity=cap)
    assert fsmi.device_status() & fsmi.STATUS_RUN_OVERFLOW
    np.testing.assert_array_equal(off.cpu().numpy(), roff)
    np.testing.assert_array_equal(rl.cpu().numpy()[:cap], rl_ref[:cap])


def test_encode_offsets_saturate_instead_of_wrapping_past_int32():
    # 2,101,250 rays along +x through a 1024-voxel-long grid, 1024 virtual cells each, runs of one
    # cell: 2.15e9 runs in all, more than an int32 offset holds. The offsets past INT32_MAX must
    # saturate there (never wrap negative) and the overflow must be flagged.
    X, P, R = 1024, 2050, 1025
    vox = np.random.default_rng(3).uniform(0.2, 0.8, (4, 4, X)).astype(np.float32)
    pose = np.zeros((P, 12), np.int32)
    pose[:, 0] = 1 << 14  # x = 0.25 (Q16): samples at x = i + 0.75, i = 0 .. 1023
    pose[:, 1] = pose[:, 2] = 5 << 15  # y = z = 2.5
    pose[:, 3] = pose[:, 7] = pose[:, 11] = 1 << 30  # identity rotation (Q30)
    dirs = np.zeros((R, 3), np.int32)
    dirs[:, 0] = 1 << 30
    gp, _ = _prms(max_range=1024.0, run_cap=1)
    fsmi.device_status()
    off, _, _ = fsmi.rle_encode_3d(_cuda(vox), _cuda(pose), _cuda(dirs), gp, capacity=0)
    assert fsmi.device_status() & fsmi.STATUS_RUN_OVERFLOW
    want = np.minimum(np.arange(P * R + 1, dtype=np.int64) * 1024, 2**31 - 1)
    np.testing.assert_array_equal(off.cpu().numpy().astype(np.int64), want)


def test_encode_full_size_voxel_scene_sampled():
    vox, poses, dirs = synth.voxel_scene()
    gp, _ = _prms()
    rng = np.random.default_rng(50)
    sel_p = rng.choice(64, 4, replace=False)
    sel_r = rng.choice(dirs.shape[0], 64, replace=False)
    # GPU encodes the whole benchmark batch; the oracle re-encodes sampled rays
    off, ro, rl = fsmi.rle_encode_3d(_cuda(vox), _cuda(poses), _cuda(dirs), gp, capacity=64 * 16384 * 96)
    off, ro, rl = off.cpu().numpy(), ro.cpu().numpy(), rl.cpu().numpy()
    assert fsmi.device_status() == 0
    for p in sel_p:
        for r in sel_r:
            i = p * dirs.shape[0] + r
            s = oracle.sample_3d(vox, poses[p], dirs[r], 384)
            ro_ref, rl_ref = oracle.rle_encode(s, 64)
            a, b = off[i], off[i + 1]
            np.testing.assert_array_equal(ro[a:b].view(np.uint32), ro_ref.view(np.uint32))
            np.testing.assert_array_equal(rl[a:b], rl_ref)


@pytest.mark.parametrize("sigma", [0.7, 2.0, 3.5])
def test_eval_rle_random_runs(sigma):
    off, ro, rl = synth.random_runs(400, 0, 50, 64, seed=int(sigma * 10))
    rl = rl.copy()
    # keep each ray within the 1024-virtual-cell maximum of the call below
    for r in range(400):
        a, b = off[r], off[r + 1]
        while rl[a:b].astype(int).sum() > 1024:
            rl[a:b] = np.maximum(1, rl[a:b] // 2)
    for kw in _rle_variants():
        gp, op = _prms(sigma=sigma, max_range=1024.0, **kw)
        got = fsmi.eval_rle(_cuda(off), _cuda(ro), _cuda(rl), gp).cpu().numpy()
        ref = oracle.eval_rle(off, ro, rl, op)
        assert_mi_close(got, ref, f"rle {kw} sigma={sigma}")


@pytest.mark.parametrize("L", [1, 2, 4, 8, 16, 32, 64, 128])
def test_eval_rle_e5_groups(L):
    # Section 5.4 shapes: n = 256 virtual cells in groups of L
    off, ro, rl = synth.e5_runs(L, nbeams=200)
    for kw in (dict(variant=fsmi.EXACT), dict(variant=fsmi.APPROX, trunc_delta=3), dict(variant=fsmi.UNIFORM, uniform_h=2)):
        gp, op = _prms(sigma=1.5, max_range=256.0, **kw)
        got = fsmi.eval_rle(_cuda(off), _cuda(ro), _cuda(rl), gp).cpu().numpy()
        ref = oracle.eval_rle(off, ro, rl, op)
        assert_mi_close(got, ref, f"e5 L={L} {kw}")


def test_eval_rle_edge_cases():
    # empty ray, one run, known runs (o in {0, 1}), long runs of 255, x = 0 and x = 1
    rays = [([], []), ([0.5], [1]), ([0.0, 1.0, 0.0], [3, 2, 9]), ([0.3] * 4, [255, 255, 255, 255]),
            ([1.0], [7]), ([0.0], [100]), ([0.999, 0.001, 0.5], [64, 64, 64])]
    off = np.concatenate([[0], np.cumsum([len(r[0]) for r in rays])]).astype(np.int32)
    ro = np.concatenate([np.array(r[0], np.float32) for r in rays]).astype(np.float32)
    rl = np.concatenate([np.array(r[1], np.uint8) for r in rays]).astype(np.uint8)
    for kw in _rle_variants():
        gp, op = _prms(max_range=1024.0, **kw)
        got = fsmi.eval_rle(_cuda(off), _cuda(ro), _cuda(rl), gp).cpu().numpy()
        ref = oracle.eval_rle(off, ro, rl, op)
        assert_mi_close(got, ref, f"rle edge {kw}")
        assert got[0] == 0.0 and abs(got[2]) <= 1e-7


def test_eval_rle_bad_ray_sets_status():
    off = np.array([0, 2, 3], np.int32)
    ro = np.array([0.5, 0.2, 0.4], np.float32)
    rl = np.array([200, 200, 0], np.uint8)  # ray 0 covers 400 > 256 cells; ray 1 has a zero-length run
    gp, _ = _prms(max_range=256.0)
    fsmi.device_status()
    got = fsmi.eval_rle(_cuda(off), _cuda(ro), _cuda(rl), gp).cpu().numpy()
    assert np.isnan(got).all()
    assert fsmi.device_status() & fsmi.STATUS_BAD_BEAM


def test_eval_3d_small_world_all_variants():
    vox, poses, dirs = _small_world(3)
    for kw in _rle_variants():
        gp, op = _prms(max_range=80.0, run_cap=16, **kw)
        got, nr = fsmi.eval_3d(_cuda(vox), _cuda(poses), _cuda(dirs), gp, with_runs=True)
        ref, nr_ref = oracle.eval_3d(vox, poses, dirs, op)
        np.testing.assert_array_equal(nr.cpu().numpy(), nr_ref)
        assert_mi_close(got.cpu().numpy(), ref, f"3d {kw}")


def test_eval_3d_voxel_scene_full_size_sampled():
    # the benchmark's launch: 512x512x128 voxels, 64 poses x 128x128 rays, 384 virtual cells
    vox, poses, dirs = synth.voxel_scene()
    rng = np.random.default_rng(51)
    sel_p = rng.choice(64, 3, replace=False)
    sel_r = np.sort(rng.choice(dirs.shape[0], 96, replace=False))
    for kw in (dict(variant=fsmi.EXACT), dict(variant=fsmi.APPROX, trunc_delta=6),
               dict(variant=fsmi.APPROX, trunc_delta=6, approx_reading=1), dict(variant=fsmi.UNIFORM, uniform_h=4)):
        gp, op = _prms(**kw)
        got, nr = fsmi.eval_3d(_cuda(vox), _cuda(poses), _cuda(dirs), gp, with_runs=True)
        got, nr = got.cpu().numpy(), nr.cpu().numpy()
        assert np.all(np.isfinite(got))
        ref, nr_ref = oracle.eval_3d(vox, poses[sel_p], dirs[sel_r], op)
        np.testing.assert_array_equal(nr[np.ix_(sel_p, sel_r)], nr_ref)
        assert_mi_close(got[np.ix_(sel_p, sel_r)], ref, f"voxel scene {kw}")
    assert fsmi.device_status() == 0


def test_fused_equals_encode_then_eval():
    vox, poses, dirs = _small_world(5)
    for kw in _rle_variants()[:6]:
        gp, _ = _prms(max_range=80.0, run_cap=16, **kw)
        fused = fsmi.eval_3d(_cuda(vox), _cuda(poses), _cuda(dirs), gp).reshape(-1)
        off, ro, rl = fsmi.rle_encode_3d(_cuda(vox), _cuda(poses), _cuda(dirs), gp, capacity=200000)
        n = int(off[-1].item())
        two = fsmi.eval_rle(off, ro[:n].contiguous(), rl[:n].contiguous(), gp)
        torch.testing.assert_close(fused, two, rtol=0, atol=0)
