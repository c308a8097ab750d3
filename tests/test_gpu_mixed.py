"""One persistent launch over a stream of 2D and 3D candidate sets (fsmi_eval_mixed): every set's
values equal the separate fsmi_eval_2d / fsmi_eval_3d call bit for bit (and the oracle within the
parity tolerance); malformed descriptors give NaN and a status bit; completion times are recorded."""
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


def _bits(a):
    return np.asarray(a.cpu() if isinstance(a, torch.Tensor) else a, np.float32).view(np.uint32)


def _case():
    grid = synth.office_grid(256, n_obst=40, seed=41)
    poses2 = synth.free_cell_poses_2d(grid, 30, seed=42)
    rng = np.random.default_rng(43)
    dirs2 = np.concatenate([synth.beam_dirs_2d(360), synth.random_dirs_2d(64, rng)])
    vols = [synth.voxel_world(64, 48, 32, n_boxes=12, seed=s, noise_seed=s + 1, noise_frac=0.05) for s in (3, 5)]
    poses3 = np.concatenate([synth.free_voxel_poses(vols[0], 4, seed=5, zlo=4, zhi=28),
                             synth.free_voxel_poses(vols[1], 4, seed=7, zlo=4, zhi=28)])
    dirs3 = np.concatenate([synth.pinhole_dirs(16, 12, 100.0), synth.pinhole_dirs(8, 8, 60.0)])
    return grid, poses2, dirs2, vols, poses3, dirs3


def _prms():
    b2 = dict(variant=fsmi.EXACT, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=200.0)
    b3 = dict(variant=fsmi.APPROX, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=80.0, run_cap=16,
              trunc_delta=6)
    return b2, b3


SETS = [(fsmi.SET_2D, 0, 3, 0, 360, 8.0), (fsmi.SET_3D, 0, 2, 0, 192, 80.0, 0), (fsmi.SET_2D, 3, 10, 0, 360, 200.0),
        (fsmi.SET_3D, 4, 3, 0, 192, 33.7, 1), (fsmi.SET_2D, 13, 1, 360, 64, 37.25), (fsmi.SET_3D, 0, 0, 0, 192, 50.0, 0),
        (fsmi.SET_3D, 7, 1, 192, 64, 8.0, 1), (fsmi.SET_2D, 20, 10, 360, 64, 128.0), (fsmi.SET_2D, 5, 2, 7, 5, 0.5)]


@pytest.mark.parametrize("variant2", [fsmi.EXACT, fsmi.APPROX, fsmi.UNIFORM])
def test_mixed_sets_equal_separate_calls(variant2):
    grid, poses2, dirs2, vols, poses3, dirs3 = _case()
    b2, b3 = _prms()
    b2 = dict(b2, variant=variant2, trunc_delta=6, uniform_h=4)
    g, p2, d2, p3, d3 = (_cuda(x) for x in (grid, poses2, dirs2, poses3, dirs3))
    vt = [_cuda(v) for v in vols]
    vd = fsmi.make_volumes(vt, "cuda")
    st, n = fsmi.make_sets(SETS, "cuda")
    times = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    fsmi.device_status()
    out = fsmi.eval_mixed(st, n, times=times, grid=g, poses2=p2, dirs2=d2, prm2=fsmi.Params(**b2), volumes=vd,
                          poses3=p3, dirs3=d3, prm3=fsmi.Params(**b3)).cpu().numpy()
    assert fsmi.device_status() == 0
    at = 0
    for s in SETS:
        kind, po, npose, do, ndir, rng = s[:6]
        if kind == fsmi.SET_2D:
            sep = fsmi.eval_2d(g, p2[po:po + npose], d2[do:do + ndir], fsmi.Params(**dict(b2, max_range=rng)))
        else:
            sep = fsmi.eval_3d(vt[s[6]], p3[po:po + npose], d3[do:do + ndir], fsmi.Params(**dict(b3, max_range=rng)))
        sep = sep.cpu().numpy().reshape(-1)
        np.testing.assert_array_equal(_bits(out[at:at + sep.size]), _bits(sep), err_msg=str(s))
        at += sep.size
    assert at == n
    # oracle on one set of each kind
    ref2 = oracle.eval_2d(grid, poses2[3:5], dirs2[:360], oracle.Params(**b2)).reshape(-1)
    o2 = sum(npose * ndir for (_, _, npose, _, ndir, *_) in SETS[:2])
    assert_mi_close(out[o2:o2 + ref2.size], ref2, "mixed 2D vs oracle")
    ref3, _ = oracle.eval_3d(vols[1], poses3[4:5], dirs3[:192], oracle.Params(**dict(b3, max_range=33.7)))
    o3 = sum(npose * ndir for (_, _, npose, _, ndir, *_) in SETS[:3])
    assert_mi_close(out[o3:o3 + 192], ref3.reshape(-1), "mixed 3D vs oracle")
    # completion times: after the start, one per item
    t = times.cpu().numpy().view(np.uint64)
    assert np.all(t[1:] >= t[0]) and t[0] > 0
    # the same call without room for the range-class plan: one launch, the same floats
    ws1 = torch.empty(fsmi.workspace_size(fsmi.FN_EVAL_2D, g.numel()), dtype=torch.uint8, device="cuda")
    assert ws1.numel() < fsmi.mixed_workspace_size(g.numel(), st.shape[0])
    one = fsmi.eval_mixed(st, n, ws=ws1, grid=g, poses2=p2, dirs2=d2, prm2=fsmi.Params(**b2), volumes=vd, poses3=p3,
                          dirs3=d3, prm3=fsmi.Params(**b3)).cpu().numpy()
    np.testing.assert_array_equal(_bits(one), _bits(out))


def test_mixed_plan_over_every_range_class():
    # sets in every 2D and 3D range class (up to 64 ... 1024 cells), interleaved in the stream: the
    # planned call (one launch per class) equals the single launch bit for bit, and the separate calls
    grid = synth.office_grid(512, n_obst=60, seed=44)
    poses2 = synth.free_cell_poses_2d(grid, 24, seed=45)
    dirs2 = synth.beam_dirs_2d(90)
    vol = synth.voxel_world(96, 80, 48, n_boxes=16, seed=9, noise_seed=10, noise_frac=0.05)
    poses3 = synth.free_voxel_poses(vol, 6, seed=11, zlo=6, zhi=40)
    dirs3 = synth.pinhole_dirs(12, 10, 100.0)
    g, p2, d2, p3, d3 = (_cuda(x) for x in (grid, poses2, dirs2, poses3, dirs3))
    vt = [_cuda(vol)]
    vd = fsmi.make_volumes(vt, "cuda")
    b2 = dict(variant=fsmi.EXACT, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=1000.0)
    b3 = dict(variant=fsmi.EXACT, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=1000.0, run_cap=64)
    sets = [(fsmi.SET_2D, 0, 2, 0, 90, 700.0), (fsmi.SET_3D, 0, 2, 0, 120, 20.0, 0), (fsmi.SET_2D, 2, 3, 0, 90, 40.0),
            (fsmi.SET_3D, 2, 1, 0, 120, 300.0, 0), (fsmi.SET_2D, 5, 2, 0, 90, 100.0), (fsmi.SET_3D, 3, 1, 0, 120, 900.0, 0),
            (fsmi.SET_2D, 7, 2, 0, 90, 250.0), (fsmi.SET_3D, 4, 1, 0, 120, 100.0, 0), (fsmi.SET_2D, 9, 2, 0, 90, 400.0),
            (fsmi.SET_3D, 5, 1, 0, 120, 200.0, 0), (fsmi.SET_2D, 11, 2, 0, 90, 64.0), (fsmi.SET_3D, 0, 1, 0, 120, 64.0, 0)]
    st, n = fsmi.make_sets(sets, "cuda")
    kw = dict(grid=g, poses2=p2, dirs2=d2, prm2=fsmi.Params(**b2), volumes=vd, poses3=p3, dirs3=d3,
              prm3=fsmi.Params(**b3))
    fsmi.device_status()
    planned = fsmi.eval_mixed(st, n, **kw).cpu().numpy()
    ws1 = torch.empty(fsmi.workspace_size(fsmi.FN_EVAL_2D, g.numel()), dtype=torch.uint8, device="cuda")
    single = fsmi.eval_mixed(st, n, ws=ws1, **kw).cpu().numpy()
    assert fsmi.device_status() == 0
    np.testing.assert_array_equal(_bits(planned), _bits(single))
    at = 0
    for s in sets:
        kind, po, npose, do, ndir, rng = s[:6]
        if kind == fsmi.SET_2D:
            sep = fsmi.eval_2d(g, p2[po:po + npose], d2[do:do + ndir], fsmi.Params(**dict(b2, max_range=rng)))
        else:
            sep = fsmi.eval_3d(vt[0], p3[po:po + npose], d3[do:do + ndir], fsmi.Params(**dict(b3, max_range=rng)))
        sep = sep.cpu().numpy().reshape(-1)
        np.testing.assert_array_equal(_bits(planned[at:at + sep.size]), _bits(sep), err_msg=str(s))
        at += sep.size
    assert at == n


def test_mixed_malformed_sets_and_single_kind():
    grid, poses2, dirs2, vols, poses3, dirs3 = _case()
    b2, b3 = _prms()
    g, p2, d2, p3, d3 = (_cuda(x) for x in (grid, poses2, dirs2, poses3, dirs3))
    vt = [_cuda(v) for v in vols]
    vd = fsmi.make_volumes(vt, "cuda")
    bad = [(fsmi.SET_2D, 0, 1, 0, 4, 16.0),          # fine
           (fsmi.SET_2D, 28, 4, 0, 4, 16.0),         # poses 30, 31 past P2 = 30
           (fsmi.SET_3D, 0, 1, 0, 4, 81.0, 0),       # more virtual cells than prm3 allows
           (fsmi.SET_3D, 0, 1, 0, 4, 20.0, 2),       # no volume 2
           (fsmi.SET_3D, 0, 1, 254, 4, 20.0, 0),     # directions 256, 257 past R3 = 256
           (fsmi.SET_3D, 0, 1, 0, 4, 20.0, 1)]       # fine
    st, n = fsmi.make_sets(bad, "cuda")
    fsmi.device_status()
    out = fsmi.eval_mixed(st, n, grid=g, poses2=p2, dirs2=d2, prm2=fsmi.Params(**b2), volumes=vd, poses3=p3,
                          dirs3=d3, prm3=fsmi.Params(**b3)).cpu().numpy()
    assert n == 36
    assert np.isfinite(out[:12]).all() and np.isnan(out[12:20]).all()  # poses 28, 29 valid; 30, 31 not
    assert np.isnan(out[20:28]).all()                                  # range and volume out of bounds
    assert np.isfinite(out[28:30]).all() and np.isnan(out[30:32]).all()  # directions 254, 255 valid
    assert np.isfinite(out[32:36]).all()
    assert fsmi.device_status() & fsmi.STATUS_BAD_BEAM
    # only 3D sets, no 2D parameters: a 2D set is refused per item
    only3 = [(fsmi.SET_3D, 0, 2, 0, 192, 60.0, 0), (fsmi.SET_2D, 0, 1, 0, 4, 16.0)]
    st, n = fsmi.make_sets(only3, "cuda")
    out = fsmi.eval_mixed(st, n, volumes=vd, poses3=p3, dirs3=d3, prm3=fsmi.Params(**b3)).cpu().numpy()
    sep = fsmi.eval_3d(vt[0], p3[:2], d3[:192], fsmi.Params(**dict(b3, max_range=60.0))).cpu().numpy().reshape(-1)
    np.testing.assert_array_equal(_bits(out[:384]), _bits(sep))
    assert np.isnan(out[384:]).all()
    assert fsmi.device_status() & fsmi.STATUS_BAD_BEAM
