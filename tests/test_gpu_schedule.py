"""Launch schedules, the work queue, candidate sets, graph replay and the autotuner (fsmi_schedule,
fsmi_eval_2d_sets, fsmi_capture_*, fsmi_autotune), through the C ABI.

A schedule only changes which warp evaluates a beam and when, so every schedule must give the
same floats bit for bit, except the RLE cell-form threshold, which changes the summation order
(both forms are checked against the FP64 oracle)."""
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


@pytest.fixture(autouse=True)
def default_schedule():
    for k in (fsmi.KIND_2D, fsmi.KIND_RLE):
        fsmi.set_schedule(k, None)
    yield
    for k in (fsmi.KIND_2D, fsmi.KIND_RLE):
        fsmi.set_schedule(k, None)


K2, KR = fsmi.KIND_2D, fsmi.KIND_RLE


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bits(t):
    return t.cpu().numpy().view(np.uint32)


def _office(size=256, n_poses=24, seed=4):
    grid = synth.office_grid(size, n_obst=40, seed=seed)
    poses = synth.free_cell_poses_2d(grid, n_poses, seed=seed + 1)
    return grid, poses


def _prm2d(variant, R, **kw):
    base = dict(variant=variant, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=R, trunc_delta=6, uniform_h=4)
    base.update(kw)
    return fsmi.Params(**base), oracle.Params(**base)


VARIANTS_2D = (fsmi.EXACT, fsmi.APPROX, fsmi.UNIFORM)


def test_every_2d_schedule_gives_identical_bits():
    grid, poses = _office()
    dirs = synth.beam_dirs_2d(90)
    g, p, d = _cuda(grid), _cuda(poses), _cuda(dirs)
    scheds = fsmi.schedule_candidates(K2) + [fsmi.Schedule(1, 1, -1, 0), fsmi.Schedule(8, 1, 7, 0),
                                             fsmi.Schedule(3, 0, 1000, 0)]
    for var in VARIANTS_2D:
        gp, _ = _prm2d(var, 96.0)
        fsmi.set_schedule(K2, None)
        ref = fsmi.eval_2d(g, p, d, gp)
        for s in scheds:
            fsmi.set_schedule(K2, s)
            assert fsmi.get_schedule(K2).warps_per_block == s.warps_per_block
            got = fsmi.eval_2d(g, p, d, gp)
            np.testing.assert_array_equal(_bits(got), _bits(ref), err_msg=f"{var} {s}")
            got = fsmi.eval_2d(g, p, d, gp, ws=torch.empty(0, dtype=torch.uint8, device="cuda"))
            np.testing.assert_array_equal(_bits(got), _bits(ref), err_msg=f"{var} {s} no workspace")
    assert fsmi.device_status() == 0


def test_queued_explicit_beams_match_oracle():
    # very uneven beam lengths (1 .. 2000 cells): the case the work queue balances
    off, o, l, lend = synth.random_beams(200, 0, 2000, seed=61)
    ref_by_var = {}
    for var in VARIANTS_2D:
        gp, op = _prm2d(var, 1.0)
        ref_by_var[var] = oracle.eval_beams(off, o, l, lend, op)
    for s in (fsmi.Schedule(4, 0, -1, 0), fsmi.Schedule(4, 0, 1, 0), fsmi.Schedule(8, 0, 3, 0),
              fsmi.Schedule(2, 1, 16, 0)):
        fsmi.set_schedule(K2, s)
        for var in VARIANTS_2D:
            gp, _ = _prm2d(var, 1.0)
            got = fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp).cpu().numpy()
            assert_mi_close(got, ref_by_var[var], f"beams {var} {s}")


def test_rle_schedules_and_cell_form_threshold():
    off, ro, rl = synth.random_runs(300, 0, 60, 64, seed=62)
    rl = rl.copy()
    for r in range(300):
        a, b = off[r], off[r + 1]
        while rl[a:b].astype(int).sum() > 1024:
            rl[a:b] = np.maximum(1, rl[a:b] // 2)
    args = (_cuda(off), _cuda(ro), _cuda(rl))
    for kw in (dict(variant=fsmi.EXACT), dict(variant=fsmi.APPROX, approx_reading=1, trunc_delta=3),
               dict(variant=fsmi.APPROX, approx_reading=0, trunc_delta=3), dict(variant=fsmi.UNIFORM, uniform_h=4)):
        base = dict(sigma=1.5, delta_occ=1.5, delta_emp=0.67, max_range=1024.0, run_cap=64, trunc_delta=6,
                    uniform_h=4)
        base.update(kw)
        gp, op = fsmi.Params(**base), oracle.Params(**base)
        ref = oracle.eval_rle(off, ro, rl, op)
        # threshold 1: every ray on the run-pair path; 100000: every ray (but Theorem 5's) per cell
        for runlen in (1, 100000):
            fsmi.set_schedule(KR, fsmi.Schedule(cell_runlen=runlen))
            first = fsmi.eval_rle(*args, gp)
            assert_mi_close(first.cpu().numpy(), ref, f"rle {kw} runlen={runlen}")
            for s in (fsmi.Schedule(2, 0, -1, runlen), fsmi.Schedule(8, 0, 1, runlen), fsmi.Schedule(4, 2, 5, runlen)):
                fsmi.set_schedule(KR, s)
                np.testing.assert_array_equal(_bits(fsmi.eval_rle(*args, gp)), _bits(first), err_msg=f"{kw} {s}")


def test_eval_3d_schedules_identical_and_match_oracle():
    vox = synth.voxel_world(64, 48, 32, n_boxes=12, seed=5, noise_seed=6, noise_frac=0.05)
    poses = synth.free_voxel_poses(vox, 5, seed=7, zlo=4, zhi=28)
    dirs = synth.pinhole_dirs(10, 8, 100.0)
    base = dict(variant=fsmi.EXACT, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=80.0, run_cap=16)
    gp, op = fsmi.Params(**base), oracle.Params(**base)
    ref, _ = oracle.eval_3d(vox, poses, dirs, op)
    v, p, d = _cuda(vox), _cuda(poses), _cuda(dirs)
    first = fsmi.eval_3d(v, p, d, gp)
    assert_mi_close(first.cpu().numpy(), ref, "3d default")
    for s in fsmi.schedule_candidates(KR):
        fsmi.set_schedule(KR, s)
        got = fsmi.eval_3d(v, p, d, gp)
        if s.cell_runlen == 32:  # the default threshold: same path for every ray as `first`
            np.testing.assert_array_equal(_bits(got), _bits(first), err_msg=str(s))
        else:
            assert_mi_close(got.cpu().numpy(), ref, f"3d {s}")


# ---- candidate sets -----------------------------------------------------------------------------

def _sets_case():
    grid, poses = _office(256, 40, seed=11)
    rng = np.random.default_rng(12)
    dirs = np.concatenate([synth.beam_dirs_2d(360), synth.random_dirs_2d(64, rng)])
    # (pose_offset, npose, dir_offset, nbeam, max_range): lengths 8 .. 200 cells, beam counts 360 or 64
    sets = [(0, 3, 0, 360, 8.0), (3, 16, 0, 360, 200.0), (19, 1, 360, 64, 37.25), (20, 0, 0, 360, 50.0),
            (20, 20, 360, 64, 128.0), (5, 2, 7, 5, 0.5)]
    return grid, poses, dirs, sets


@pytest.mark.parametrize("variant", VARIANTS_2D)
def test_sets_equal_separate_calls_and_oracle(variant):
    grid, poses, dirs, sets = _sets_case()
    g, p, d = _cuda(grid), _cuda(poses), _cuda(dirs)
    st, nb = fsmi.make_sets_2d(sets, "cuda")
    gp, _ = _prm2d(variant, 200.0)
    for s in (fsmi.Schedule(4, 0, -1, 0), fsmi.Schedule(8, 0, 2, 0)):
        fsmi.set_schedule(K2, s)
        got = fsmi.eval_2d_sets(g, p, d, st, nb, gp).cpu().numpy()
        at = 0
        for po, npose, do, nbeam, rng in sets:
            gps, ops = _prm2d(variant, rng)
            sep = fsmi.eval_2d(g, p[po:po + npose], d[do:do + nbeam], gps).cpu().numpy().reshape(-1)
            np.testing.assert_array_equal(got[at:at + sep.size].view(np.uint32), sep.view(np.uint32),
                                          err_msg=f"set {po, npose, do, nbeam, rng} {s}")
            if npose and s.queue_chunk < 0:
                ref = oracle.eval_2d(grid, poses[po:po + min(npose, 2)], dirs[do:do + nbeam], ops).reshape(-1)
                assert_mi_close(got[at:at + ref.size], ref, f"set oracle {variant} {rng}")
            at += sep.size
        assert at == nb
    assert fsmi.device_status() == 0


def test_malformed_sets_give_nan_and_status():
    grid, poses, dirs, _ = _sets_case()
    g, p, d = _cuda(grid), _cuda(poses), _cuda(dirs)
    gp, _ = _prm2d(fsmi.EXACT, 64.0)
    bad = [(0, 1, 0, 4, 16.0),      # fine
           (38, 4, 0, 4, 16.0),     # poses 40, 41 past P = 40
           (0, 1, 420, 8, 16.0),    # directions 424 .. 427 past B = 424
           (0, 1, 0, 4, 64.5),      # range above the call's max_range
           (0, 1, 0, 4, -1.0),      # non-positive range
           (0, 1, 0, 4, 16.0)]      # fine
    st, nb = fsmi.make_sets_2d(bad, "cuda")
    fsmi.device_status()
    got = fsmi.eval_2d_sets(g, p, d, st, nb + 3, gp).cpu().numpy()  # 3 beams beyond the last set
    assert np.isfinite(got[:4]).all()
    # poses 38, 39 are valid, 40, 41 are not
    assert np.isfinite(got[4:12]).all() and np.isnan(got[12:20]).all()
    assert np.isfinite(got[20:24]).all() and np.isnan(got[24:28]).all()
    assert np.isnan(got[28:36]).all()
    assert np.isfinite(got[36:40]).all() and np.isnan(got[40:43]).all()
    assert fsmi.device_status() & fsmi.STATUS_BAD_BEAM
    assert fsmi.device_status() == 0


# ---- graphs and the autotuner -------------------------------------------------------------------

def test_graph_replay_of_sets_and_3d():
    grid, poses, dirs, sets = _sets_case()
    g, p, d = _cuda(grid), _cuda(poses), _cuda(dirs)
    st, nb = fsmi.make_sets_2d(sets, "cuda")
    gp2, _ = _prm2d(fsmi.EXACT, 200.0)
    vox = synth.voxel_world(64, 48, 32, n_boxes=12, seed=13, noise_seed=14, noise_frac=0.05)
    vposes = synth.free_voxel_poses(vox, 4, seed=15, zlo=4, zhi=28)
    vdirs = synth.pinhole_dirs(8, 8, 90.0)
    v, vp, vd = _cuda(vox), _cuda(vposes), _cuda(vdirs)
    gp3 = fsmi.Params(variant=fsmi.APPROX, sigma=2.0, trunc_delta=6, max_range=80.0, run_cap=16)
    fsmi.set_schedule(K2, fsmi.Schedule(4, 0, 2, 0))  # queued: the captured memsets must reset the counters
    fsmi.set_schedule(KR, fsmi.Schedule(2, 0, 3, 0))
    out2 = torch.empty(nb, dtype=torch.float32, device="cuda")
    out3 = torch.empty((vp.shape[0], vd.shape[0]), dtype=torch.float32, device="cuda")
    ws2 = torch.empty(fsmi.workspace_size(fsmi.FN_EVAL_2D, g.numel()), dtype=torch.uint8, device="cuda")
    ws3 = torch.empty(fsmi.QUEUE_BYTES, dtype=torch.uint8, device="cuda")

    def step():
        fsmi.eval_2d_sets(g, p, d, st, nb, gp2, out=out2, ws=ws2)
        fsmi.eval_3d(v, vp, vd, gp3, out=out3, ws=ws3)

    graph = fsmi.Graph(step)
    for it in range(3):
        # move the poses between replays: the graph reads the same buffers each time
        p.copy_(_cuda(np.roll(poses, it, axis=0)))
        vp.copy_(_cuda(np.roll(vposes, it, axis=0)))
        out2.fill_(-1.0)
        out3.fill_(-1.0)
        graph.replay()
        torch.cuda.synchronize()
        ref2 = fsmi.eval_2d_sets(g, p, d, st, nb, gp2)
        ref3 = fsmi.eval_3d(v, vp, vd, gp3)
        np.testing.assert_array_equal(_bits(out2), _bits(ref2))
        np.testing.assert_array_equal(_bits(out3), _bits(ref3))
    graph.close()
    assert fsmi.device_status() == 0


def test_benchmark_launch_configuration_against_oracle():
    # exactly what the benchmark times: the 2048x2048 office batch at full size with the per-cell gains workspace,
    # the autotuned 2D schedule and one CUDA-graph replay per step; the 512x512x128 voxel batch likewise for the 3D
    # batch. The replayed results equal a plain call bit for bit and match the oracle on samples.
    grid, poses, dirs = synth.office_scene()
    g, p, d = _cuda(grid), _cuda(poses), _cuda(dirs)
    gp = fsmi.Params(variant=fsmi.EXACT, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=256.0)
    op = oracle.Params(variant=oracle.EXACT, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=256.0)
    out = torch.empty((1024, 360), dtype=torch.float32, device="cuda")
    ws = torch.empty(fsmi.workspace_size(fsmi.FN_EVAL_2D, g.numel()), dtype=torch.uint8, device="cuda")
    saved2, saved3 = fsmi.get_schedule(K2), fsmi.get_schedule(KR)
    try:
        fsmi.autotune(K2, lambda: fsmi.eval_2d(g, p, d, gp, out=out, ws=ws), reps=1)
        graph = fsmi.Graph(lambda: fsmi.eval_2d(g, p, d, gp, out=out, ws=ws))
        out.fill_(-1.0)
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
        graph.close()
        plain = fsmi.eval_2d(g, p, d, gp)
        np.testing.assert_array_equal(_bits(out), _bits(plain))
        rows = [5, 517, 1000]
        assert_mi_close(out.cpu().numpy()[rows], oracle.eval_2d(grid, poses[rows], dirs, op), "office graph")

        vox, vposes, vdirs = synth.voxel_scene()
        v, vp, vd = _cuda(vox), _cuda(vposes), _cuda(vdirs)
        gp3 = fsmi.Params(variant=fsmi.EXACT, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=384.0, run_cap=64)
        op3 = oracle.Params(variant=oracle.EXACT, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=384.0, run_cap=64)
        out3 = torch.empty((64, vd.shape[0]), dtype=torch.float32, device="cuda")
        ws3 = torch.empty(fsmi.QUEUE_BYTES, dtype=torch.uint8, device="cuda")
        fsmi.autotune(KR, lambda: fsmi.eval_3d(v, vp, vd, gp3, out=out3, ws=ws3), reps=1)
        graph3 = fsmi.Graph(lambda: fsmi.eval_3d(v, vp, vd, gp3, out=out3, ws=ws3))
        graph3.replay()
        torch.cuda.synchronize()
        graph3.close()
        np.testing.assert_array_equal(_bits(out3), _bits(fsmi.eval_3d(v, vp, vd, gp3)))
        sel_r = np.arange(0, vd.shape[0], 257)
        ref3, _ = oracle.eval_3d(vox, vposes[[3, 40]], vdirs[sel_r], op3)
        assert_mi_close(out3.cpu().numpy()[np.ix_([3, 40], sel_r)], ref3, "voxel scene graph")
    finally:
        fsmi.set_schedule(K2, saved2)
        fsmi.set_schedule(KR, saved3)
    assert fsmi.device_status() == 0


def test_autotune_picks_a_candidate_and_sets_it():
    grid, poses = _office(256, 32, seed=21)
    g, p, d = _cuda(grid), _cuda(poses), _cuda(synth.beam_dirs_2d(180))
    gp, _ = _prm2d(fsmi.EXACT, 128.0)
    out = torch.empty((p.shape[0], d.shape[0]), dtype=torch.float32, device="cuda")
    ws = torch.empty(fsmi.workspace_size(fsmi.FN_EVAL_2D, g.numel()), dtype=torch.uint8, device="cuda")
    best, cands, ms = fsmi.autotune(K2, lambda: fsmi.eval_2d(g, p, d, gp, out=out, ws=ws), reps=2)
    assert best in cands
    assert all(t > 0 for t in ms)
    assert ms[cands.index(best)] == min(ms)
    assert fsmi.get_schedule(K2) == best
    assert fsmi.get_schedule(KR) == fsmi.Schedule(2, 0, 4, 32)  # the other family is untouched
    ref = fsmi.eval_2d(g, p, d, gp)
    fsmi.set_schedule(K2, None)
    np.testing.assert_array_equal(_bits(ref), _bits(fsmi.eval_2d(g, p, d, gp)))


def test_autotune_skips_failing_candidates():
    grid, poses = _office(128, 4, seed=22)
    g, p, d = _cuda(grid), _cuda(poses), _cuda(synth.beam_dirs_2d(16))
    gp, _ = _prm2d(fsmi.EXACT, 32.0)
    calls = []

    def fn():
        s = fsmi.get_schedule(K2)
        calls.append(s)
        if s.warps_per_block == 2:
            raise fsmi.FsmiError("rejected")
        fsmi.eval_2d(g, p, d, gp)

    cands = [fsmi.Schedule(2, 0, -1, 0), fsmi.Schedule(4, 0, -1, 0)]
    best, _, ms = fsmi.autotune(K2, fn, cands, reps=1)
    assert best == fsmi.Schedule(4, 0, -1, 32) and ms[0] == -1.0 and ms[1] > 0
    fsmi.set_schedule(K2, fsmi.Schedule(8, 0, 0, 0))
    with pytest.raises(fsmi.FsmiError):
        fsmi.autotune(K2, fn, cands[:1], reps=1)
    assert fsmi.get_schedule(K2) == fsmi.Schedule(8, 0, 1, 32)  # left as it was


def test_pipeline_2d_equals_separate_calls():
    # consecutive submits alternate between two device buffer sets; each result must be the floats
    # of its own inputs (not of the batch before it), whatever the overlap of copies and evaluation
    grid, _ = _office(size=256)
    dirs = synth.beam_dirs_2d(90)
    prm, _ = _prm2d(fsmi.EXACT, 96.0)
    P = 12
    batches = [synth.free_cell_poses_2d(grid, P, seed=20 + i) for i in range(5)]
    hg = torch.from_numpy(grid).pin_memory()
    hd = torch.from_numpy(dirs).pin_memory()
    pipe = fsmi.Pipeline2D(prm, grid.shape[1], grid.shape[0], P, dirs.shape[0])
    outs = [torch.empty((P, dirs.shape[0]), dtype=torch.float32).pin_memory() for _ in batches]
    hp = [torch.from_numpy(b).pin_memory() for b in batches]  # alive until the copies have run
    for p, o in zip(hp, outs):
        pipe.submit(hg, p, hd, o)
    pipe.wait()
    for b, o in zip(batches, outs):
        ref = fsmi.eval_2d(_cuda(grid), _cuda(b), _cuda(dirs), prm).cpu()
        assert torch.equal(o, ref)
    with pytest.raises(ValueError):
        pipe.submit(hg.cuda(), torch.from_numpy(batches[0]), hd, outs[0])
