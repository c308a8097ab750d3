"""GPU parity of the 2D path (fsmi_trace_2d, fsmi_eval_beams, fsmi_eval_2d) against the FP64
oracle, through the C ABI. Cell lists bit for bit; MI within the tolerance of tests/parity.py."""
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


def _variants():
    return [
        dict(variant=fsmi.EXACT),
        dict(variant=fsmi.APPROX, trunc_delta=0),
        dict(variant=fsmi.APPROX, trunc_delta=3),
        dict(variant=fsmi.APPROX, trunc_delta=6),
        dict(variant=fsmi.UNIFORM, uniform_h=0),
        dict(variant=fsmi.UNIFORM, uniform_h=2),
        dict(variant=fsmi.UNIFORM, uniform_h=4),
    ]


def _prms(sigma, R, e0=0, **kw):
    base = dict(sigma=sigma, delta_occ=1.5, delta_emp=0.67, max_range=R, e0_mode=e0)
    base.update(kw)
    return fsmi.Params(**base), oracle.Params(**{k: v for k, v in base.items() if k != "flags"})


# ---- traversal ------------------------------------------------------------------------------------

def _trace_compare(W, H, poses, dirs, R):
    cap = int(R * 1.5) + 4
    cells, l, n = fsmi.trace_2d(W, H, _cuda(poses), _cuda(dirs), R, cap)
    cells, l, n = cells.cpu().numpy(), l.cpu().numpy(), n.cpu().numpy()
    B = dirs.shape[0]
    for i in range(poses.shape[0] * B):
        p, b = divmod(i, B)
        d = oracle.beam_dir_2d(poses[p], dirs[b])
        rc, rl = oracle.trace_2d(W, H, int(poses[p, 0]), int(poses[p, 1]), int(d[0]), int(d[1]), R, cap)
        assert n[i] == len(rc), (i, n[i], len(rc))
        np.testing.assert_array_equal(cells[i, :n[i]], rc)
        np.testing.assert_allclose(l[i, :n[i] + 1], rl, rtol=4e-7, atol=1e-6)


def test_trace_random_grid_bit_exact():
    grid, poses, dirs = synth.random_grid_200()
    _trace_compare(200, 200, poses, dirs, 64.0)


def test_trace_random_poses_bit_exact():
    rng = np.random.default_rng(40)
    W, H = 61, 47
    poses = []
    for k in range(24):
        x = rng.integers(0, W * 65536) if k % 3 else rng.integers(0, W) * 65536  # some on grid lines
        y = rng.integers(0, H * 65536) if k % 4 else rng.integers(0, H) * 65536
        yaw = rng.uniform(0, 2 * np.pi) if k % 5 else 0.0
        p = synth.pose_2d(0, 0, yaw)
        p[0], p[1] = x, y
        poses.append(p)
    poses = np.stack(poses)
    dirs = np.concatenate([synth.beam_dirs_2d(72), synth.random_dirs_2d(40, rng)])
    _trace_compare(W, H, poses, dirs, 40.5)


def test_trace_lattice_diagonals_bit_exact():
    # directions with exact integer slope ratios from cell centres and corners: minor crossings
    # coincide with major ones (diagonal steps) all along the beam, which moves the cell offsets
    # of every later lane of the warp
    W, H = 64, 48
    poses = []
    for ix, iy, frac in ((5, 7, 0.5), (30, 20, 0.5), (12, 40, 0.0), (63, 0, 0.5), (0, 47, 0.0), (33, 9, 0.25)):
        p = synth.pose_2d(0, 0, 0.0)
        p[0], p[1] = int((ix + frac) * 65536), int((iy + frac) * 65536)
        poses.append(p)
    poses = np.stack(poses)
    ratios = [(1, 1), (-1, 1), (1, -1), (-1, -1), (2, 1), (1, 2), (-2, 1), (3, 2), (2, -3), (4, 1), (1, 0), (0, -1)]
    dirs = []
    for a, b in ratios:  # near-unit Q30 vectors with an exact integer ratio a : b
        c = int(round(2 ** 30 / np.hypot(a, b)))
        dirs.append([a * c, b * c])
    dirs = np.array(dirs, np.int32)
    _trace_compare(W, H, poses, dirs, 60.0)
    _trace_compare(W, H, poses, dirs, 9.0)


def test_trace_tight_capacity():
    # capacity exactly the beam's cell count, and one less: along lattice diagonals the lanes'
    # predicted counts include the diagonal steps, so their total exceeds the capacity and the
    # traversal writes with its capacity checks; one cell short, the beam reports the overflow (-1)
    W, H = 64, 48
    p = synth.pose_2d(0, 0, 0.0)
    p[0], p[1] = int(30.5 * 65536), int(20.5 * 65536)
    poses = p[None, :]
    c = int(round(2 ** 30 / np.sqrt(2.0)))
    dirs = np.array([[c, c], [-c, c], [2 * int(round(2 ** 30 / np.sqrt(5.0))), int(round(2 ** 30 / np.sqrt(5.0)))],
                     [2 ** 30, 0]], np.int32)
    R = 40.0
    for b in range(dirs.shape[0]):
        d = oracle.beam_dir_2d(poses[0], dirs[b])
        rc, rl = oracle.trace_2d(W, H, int(poses[0, 0]), int(poses[0, 1]), int(d[0]), int(d[1]), R, 4096)
        m = len(rc)
        cells, l, n = fsmi.trace_2d(W, H, _cuda(poses), _cuda(dirs[b:b + 1]), R, m)
        n = n.cpu().numpy()
        assert n[0] == m, (b, n[0], m)
        np.testing.assert_array_equal(cells.cpu().numpy()[0, :m], rc)
        np.testing.assert_allclose(l.cpu().numpy()[0, :m + 1], rl, rtol=4e-7, atol=1e-6)
        _, _, n = fsmi.trace_2d(W, H, _cuda(poses), _cuda(dirs[b:b + 1]), R, m - 1)
        assert int(n.cpu().numpy()[0]) == -1, b


def test_trace_office_map_sampled():
    grid, poses, dirs = synth.office_scene(n_poses=16, size=512)
    _trace_compare(512, 512, poses, dirs, 256.0)


# ---- explicit beams ---------------------------------------------------------------------------------

@pytest.mark.parametrize("sigma", [0.5, 1.5, 2.0, 5.0])
@pytest.mark.parametrize("e0", [0, 1])
def test_eval_beams_all_variants(sigma, e0):
    off, o, l, lend = synth.random_beams(300, 0, 420, seed=int(sigma * 10) + e0)
    for kw in _variants():
        gp, op = _prms(sigma, 64.0, e0, **kw)
        got = fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp).cpu().numpy()
        ref = oracle.eval_beams(off, o, l, lend, op)
        assert_mi_close(got, ref, f"beams {kw} sigma={sigma} e0={e0}")


@pytest.mark.parametrize("e0", [0, 1])
def test_exact_windows_wider_than_padding_and_longer_than_cells(e0):
    # sigma = 20 cells: a slot's window holds ~100 boundaries on each side, more than the 32 padding
    # boundaries beyond a beam's ends, so lanes near the ends run shorter loops than the round;
    # cells of 30-60 at sigma = 0.5: windows that end inside the slot's own cell
    for sigma, (wlo, whi), seed in ((20.0, (0.05, 1.4142), 91), (0.5, (30.0, 60.0), 92)):
        off, o, l, lend = synth.random_beams(120, 1, 400, seed=seed + e0, w_lo=wlo, w_hi=whi)
        gp, op = _prms(sigma, 4096.0, e0)
        got = fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp).cpu().numpy()
        assert_mi_close(got, oracle.eval_beams(off, o, l, lend, op), f"wide windows sigma={sigma} e0={e0}")
        gp.flags = fsmi.FLAG_FULL_SWEEP
        full = fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp).cpu().numpy()
        assert np.all(np.abs(got.astype(np.float64) - full) <= 2.0 ** -20 * np.abs(full) + 1e-9)


def test_eval_beams_edge_cases():
    # empty beams, single cells, known cells (o in {0, 1}), tiny and wide cells, long beams
    rng = np.random.default_rng(41)
    beams = [np.zeros(0), np.array([0.5]), np.array([0.0]), np.array([1.0]), rng.integers(0, 2, 50).astype(float),
             rng.uniform(0, 1, 1000), np.full(700, 0.1), np.full(64, 0.999)]
    widths = [np.zeros(0), np.array([1.0]), np.array([0.3]), np.array([2.0]), rng.uniform(0.01, 1.4, 50),
              rng.uniform(0.001, 1.4, 1000), np.ones(700), rng.uniform(0.5, 1.5, 64)]
    off = np.concatenate([[0], np.cumsum([len(b) for b in beams])]).astype(np.int32)
    o = np.concatenate(beams).astype(np.float32)
    l = np.concatenate([np.concatenate([[0.0], np.cumsum(w)])[:-1] for w in widths]).astype(np.float32)
    lend = np.array([np.sum(w) for w in widths], np.float32)
    for kw in _variants():
        for e0 in (0, 1):
            gp, op = _prms(1.5, 64.0, e0, **kw)
            got = fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp).cpu().numpy()
            ref = oracle.eval_beams(off, o, l, lend, op)
            assert_mi_close(got, ref, f"edge {kw} e0={e0}")
            assert got[0] == 0.0 and abs(got[4]) <= 1e-7


# ---- full 2D path -----------------------------------------------------------------------------------

@pytest.mark.parametrize("e0", [0, 1])
def test_eval_2d_random_grid(e0):
    grid, poses, dirs = synth.random_grid_200()
    for kw in _variants():
        gp, op = _prms(1.5, 64.0, e0, **kw)
        got = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp).cpu().numpy()
        ref = oracle.eval_2d(grid, poses, dirs, op)
        assert_mi_close(got, ref, f"random grid {kw}")


def test_eval_2d_office_midsize():
    grid, poses, dirs = synth.office_scene(n_poses=12, size=512)
    for kw in (dict(variant=fsmi.EXACT), dict(variant=fsmi.APPROX, trunc_delta=6), dict(variant=fsmi.UNIFORM, uniform_h=4)):
        gp, op = _prms(2.0, 256.0, 0, **kw)
        got = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp).cpu().numpy()
        ref = oracle.eval_2d(grid, poses, dirs, op)
        assert_mi_close(got, ref, f"office512 {kw}")


def test_eval_2d_office_full_size_sampled():
    # the benchmark's launch: 2048^2 map, 1024 poses x 360 beams, R = 256, sigma = 2; the oracle
    # checks every beam of four poses spread over the batch
    grid, poses, dirs = synth.office_scene()
    rows = [0, 341, 682, 1023]
    for kw in (dict(variant=fsmi.EXACT), dict(variant=fsmi.APPROX, trunc_delta=6), dict(variant=fsmi.UNIFORM, uniform_h=4)):
        gp, op = _prms(2.0, 256.0, 0, **kw)
        got = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp).cpu().numpy()
        assert got.shape == (1024, 360) and np.all(np.isfinite(got))
        ref = oracle.eval_2d(grid, poses[rows], dirs, op)
        assert_mi_close(got[rows], ref, f"office {kw}")
    assert fsmi.device_status() == 0


def test_eval_2d_long_beams():
    # R = 1024 cells: beams of up to ~1450 cells take several register-blocked passes
    grid = synth.office_grid(2048, seed=5)
    poses = synth.free_cell_poses_2d(grid, 3, seed=6, margin=700)
    dirs = synth.beam_dirs_2d(24)
    for kw in (dict(variant=fsmi.EXACT), dict(variant=fsmi.APPROX, trunc_delta=6), dict(variant=fsmi.UNIFORM, uniform_h=4)):
        gp, op = _prms(2.0, 1024.0, 1, **kw)
        got = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp).cpu().numpy()
        ref = oracle.eval_2d(grid, poses, dirs, op)
        assert_mi_close(got, ref, f"long {kw}")


def test_eval_2d_host_buffers_match_device():
    grid, poses, dirs = synth.random_grid_200()
    gp, _ = _prms(1.5, 64.0)
    dev = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp).cpu()
    host = fsmi.eval_2d(torch.from_numpy(grid).pin_memory(), torch.from_numpy(poses).pin_memory(),
                        torch.from_numpy(dirs).pin_memory(), gp)
    assert not host.is_cuda
    assert torch.equal(dev, host)


def test_invalid_arguments_launch_nothing():
    grid, poses, dirs = synth.random_grid_200()
    out = torch.full((1, 360), 7.0, device="cuda")
    for bad in (dict(sigma=0.0), dict(sigma=float("nan")), dict(delta_occ=-1.0), dict(max_range=2000.0),
                dict(variant=7), dict(e0_mode=3)):
        gp, _ = _prms(1.5, 64.0)
        for k, v in bad.items():
            setattr(gp, k, v)
        with pytest.raises(fsmi.FsmiError):
            fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp, out=out)
    torch.cuda.synchronize()
    assert torch.all(out == 7.0)
    # an empty batch is a no-op
    gp, _ = _prms(1.5, 64.0)
    assert fsmi.eval_2d(_cuda(grid), _cuda(poses[:0]), _cuda(dirs), gp).shape == (0, 360)


@pytest.mark.parametrize("e0", [0, 1])
def test_eval_beams_at_the_cell_limit(e0):
    # beams of exactly FSMI_MAX_CELLS cells: the per-warp arrays and their padding at full extent
    rng = np.random.default_rng(60 + e0)
    nb, n = 4, 2048
    w = rng.uniform(0.05, 1.4142, (nb, n))
    w[:, rng.random(n) < 0.02] = 0.0  # a few zero-length cells
    edges = np.concatenate([np.zeros((nb, 1)), np.cumsum(w, axis=1)], axis=1).astype(np.float32)
    off = (np.arange(nb + 1) * n).astype(np.int32)
    o = rng.uniform(0.0, 1.0, nb * n).astype(np.float32)
    l = edges[:, :n].reshape(-1).copy()
    lend = edges[:, n].copy()
    for kw in _variants():
        gp, op = _prms(2.0, 64.0, e0, **kw)
        got = fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp).cpu().numpy()
        assert_mi_close(got, oracle.eval_beams(off, o, l, lend, op), f"limit {kw} e0={e0}")
    gp, _ = _prms(2.0, 64.0, e0)
    gp.flags = fsmi.FLAG_FULL_WINDOW
    win = fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp)
    gp.flags = fsmi.FLAG_FULL_SWEEP
    assert torch.equal(win, fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp))
    assert fsmi.device_status() == 0


def test_bad_explicit_beam_sets_status():
    off = np.array([0, 3000], np.int32)  # longer than FSMI_MAX_CELLS
    o = np.full(3000, 0.5, np.float32)
    l = np.arange(3000, dtype=np.float32)
    lend = np.array([3000.0], np.float32)
    gp, _ = _prms(1.5, 64.0)
    fsmi.device_status()
    got = fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp).cpu().numpy()
    assert np.isnan(got[0])
    assert fsmi.device_status() & fsmi.STATUS_BAD_BEAM
    assert fsmi.device_status() == 0


def test_gauss_tail_against_cuda_erfc():
    # the library's tail against torch's CUDA erfc (double) on a dense grid of the scaled variable
    k = float(np.sqrt(np.log2(np.e)))
    s = torch.cat([torch.linspace(0, 8, 2_000_001), torch.linspace(8, 300, 10001)]).cuda()
    got = fsmi.gauss_tail(s).double()
    ref = 0.5 * torch.special.erfc(s.double() / k)
    err = (got - ref).abs()
    assert err.max().item() <= 3e-7
    assert bool(torch.all(err <= 4e-6 * ref + 6e-8))


WINDOW_CASES = ((64.0, 1.5, 0), (256.0, 2.0, 24), (256.0, 0.4, 8), (256.0, 12.0, 8))


def _window_case(R, sigma, n_poses):
    if n_poses == 0:
        return synth.random_grid_200()
    return synth.office_scene(n_poses=n_poses, size=512)


@pytest.mark.parametrize("e0", [0, 1])
def test_exact_full_window_is_bit_identical_to_full_sweep(e0):
    # skipping only the tail terms that flush to zero in FP32 must not change a single bit
    for R, sigma, npo in WINDOW_CASES:
        grid, poses, dirs = _window_case(R, sigma, npo)
        gp, _ = _prms(sigma, R, e0)
        gp.flags = fsmi.FLAG_FULL_WINDOW
        win = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp)
        gp.flags = fsmi.FLAG_FULL_SWEEP
        full = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp)
        assert torch.equal(win, full)
    off, o, l, lend = synth.random_beams(200, 0, 400, seed=77)
    gp, _ = _prms(3.0, 64.0, e0)
    gp.flags = fsmi.FLAG_FULL_WINDOW
    win = fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp)
    gp.flags = fsmi.FLAG_FULL_SWEEP
    assert torch.equal(win, fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp))


@pytest.mark.parametrize("e0", [0, 1])
def test_exact_default_window_against_full_sweep(e0):
    # the default window skips terms below 2^-27 of their weights (together below one FP32 ulp of
    # the largest weight for sigma up to 19 cells): the MI moves by a few FP32 roundings of the
    # running sums at most, far inside the parity tolerance
    for R, sigma, npo in WINDOW_CASES:
        grid, poses, dirs = _window_case(R, sigma, npo)
        gp, _ = _prms(sigma, R, e0)
        win = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp).cpu().numpy().astype(np.float64)
        gp.flags = fsmi.FLAG_FULL_SWEEP
        full = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp).cpu().numpy().astype(np.float64)
        err = np.abs(win - full)
        assert np.all(err <= 2.0 ** -20 * np.abs(full) + 1e-9), (sigma, err.max())
    off, o, l, lend = synth.random_beams(200, 0, 400, seed=77)
    gp, _ = _prms(3.0, 64.0, e0)
    win = fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp).cpu().numpy().astype(np.float64)
    gp.flags = fsmi.FLAG_FULL_SWEEP
    full = fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(win - full) <= 2.0 ** -20 * np.abs(full) + 1e-9)


def test_zero_length_cells():
    # consecutive equal distances (a cell shorter than FP32 resolution, as near-corner traversal
    # cuts produce): the boundary below the cell centre must still count as below
    rng = np.random.default_rng(42)
    beams, dists = [], []
    for k in range(64):
        n = int(rng.integers(2, 200))
        w = rng.uniform(0.2, 1.4, n)
        w[rng.random(n) < 0.15] = 0.0  # zero-length cells
        l = np.concatenate([[0.0], np.cumsum(w)]).astype(np.float32)
        beams.append(rng.uniform(0.02, 0.98, n))
        dists.append(l)
    off = np.concatenate([[0], np.cumsum([len(b) for b in beams])]).astype(np.int32)
    o = np.concatenate(beams).astype(np.float32)
    l = np.concatenate([d[:-1] for d in dists]).astype(np.float32)
    lend = np.array([d[-1] for d in dists], np.float32)
    for kw in (dict(variant=fsmi.EXACT), dict(variant=fsmi.EXACT, flags=fsmi.FLAG_FULL_SWEEP),
               dict(variant=fsmi.EXACT, flags=fsmi.FLAG_FULL_WINDOW), dict(variant=fsmi.APPROX, trunc_delta=3)):
        for e0 in (0, 1):
            gp, op = _prms(1.0, 64.0, e0, **kw)
            op_kw = {k: v for k, v in kw.items() if k != "flags"}
            op = oracle.Params(sigma=1.0, delta_occ=1.5, delta_emp=0.67, max_range=64.0, e0_mode=e0, **op_kw)
            got = fsmi.eval_beams(_cuda(off), _cuda(o), _cuda(l), _cuda(lend), gp).cpu().numpy()
            ref = oracle.eval_beams(off, o, l, lend, op)
            assert_mi_close(got, ref, f"zero-length {kw} e0={e0}")


def test_map_gains_workspace_is_bit_identical():
    # per-map-cell gains (workspace) against per-visit gains (no workspace), all three variants
    grid, poses, dirs = synth.office_scene(n_poses=64, size=1024)
    for kw in (dict(variant=fsmi.EXACT), dict(variant=fsmi.APPROX, trunc_delta=6), dict(variant=fsmi.UNIFORM, uniform_h=4)):
        gp, _ = _prms(2.0, 256.0, 0, **kw)
        a = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp)
        b = fsmi.eval_2d(_cuda(grid), _cuda(poses), _cuda(dirs), gp, ws=torch.empty(0, dtype=torch.uint8, device="cuda"))
        assert torch.equal(a, b)
