"""GPU parity of the learned surrogate's kernels (profiles, training forward/backward, Adam,
tensor-core inference, top-k, gather) against the FP64 oracle in oracle/surrogate.py, and the
properties of training (determinism, checkpoint resume)."""
import numpy as np
import pytest
import torch

from oracle import surrogate as S
from paper_1905_02238_gb300 import fsmi, synth
from paper_1905_02238_gb300 import surrogate as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1905_02238_gb300 import build

    build.build()
    return fsmi.load()


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _case(seed=1, n_poses=6, nb=40):
    grid = synth.office_grid(300, n_obst=40, seed=seed)
    poses = synth.free_cell_poses_2d(grid, n_poses, seed=seed + 1)
    rng = np.random.default_rng(seed + 2)
    dirs = np.concatenate([synth.beam_dirs_2d(nb - 8), synth.random_dirs_2d(8, rng)])
    return grid, poses, dirs


def _theta(seed=3):
    rng = np.random.default_rng(seed)
    th = sg.init_params(seed)
    th += rng.normal(0, 0.02, th.shape).astype(np.float32)  # non-zero biases
    return th


def test_param_layout_matches_oracle():
    assert fsmi.SURR_NPARAMS == S.n_params()
    assert [n for n, _ in sg.LAYOUT] == [n for n, _ in S.LAYOUT]
    assert all(tuple(a) == tuple(b) for (_, a), (_, b) in zip(sg.LAYOUT, S.LAYOUT))


def test_profiles_bit_exact():
    grid, poses, dirs = _case()
    x = fsmi.profiles_2d(_cuda(grid), _cuda(poses), _cuda(dirs)).float().cpu().numpy().astype(np.float64)
    ref = S.bf16_round(S.profiles_2d(grid, poses, dirs))
    np.testing.assert_array_equal(x, ref)
    ids = np.array([5, 0, 77, 239, 3], np.int32)
    xs = fsmi.profiles_2d(_cuda(grid), _cuda(poses), _cuda(dirs), beam_ids=_cuda(ids)).float().cpu().numpy()
    np.testing.assert_array_equal(xs, x[ids])
    for R in (0.5, 0.51, 17.0, 63.5, 100.25, 255.5, 300.0):  # profiles cut at a range
        xr = fsmi.profiles_2d(_cuda(grid), _cuda(poses), _cuda(dirs), max_range=R).float().cpu().numpy()
        np.testing.assert_array_equal(xr, S.bf16_round(S.profiles_2d(grid, poses, dirs, max_range=R)))


def _profiles(grid, poses, dirs):
    x = fsmi.profiles_2d(_cuda(grid), _cuda(poses), _cuda(dirs))
    return x, x.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("nb", [40, 41])
def test_loss_and_gradient_match_oracle(nb):
    # 3 x 41 = 123 beams: a batch that is not a multiple of 4 (the workspace's buffers stay aligned)
    grid, poses, dirs = _case(n_poses=3, nb=nb)
    x, xh = _profiles(grid, poses, dirs)
    N = x.shape[0]
    rng = np.random.default_rng(4)
    y = rng.uniform(0, 3, N).astype(np.float32)
    th = _theta()
    params = _cuda(th)
    wb = torch.empty(fsmi.SURR_NPARAMS, dtype=torch.bfloat16, device="cuda")
    fsmi.surrogate_cast(params, wb)
    np.testing.assert_array_equal(wb.float().cpu().numpy().astype(np.float64), S.bf16_round(th))
    grad = torch.zeros(fsmi.SURR_NPARAMS, device="cuda")
    loss = torch.zeros(1, device="cuda")
    pred = torch.zeros(N, device="cuda")
    ws = torch.zeros(fsmi.surrogate_workspace_size(0, N), dtype=torch.uint8, device="cuda")
    fsmi.surrogate_loss_grad(params, wb, x, _cuda(y), grad, loss, pred=pred, ws=ws)
    rpred, cache = S.forward(th, xh)
    rloss, dpred = S.mse(rpred, y)
    np.testing.assert_allclose(pred.cpu().numpy(), rpred, rtol=2e-5, atol=2e-5 * np.abs(rpred).max())
    assert abs(float(loss.item()) - rloss) <= 5e-5 * rloss
    # The forward pass element by element: the step leaves its FP32 pre-activations z1, z2, z3, z4 at
    # the start of the workspace; each lies within 1e-5 of the sum of its terms' absolute values (the
    # oracle's forward on |weights| and |x|) of the oracle's, which covers FP32 accumulation of a
    # conv's 96 terms in the worst case (96 x 2^-24 = 5.7e-6) and of fc1's 1024 as a random walk.
    _, zabs = S.forward(np.abs(th), np.abs(xh))
    zf = ws.view(torch.float32).cpu().numpy().astype(np.float64)
    at = 0
    gcache = dict(cache)
    for k, shape in (("z1", (N, 128, 32)), ("z2", (N, 64, 32)), ("z3", (N, 32, 32)), ("z4", (N, 256))):
        n = int(np.prod(shape))
        zg = zf[at:at + n].reshape(shape)
        at += n
        assert np.all(np.abs(zg - cache[k]) <= 1e-5 * zabs[k]), k
        gcache[k] = zg
    # The backward pass is then compared at the step's own forward state: the oracle differentiates
    # the GPU's pre-activations (ReLU masks included: a pre-activation within rounding of zero may
    # take either side) with dpred = 2 (pred - y) / N of the GPU's predictions.
    gcache["a1"], gcache["a2"], gcache["a3"] = (np.maximum(gcache[k], 0.0) for k in ("z1", "z2", "z3"))
    gcache["h0"] = gcache["a3"].reshape(N, -1)
    gcache["a4"] = np.maximum(gcache["z4"], 0.0)
    _, dpred = S.mse(pred.cpu().numpy().astype(np.float64), y)
    cache = gcache
    rgrad = S.backward(cache, dpred)
    g = grad.cpu().numpy().astype(np.float64)
    # Element by element: each gradient entry is a sum of products (over beams, positions and the
    # layers above); the FP32 sums can cancel, so the bound scales with the sum of the absolute
    # values of those products, which the oracle's backward pass gives when it runs on |weights|,
    # |dpred| and the (non-negative) activations with the same ReLU masks. The bound, 2e-4 of that
    # sum, covers the backward pass's split-BF16 products (2^-17 per product) and FP32 accumulation.
    acache = dict(cache)
    acache["p"] = {k: np.abs(v) for k, v in cache["p"].items()}
    for k in ("a0", "a1", "a2", "a3", "a4", "h0"):
        acache[k] = np.abs(cache[k])
    bound = S.backward(acache, np.abs(dpred))
    err = np.abs(g - rgrad)
    worst = {}
    for name, (o, shape) in S.offsets().items():
        n = int(np.prod(shape))
        e, bnd = err[o:o + n], bound[o:o + n]
        worst[name] = float(np.max(e / (bnd + 1e-30)))
        assert np.all(e <= 2e-4 * bnd + 1e-12), (name, worst[name])
    print('gradient error / abs-sum bound, worst per layer:', worst)
    # the same step twice gives the same floats
    g2 = torch.zeros_like(grad)
    fsmi.surrogate_loss_grad(params, wb, x, _cuda(y), g2, loss)
    assert torch.equal(g2, grad)


def test_adam_matches_oracle():
    rng = np.random.default_rng(5)
    th = _theta(6)
    g = rng.normal(0, 1e-2, th.shape).astype(np.float32)
    m0 = rng.normal(0, 1e-3, th.shape).astype(np.float32)
    v0 = rng.uniform(0, 1e-5, th.shape).astype(np.float32)
    p, m, v = _cuda(th), _cuda(m0), _cuda(v0)
    wb = torch.empty(fsmi.SURR_NPARAMS, dtype=torch.bfloat16, device="cuda")
    fsmi.surrogate_adam(p, m, v, _cuda(g), 1e-3, 7, wb)
    # the kernel's hyperparameters are the FP32 values of 0.9, 0.999, 1e-3, 1e-8 (1 - beta is then
    # exact in FP32); the oracle takes the same values
    b1, b2, lr, eps = (float(np.float32(x)) for x in (0.9, 0.999, 1e-3, 1e-8))
    rp, rm, rv = S.adam(th.astype(np.float64), m0.astype(np.float64), v0.astype(np.float64), g.astype(np.float64), 7,
                        lr, b1, b2, eps)
    # FP32 moments: within a few units in the last place of the two terms they add (the sum can
    # cancel, so the bound is on the terms, not on the result)
    u = 2.0 ** -22
    gm, gv, gp = (t.cpu().numpy().astype(np.float64) for t in (m, v, p))
    assert np.all(np.abs(gm - rm) <= u * (b1 * np.abs(m0) + (1 - b1) * np.abs(g)))
    assert np.all(np.abs(gv - rv) <= u * (b2 * v0 + (1 - b2) * g.astype(np.float64) ** 2))
    # the parameter update from the GPU's own moments: a few ulp of theta and of the step
    c1, c2 = float(np.float32(1 - b1 ** 7)), float(np.float32(1 - b2 ** 7))
    step = lr * (gm / c1) / (np.sqrt(gv / c2) + eps)
    ref_p = th.astype(np.float64) - step
    assert np.all(np.abs(gp - ref_p) <= u * (np.abs(th) + 4 * np.abs(step)))
    np.testing.assert_allclose(gp, rp, rtol=0, atol=2e-6)  # and close to the all-FP64 step
    np.testing.assert_array_equal(wb.float().cpu().numpy().astype(np.float64), S.bf16_round(p.cpu().numpy()))


def test_tensor_core_inference_matches_oracle():
    grid, poses, dirs = _case(seed=8, n_poses=7, nb=48)  # 336 beams: 2 full fc row tiles + a tail
    x, xh = _profiles(grid, poses, dirs)
    th = _theta(9)
    params = _cuda(th)
    wb = torch.empty(fsmi.SURR_NPARAMS, dtype=torch.bfloat16, device="cuda")
    fsmi.surrogate_cast(params, wb)
    got = fsmi.surrogate_predict(params, wb, x=x).cpu().numpy().astype(np.float64)
    ref, _ = S.forward(th, xh, act_bf16=True)
    ref32, _ = S.forward(th, xh)
    err = np.abs(got - ref)
    scale = np.abs(ref).max()
    # BF16 activations: the GPU rounds FP32 sums and the oracle FP64 sums to BF16; the two differ
    # by one BF16 step (2^-8 relative) where the sums straddle a rounding boundary
    assert err.max() <= 1e-3 * scale, (err.max(), scale)
    assert np.median(err) <= 1e-5 * scale
    # and the BF16-activation network stays close to the FP32-activation one
    assert np.abs(got - ref32).max() <= 3e-2 * scale
    # profiles sampled inside the kernel give the same floats
    got_map = fsmi.surrogate_predict(params, wb, grid=_cuda(grid), poses=_cuda(poses), dirs=_cuda(dirs))
    np.testing.assert_array_equal(got_map.cpu().numpy(), got.astype(np.float32))
    # ... and cut at a range, the same floats as the cut profiles given as input
    xr = fsmi.profiles_2d(_cuda(grid), _cuda(poses), _cuda(dirs), max_range=37.5)
    got_r = fsmi.surrogate_predict(params, wb, grid=_cuda(grid), poses=_cuda(poses), dirs=_cuda(dirs), max_range=37.5)
    np.testing.assert_array_equal(got_r.cpu().numpy(), fsmi.surrogate_predict(params, wb, x=xr).cpu().numpy())
    assert not torch.equal(got_r, got_map)
    # many row tiles per persistent block and a ragged last tile: every row equals its own value
    # from the small launch (rows are independent and each row's sums run in a fixed order)
    idx = np.random.default_rng(11).integers(0, x.shape[0], 152 * 128 * 3 + 77)
    big = fsmi.surrogate_predict(params, wb, x=x[torch.from_numpy(idx).cuda()]).cpu().numpy()
    np.testing.assert_array_equal(big, got.astype(np.float32)[idx])


def test_inference_wait_that_runs_out_sets_timeout_and_nan():
    # The epilogue's bounded wait for its tensor-core accumulator, limited to zero polls, gives up
    # before any MMA can finish: the call must flag FSMI_STATUS_TIMEOUT, write NaN for every row,
    # still return (its copies and MMAs in flight land under the full limit), and leave the device
    # usable: the next call with the default limit is clean and equals the one before.
    grid, poses, dirs = _case(seed=8, n_poses=7, nb=48)
    x, _ = _profiles(grid, poses, dirs)
    th = _theta(9)
    params = _cuda(th)
    wb = torch.empty(fsmi.SURR_NPARAMS, dtype=torch.bfloat16, device="cuda")
    fsmi.surrogate_cast(params, wb)
    assert fsmi.device_status() == 0
    before = fsmi.surrogate_predict(params, wb, x=x)
    try:
        fsmi.set_wait_limit(0)
        bad = fsmi.surrogate_predict(params, wb, x=x)
        torch.cuda.synchronize()
    finally:
        fsmi.set_wait_limit(-1)
    assert fsmi.device_status() & fsmi.STATUS_TIMEOUT
    assert bool(torch.isnan(bad).all())
    after = fsmi.surrogate_predict(params, wb, x=x)
    assert fsmi.device_status() == 0
    assert torch.equal(after, before)


def test_topk_and_gather():
    rng = np.random.default_rng(10)
    for n, k in ((1, 1), (100, 10), (4096, 64), (5000, 5000), (16384, 7)):
        v = rng.normal(size=n).astype(np.float32)
        v[rng.choice(n, n // 10, replace=False)] = 0.5  # ties
        if n > 10:
            v[3] = np.nan
        idx = fsmi.topk(_cuda(v), k).cpu().numpy()
        key = np.where(np.isnan(v), -np.inf, v)
        ref = np.lexsort((np.arange(n), -key))[:k]
        np.testing.assert_array_equal(idx, ref)
    src = rng.integers(-100, 100, (50, 4)).astype(np.int32)
    ii = np.array([3, 3, 49, 0], np.int32)
    np.testing.assert_array_equal(fsmi.gather_rows(_cuda(src), _cuda(ii)).cpu().numpy(), src[ii])


def _tiny_training_set():
    dirs = synth.beam_dirs_2d(90)
    prm = fsmi.Params(variant=fsmi.EXACT, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=256.0)
    return sg.label_maps(2, 64, dirs, prm, seed=300, size=512), dirs


def test_training_is_deterministic_and_resumable(tmp_path):
    maps, dirs = _tiny_training_set()
    scale = float(torch.cat([m.labels for m in maps]).mean())
    a = sg.Surrogate(seed=1, scale=scale)
    losses = a.train(maps, dirs, steps=60, batch=512, lr=2e-3, log_every=10)
    assert losses[-1] < losses[0]
    b = sg.Surrogate(seed=1, scale=scale)
    b.train(maps, dirs, steps=60, batch=512, lr=2e-3)
    assert torch.equal(a.params, b.params)
    # checkpoint after 30 steps, resume for the rest: same floats as the 60-step run when the
    # learning-rate schedule of the two halves is the same
    c = sg.Surrogate(seed=1, scale=scale)
    c.train(maps, dirs, steps=30, batch=512, lr=1e-3, lr_min=1e-3)
    path = str(tmp_path / "ckpt.npz")
    c.save(path)
    c.train(maps, dirs, steps=30, batch=512, lr=1e-3, lr_min=1e-3)
    d = sg.Surrogate.load(path)
    d.train(maps, dirs, steps=30, batch=512, lr=1e-3, lr_min=1e-3)
    assert torch.equal(c.params, d.params) and torch.equal(c.m, d.m) and torch.equal(c.v, d.v)


@pytest.mark.slow
def test_trained_surrogate_prescreen_beats_exact_all():
    """The gain of the learned part: on a held-out 2048x2048 office map with 4096 candidate poses,
    the surrogate prescreen plus exact rerank of its top 64 finds the exact top-10 (up to exact
    ties at 1e-4) in less time than exact FSMI of every beam; an untrained network does not. On
    candidates at the map's frontiers, whose exact top 10 has no ties, it finds it strictly."""
    dirs = synth.beam_dirs_2d(360)
    d = _cuda(dirs)
    prm = fsmi.Params(variant=fsmi.EXACT, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=256.0)
    maps = sg.label_maps(7, 4096, d, prm, seed=100)  # 10.3 M labelled beams
    lab = torch.cat([m.labels for m in maps])
    net = sg.Surrogate(seed=0, scale=float(lab.std()), shift=float(lab.mean()))
    net.train(maps, d, steps=2500, batch=4096, lr=2e-3)
    grid, poses, _ = synth.office_scene(n_poses=4096, seed=200, pose_seed=201)
    g, p = _cuda(grid), _cuda(poses)
    ex = sg.ExactAll(g, p, d, prm)
    ex.run()
    scores = ex.score.clone()
    pre = sg.Prescreen(net, g, p, d, prm, k=64)
    found = pre.run()
    assert sg.recall_with_ties(found, scores) >= 0.95
    assert sg.regret(found, scores) <= 1e-4

    def ms(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            fn()
        e.record()
        torch.cuda.synchronize()
        return s.elapsed_time(e) / reps

    assert ms(pre.run) < ms(ex.run)
    untrained = sg.Prescreen(sg.Surrogate(seed=0, scale=net.scale, shift=net.shift), g, p, d, prm, k=64)
    assert sg.recall_with_ties(untrained.run(), scores) < sg.recall_with_ties(found, scores)
    # Candidates at the map's frontiers (free cells 1-8 cells from unknown space): there the exact
    # top 10 is separated from the 11th (no tie at 1e-5), so strict recall can fail, and must not
    fp = _cuda(synth.frontier_poses_2d(grid, 4096, seed=204, rmin=1.0, rmax=8.0))
    fex = sg.ExactAll(g, fp, d, prm)
    truth = fex.run().clone()
    assert sg.tie_band(fex.score, 10, 1e-5) == 10  # the workload discriminates
    ffound = sg.Prescreen(net, g, fp, d, prm, k=64).run()
    assert sg.recall(ffound, truth) >= 0.95
    assert sg.regret(ffound, fex.score) <= 1e-5
    assert sg.recall(sg.Prescreen(sg.Surrogate(seed=0, scale=net.scale, shift=net.shift), g, fp, d, prm, k=64).run(),
                     truth) < 0.95
