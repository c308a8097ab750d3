"""Learned surrogate of the beam FSMI: training on FSMI-labelled beams, prescreening of candidate
poses, and the exact rerank (not part of the paper; exact FSMI stays the labeller, the fallback
and the final arbiter of the ranking).

Every numerical step runs in the library's kernels (``fsmi.py``): profile sampling, the network's
forward and backward passes, Adam, the tensor-core inference, per-pose sums, top-k selection,
pose gathering and the exact FSMI of the reranked poses. This module only orders those calls,
draws the training batches' beam indices (numpy, seeded) and keeps the parameters.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass

import numpy as np
import torch

from . import fsmi, synth

# flat parameter layout (fsmi.h): name, shape
LAYOUT = [("W1", (32, 3, 2)), ("b1", (32,)), ("W2", (32, 3, 32)), ("b2", (32,)), ("W3", (32, 3, 32)), ("b3", (32,)),
          ("W4", (256, 1024)), ("b4", (256,)), ("W5", (256,)), ("b5", (1,))]


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, float32."""
    rng = np.random.default_rng(seed)
    out = []
    for name, shape in LAYOUT:
        n = int(np.prod(shape))
        if name.startswith("W"):
            fan_in = int(np.prod(shape[1:])) if len(shape) > 1 else shape[0]
            lim = math.sqrt(6.0 / fan_in)
            out.append(rng.uniform(-lim, lim, n).astype(np.float32))
        else:
            out.append(np.zeros(n, np.float32))
    theta = np.concatenate(out)
    assert theta.size == fsmi.SURR_NPARAMS
    return theta


@dataclass
class TrainingMap:
    grid: torch.Tensor    # float32 [H][W]
    poses: torch.Tensor   # int32 [P][4]
    labels: torch.Tensor  # float32 [P * B], exact FSMI of every beam at max_range
    max_range: float = 0.0  # the labels' beam range; the profiles are cut there (0: all 256 samples)


def label_maps(n_maps: int, poses_per_map: int, dirs, prm: fsmi.Params, seed: int = 100, size: int = 2048,
               ranges=None):
    """Office maps as in the 2048x2048 benchmark (office generator, seeds seed, seed+1, ...) with every beam of every pose
    labelled by exact FSMI on the GPU, at prm.max_range or, with `ranges`, map k at ranges[k % len]
    (ranges up to 256, the samples of a profile)."""
    out = []
    d = dirs if isinstance(dirs, torch.Tensor) else torch.from_numpy(dirs).cuda()
    for k in range(n_maps):
        grid, poses, _ = synth.office_scene(n_poses=poses_per_map, size=size, seed=seed + k, pose_seed=seed + 1000 + k)
        g = torch.from_numpy(grid).cuda()
        p = torch.from_numpy(poses).cuda()
        r = float(ranges[k % len(ranges)]) if ranges else float(prm.max_range)
        lab = fsmi.eval_2d(g, p, d, dataclasses.replace(prm, max_range=r)).reshape(-1)
        out.append(TrainingMap(g, p, lab, r))
    return out


class Surrogate:
    """Parameters (FP32 master + BF16 copy) and Adam state of one surrogate network on the device."""

    def __init__(self, seed: int = 0, scale: float = 1.0, device: str = "cuda", shift: float = 0.0):
        self.params = torch.from_numpy(init_params(seed)).to(device)
        self.wbf16 = torch.empty(fsmi.SURR_NPARAMS, dtype=torch.bfloat16, device=device)
        fsmi.surrogate_cast(self.params, self.wbf16)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.step = 0
        self.scale = float(scale)  # shift + network output x scale = predicted MI (nats)
        self.shift = float(shift)
        self._ws = {}

    # ---- checkpoints ---------------------------------------------------------------------------
    def state(self) -> dict:
        return {"params": self.params.cpu().numpy(), "m": self.m.cpu().numpy(), "v": self.v.cpu().numpy(),
                "step": self.step, "scale": self.scale, "shift": self.shift}

    def save(self, path: str) -> None:
        np.savez(path, **self.state())

    @classmethod
    def load(cls, path_or_state, device: str = "cuda") -> "Surrogate":
        st = np.load(path_or_state) if isinstance(path_or_state, str) else path_or_state
        s = cls(0, float(st["scale"]), device, float(st["shift"]) if "shift" in st else 0.0)
        s.params.copy_(torch.from_numpy(np.asarray(st["params"], np.float32)))
        s.m.copy_(torch.from_numpy(np.asarray(st["m"], np.float32)))
        s.v.copy_(torch.from_numpy(np.asarray(st["v"], np.float32)))
        s.step = int(st["step"])
        fsmi.surrogate_cast(s.params, s.wbf16)
        return s

    # ---- training -------------------------------------------------------------------------------
    def _workspace(self, mode: int, n: int) -> torch.Tensor:
        key = (mode, n)
        if key not in self._ws:
            self._ws[key] = torch.empty(fsmi.surrogate_workspace_size(mode, n), dtype=torch.uint8,
                                        device=self.params.device)
        return self._ws[key]

    def train(self, maps: list[TrainingMap], dirs, steps: int, batch: int = 4096, lr: float = 2e-3,
              lr_min: float = 1e-4, seed: int = 0, log_every: int = 0) -> list[float]:
        """`steps` Adam steps on random beams (uniform over maps, poses and beams), cosine learning
        rate from lr to lr_min over the steps of this call. Returns the losses read back every
        log_every steps (reading synchronises; 0 = never)."""
        rng = np.random.default_rng(seed + 7919 * self.step)
        d = dirs if isinstance(dirs, torch.Tensor) else torch.from_numpy(dirs).cuda()
        B = d.shape[0]
        ws = self._workspace(0, batch)
        x = torch.empty((batch, fsmi.SURR_L, 2), dtype=torch.bfloat16, device=self.params.device)
        y = torch.empty(batch, dtype=torch.float32, device=self.params.device)
        scaled = [(m.labels - self.shift) / self.scale for m in maps]
        # every batch's map and beams, drawn up front and copied once
        which = rng.integers(len(maps), size=steps)
        ids_all = np.empty((steps, batch), np.int32)
        for i in range(steps):
            ids_all[i] = rng.integers(0, maps[which[i]].poses.shape[0] * B, batch)
        ids_dev = torch.from_numpy(ids_all).to(self.params.device)
        losses = []
        for i in range(steps):
            k = int(which[i])
            mp = maps[k]
            ids = ids_dev[i]
            fsmi.profiles_2d(mp.grid, mp.poses, d, beam_ids=ids, out=x, max_range=mp.max_range)
            fsmi.gather_rows(scaled[k].view(torch.int32).reshape(-1, 1), ids, out=y.view(torch.int32).reshape(-1, 1))
            fsmi.surrogate_loss_grad(self.params, self.wbf16, x, y, self.grad, self.loss, ws=ws)
            self.step += 1
            frac = i / max(1, steps - 1)
            lr_i = lr_min + 0.5 * (lr - lr_min) * (1.0 + math.cos(math.pi * frac))
            fsmi.surrogate_adam(self.params, self.m, self.v, self.grad, lr_i, self.step, self.wbf16)
            if log_every and (i % log_every == 0 or i == steps - 1):
                losses.append(float(self.loss.item()))
        return losses

    # ---- inference ------------------------------------------------------------------------------
    def predict(self, grid, poses, dirs, out=None, ws=None, max_range: float = 0.0) -> torch.Tensor:
        """Network outputs ((predicted MI - shift) / scale) of every beam of every pose, [P * B]
        (tensor cores), for beams cut at max_range (0: all 256 samples)."""
        n = poses.shape[0] * dirs.shape[0]
        if ws is None:
            ws = self._workspace(1, n)
        pred = fsmi.surrogate_predict(self.params, self.wbf16, grid=grid, poses=poses, dirs=dirs, out=out, ws=ws,
                                      max_range=max_range)
        return pred


class Prescreen:
    """Surrogate prescreen + exact rerank over a fixed candidate batch, with every buffer allocated
    once so that the whole selection can be replayed (and captured in a CUDA graph)."""

    def __init__(self, net: Surrogate, grid, poses, dirs, prm: fsmi.Params, k: int = 64, top: int = 10):
        self.net, self.grid, self.poses, self.dirs, self.prm = net, grid, poses, dirs, prm
        P, B = poses.shape[0], dirs.shape[0]
        dev = grid.device
        self.k, self.top = k, top
        self.pred = torch.empty(P * B, dtype=torch.float32, device=dev)
        self.ws_pred = torch.empty(fsmi.surrogate_workspace_size(1, P * B), dtype=torch.uint8, device=dev)
        self.score = torch.empty(P, dtype=torch.float32, device=dev)
        self.cand = torch.empty(k, dtype=torch.int32, device=dev)
        self.sel = torch.empty((k, 4), dtype=torch.int32, device=dev)
        self.exact = torch.empty((k, B), dtype=torch.float32, device=dev)
        self.ws_exact = torch.empty(fsmi.workspace_size(fsmi.FN_EVAL_2D, grid.numel()), dtype=torch.uint8, device=dev)
        self.exact_score = torch.empty(k, dtype=torch.float32, device=dev)
        self.rank = torch.empty(top, dtype=torch.int32, device=dev)
        self.best = torch.empty((top, 1), dtype=torch.int32, device=dev)

    def run(self) -> torch.Tensor:
        """Pose indices [top] (int32, device): the best by exact FSMI among the surrogate's top k."""
        self.net.predict(self.grid, self.poses, self.dirs, out=self.pred, ws=self.ws_pred, max_range=self.prm.max_range)
        fsmi.scan_sums_into(self.pred.view(self.poses.shape[0], self.dirs.shape[0]), self.score)
        fsmi.topk(self.score, self.k, out=self.cand)
        fsmi.gather_rows(self.poses, self.cand, out=self.sel)
        fsmi.eval_2d(self.grid, self.sel, self.dirs, self.prm, out=self.exact, ws=self.ws_exact)
        fsmi.scan_sums_into(self.exact, self.exact_score)
        fsmi.topk(self.exact_score, self.top, out=self.rank)
        fsmi.gather_rows(self.cand.view(-1, 1), self.rank, out=self.best)
        return self.best.view(-1)


class ExactAll:
    """The method without the surrogate: exact FSMI of every beam, per-pose sums, top poses."""

    def __init__(self, grid, poses, dirs, prm: fsmi.Params, top: int = 10):
        self.grid, self.poses, self.dirs, self.prm, self.top = grid, poses, dirs, prm, top
        P, B = poses.shape[0], dirs.shape[0]
        dev = grid.device
        self.mi = torch.empty((P, B), dtype=torch.float32, device=dev)
        self.ws = torch.empty(fsmi.workspace_size(fsmi.FN_EVAL_2D, grid.numel()), dtype=torch.uint8, device=dev)
        self.score = torch.empty(P, dtype=torch.float32, device=dev)
        self.best = torch.empty(top, dtype=torch.int32, device=dev)

    def run(self) -> torch.Tensor:
        fsmi.eval_2d(self.grid, self.poses, self.dirs, self.prm, out=self.mi, ws=self.ws)
        fsmi.scan_sums_into(self.mi, self.score)
        fsmi.topk(self.score, self.top, out=self.best)
        return self.best


def _np(x):
    return np.asarray(x.cpu() if isinstance(x, torch.Tensor) else x)


def recall(found, truth) -> float:
    """Strict recall: the fraction of the index set `truth` that `found` contains."""
    a, b = set(_np(found).tolist()), set(_np(truth).tolist())
    return len(a & b) / len(b)


def recall_with_ties(found, exact_scores, top: int = 10, rel_tol: float = 1e-4) -> float:
    """Top-`top` recall when exact scores tie: a found pose counts as a hit when its exact score is
    at least the top-th best exact score minus rel_tol of it (the exact method resolves per-beam MI
    to 1e-4 relative, so smaller differences do not order poses). Many candidate poses in open
    space reach the same saturated score, and then the strict top-10 is decided by rounding."""
    sc = _np(exact_scores).astype(np.float64)
    kth = np.sort(sc)[::-1][top - 1]
    hits = sc[_np(found)] >= kth - rel_tol * abs(kth)
    return float(min(hits.sum(), top)) / top


def tie_band(exact_scores, top: int = 10, rel_tol: float = 1e-4) -> int:
    """How many candidates score within rel_tol (relative) of the top-th best exact score: `top`
    when the exact top set is separated at that level, more when the cut falls among ties."""
    sc = _np(exact_scores).astype(np.float64)
    kth = np.sort(sc)[::-1][top - 1]
    return int((sc >= kth - rel_tol * abs(kth)).sum())


def regret(found, exact_scores) -> float:
    """1 - (best exact score among `found`) / (best exact score overall)."""
    sc = _np(exact_scores).astype(np.float64)
    return float(1.0 - sc[_np(found)].max() / sc.max())


def _main():
    """Times the surrogate inference on a 2048x2048 office map (used for profiling):
    python -m paper_1905_02238_gb300.surrogate --poses 512 --repeat 4"""
    import argparse

    ap = argparse.ArgumentParser()
    ap.add_argument("--poses", type=int, default=4096)
    ap.add_argument("--beams", type=int, default=360)
    ap.add_argument("--repeat", type=int, default=4)
    args = ap.parse_args()
    from . import build

    build.build()
    grid, poses, _ = synth.office_scene(n_poses=args.poses, seed=200, pose_seed=201)
    g, p = torch.from_numpy(grid).cuda(), torch.from_numpy(poses).cuda()
    d = torch.from_numpy(synth.beam_dirs_2d(args.beams)).cuda()
    net = Surrogate(seed=0, scale=0.01, shift=0.06)
    out = torch.empty(args.poses * args.beams, dtype=torch.float32, device="cuda")
    ws = torch.empty(fsmi.surrogate_workspace_size(1, out.numel()), dtype=torch.uint8, device="cuda")
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    net.predict(g, p, d, out=out, ws=ws)
    torch.cuda.synchronize()
    s.record()
    for _ in range(args.repeat):
        net.predict(g, p, d, out=out, ws=ws)
    e.record()
    torch.cuda.synchronize()
    print(f"surrogate predict {args.poses} x {args.beams} beams: {s.elapsed_time(e) / args.repeat:.3f} ms")


if __name__ == "__main__":
    _main()
