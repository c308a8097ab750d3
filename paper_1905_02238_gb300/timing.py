"""Timing entry point for profiling single calls of the library on the benchmark workloads:

    python -m paper_1905_02238_gb300.timing --path 3d --variant exact --poses 64 --repeat 4
    python -m paper_1905_02238_gb300.timing --path 2d --variant approx --poses 1024
    python -m paper_1905_02238_gb300.timing --path surrogate --poses 4096
    python -m paper_1905_02238_gb300.timing --path train --repeat 50

2d: the 2048x2048 office map (poses x 360 beams, R = 256, sigma = 2); 3d: the 512x512x128 voxel
world (poses x 128x128 rays, 384 virtual cells, run cap 64); surrogate: inference on the office
map; train: surrogate training steps (batch 4096) on one office map of `poses` poses (256) whose
beams exact FSMI labels. One untimed call, then `repeat` calls timed with CUDA events; prints ms
per call.
"""
from __future__ import annotations

import argparse

import torch

from . import build, fsmi, synth


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--path", choices=["2d", "3d", "surrogate", "train"], default="2d")
    ap.add_argument("--variant", choices=["exact", "approx", "approx_band", "uniform"], default="exact")
    ap.add_argument("--poses", type=int, default=None)
    ap.add_argument("--repeat", type=int, default=4)
    args = ap.parse_args()
    build.build()
    dev = torch.device("cuda")
    var = {"exact": dict(variant=fsmi.EXACT), "approx": dict(variant=fsmi.APPROX),
           "approx_band": dict(variant=fsmi.APPROX, approx_reading=1), "uniform": dict(variant=fsmi.UNIFORM)}[args.variant]
    if args.path == "2d":
        grid, poses, dirs = synth.office_scene(n_poses=args.poses or 1024)
        g, p, d = (torch.from_numpy(x).to(dev) for x in (grid, poses, dirs))
        prm = fsmi.Params(sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=256.0, trunc_delta=6, uniform_h=4, **var)
        out = torch.empty((p.shape[0], d.shape[0]), dtype=torch.float32, device=dev)
        ws = torch.empty(fsmi.workspace_size(fsmi.FN_EVAL_2D, g.numel()), dtype=torch.uint8, device=dev)

        def call():
            fsmi.eval_2d(g, p, d, prm, out=out, ws=ws)
        what = f"eval_2d {args.variant} {p.shape[0]} x {d.shape[0]} beams"
    elif args.path == "3d":
        vox, vp, vd = synth.voxel_scene(n_poses=args.poses or 64)
        v, p, d = (torch.from_numpy(x).to(dev) for x in (vox, vp, vd))
        prm = fsmi.Params(sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=384.0, run_cap=64, trunc_delta=6,
                          uniform_h=4, **var)
        out = torch.empty((p.shape[0], d.shape[0]), dtype=torch.float32, device=dev)
        ws = torch.empty(fsmi.QUEUE_BYTES, dtype=torch.uint8, device=dev)

        def call():
            fsmi.eval_3d(v, p, d, prm, out=out, ws=ws)
        what = f"eval_3d {args.variant} {p.shape[0]} x {d.shape[0]} rays"
    elif args.path == "train":
        from . import surrogate as sg

        # surrogate training steps of 4096 beams drawn from one exact-labelled office map
        d = torch.from_numpy(synth.beam_dirs_2d(360)).to(dev)
        prm = fsmi.Params(variant=fsmi.EXACT, sigma=2.0, delta_occ=1.5, delta_emp=0.67, max_range=256.0)
        maps = sg.label_maps(1, args.poses or 256, d, prm, seed=100)
        lab = maps[0].labels
        net = sg.Surrogate(seed=0, scale=float(lab.std()), shift=float(lab.mean()))
        net.train(maps, d, steps=3, batch=4096)

        def call():
            net.train(maps, d, steps=1, batch=4096)
        what = "surrogate training step of 4096 beams"
    else:
        from . import surrogate as sg

        grid, poses, _ = synth.office_scene(n_poses=args.poses or 4096, seed=200, pose_seed=201)
        g, p = torch.from_numpy(grid).to(dev), torch.from_numpy(poses).to(dev)
        d = torch.from_numpy(synth.beam_dirs_2d(360)).to(dev)
        net = sg.Surrogate(seed=0, scale=0.01, shift=0.06)
        out = torch.empty(p.shape[0] * d.shape[0], dtype=torch.float32, device=dev)
        ws = torch.empty(fsmi.surrogate_workspace_size(1, out.numel()), dtype=torch.uint8, device=dev)

        def call():
            net.predict(g, p, d, out=out, ws=ws)
        what = f"surrogate predict {p.shape[0]} x {d.shape[0]} beams"
    call()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(args.repeat):
        call()
    e.record()
    torch.cuda.synchronize()
    print(f"{what}: {s.elapsed_time(e) / args.repeat:.3f} ms")


if __name__ == "__main__":
    main()
