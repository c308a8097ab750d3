"""Benchmark of the FSMI hot path on GB300.

Workload (one step): exact FSMI (Theorem 1) of every beam of a batch on the 2D office map:
2048x2048 grid (background 0.1, 400 obstacles at 0.9, 40% unknown at 0.5), 1024 candidate poses
x 360 beams, range 256 cells, sigma = 2 cells, delta_occ = 1.5, delta_emp = 0.67, through
fsmi_eval_2d (traversal, first-hit probabilities, C_k and the full pair sum, all in one kernel),
with the schedule picked by fsmi_autotune and the call captured once in a CUDA graph that each
step replays.
Synthetic, seeded inputs (paper_1905_02238_gb300.synth); no dataset is involved.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {fsmi,reference}]

Multi-GPU (torchrun, one process per GPU): every rank evaluates its own 1024 poses (weak scaling,
the map replicated, no collective on the data path); value = all ranks' beams / the slowest rank's
time. The reference arm (--impl reference) times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact FSMI beams/s & % roofline; surrogate+rerank poses/s at top-10 recall"
WORKLOAD = "2D exact FSMI, 2048x2048 office grid, 1024 poses x 360 beams, R=256, sigma=2"
SIGMA, R_MAX, DOCC, DEMP = 2.0, 256.0, 1.5, 0.67
N_POSES = 1024
L2_FLUSH_BYTES = 512 << 20  # > the 126 MB L2
SM_COUNT_NOMINAL = 152
FMA_LANES_PER_SM_CLK = 128  # FP32 FMA-pipe lane operations per SM per clock (4 x 32)
EX2_PER_SM_CLK = 32  # SFU ex2.approx results per SM per clock (csrc/pipe_probe.cu measured 31.8)
RCP_PER_SM_CLK = 16  # SFU rcp.approx results per SM per clock (measured 15.95)
SFU_CLK_PER_TERM = 1.0 / EX2_PER_SM_CLK + 1.0 / RCP_PER_SM_CLK  # one ex2 and one rcp per tail term
OPS_PER_TERM = 10  # FP32 FMA-pipe operations per boundary tail term (csrc/gauss_tail.cuh): distance,
#                    square, 1 + p|d|, 4 Horner FMAs, two products, accumulate
TAIL_CUT = 4.81  # scaled half-width of the exact kernel's default window (csrc/eval2d.cuh)

# DRAM bytes (read + write) per launch of the 2D kernel on the benchmark workload (exact; the
# Approx and Uniform legs by name), from an ncu capture of one full-size launch each
# (dram__bytes_read.sum + dram__bytes_write.sum), valid only for the kernel sources whose hash is
# recorded with them; reported as null once those sources change.
TRAFFIC = {"sources_sha1": "d04b34a3db90ae157f6964bfca6621c5e603dcaa", "bytes_per_launch": 111.34e6,
           "approx_fsmi_delta6": 82.83e6, "uniform_fsmi_h4": 83.00e6}
KERNEL_SOURCES = ["paper_1905_02238_gb300/csrc/fsmi_2d.cu", "paper_1905_02238_gb300/csrc/eval2d.cuh",
                  "paper_1905_02238_gb300/csrc/dda2d.cuh", "paper_1905_02238_gb300/csrc/gauss_tail.cuh",
                  "paper_1905_02238_gb300/csrc/fsmi_device.cuh"]


# DRAM bytes per launch of the fused 3D kernel on the 512x512x128 batch, per variant, from one
# ncu capture each (valid for the sources hashed with them, like TRAFFIC)
KERNEL_SOURCES_3D = ["paper_1905_02238_gb300/csrc/fsmi_rle.cu", "paper_1905_02238_gb300/csrc/evalrle.cuh",
                     "paper_1905_02238_gb300/csrc/fsmi_device.cuh"]
TRAFFIC_3D = {"sources_sha1": "8140517dbdd4473d1c65def9bad5f71ddea9e91f", "fsmi_rle_3d": 563.77e6, "approx_fsmi_rle_3d_delta6": 566.51e6,
              "approx_fsmi_rle_3d_delta6_band": 563.41e6, "uniform_fsmi_rle_3d_h4": 563.24e6}


def kernel_sources_sha1(files=None) -> str:
    import hashlib

    h = hashlib.sha1()
    for f in files or KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def max_over_ranks(x: float, ws: int, device) -> float:
    """The slowest rank's value (all ranks take part); x itself when ws == 1."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, ws: int, seconds: float) -> float:
    """Weak scaling: every rank processes units_per_rank; the job takes the slowest rank's time."""
    return units_per_rank * ws / seconds


def workload(rank: int, n_poses: int = N_POSES):
    from paper_1905_02238_gb300 import synth

    grid, poses, dirs = synth.office_scene(n_poses=n_poses, pose_seed=1 + rank)
    return grid, poses, dirs


def cpu_baseline(grid, poses, dirs, gpu_out=None, n_pose_sample: int = 288, n_single: int = 4):
    """The FP64 oracle as it stands, on all host cores, on the first n_pose_sample poses (and on one
    core on the first n_single); with gpu_out (the timed kernel's [P][B] result) also the parity of
    those beams against the oracle."""
    import numpy as np

    import oracle

    prm = oracle.Params(variant=oracle.EXACT, sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP, max_range=R_MAX)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    ref = oracle.eval_2d(grid, poses[:n_pose_sample], dirs, prm, nthreads=threads)
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    oracle.eval_2d(grid, poses[:n_single], dirs, prm, nthreads=1)
    dt1 = time.perf_counter() - t1
    nb = n_pose_sample * dirs.shape[0]
    res = {"value": nb / dt, "unit": "beams/s", "cores": threads, "kind": "oracle",
           "sample": f"first {n_pose_sample} poses x {dirs.shape[0]} beams ({nb} beams), FP64, {dt:.1f} s wall",
           "single_core": {"value": n_single * dirs.shape[0] / dt1, "unit": "beams/s",
                           "sample": f"first {n_single} poses x {dirs.shape[0]} beams, 1 thread, {dt1:.1f} s"}}
    if gpu_out is not None:
        got = np.asarray(gpu_out[:n_pose_sample], np.float64).reshape(ref.shape)
        ref = np.asarray(ref, np.float64)
        err = np.abs(got - ref)
        rel = err / np.maximum(np.abs(ref), 1e-30)
        res["parity_vs_oracle"] = {
            "beams": int(ref.size), "max_abs_err": float(err.max()), "max_rel_err": float(rel.max()),
            "median_rel_err": float(np.median(rel)),
            "within_tolerance": bool(np.all(err <= 1e-4 * np.abs(ref) + 1e-7)),
            "tolerance": "|gpu - oracle| <= 1e-4 |oracle| + 1e-7 nats per beam"}
    return res


def band_terms(n, delta):
    """Sum over first-hit cells j of the Approx-FSMI band size |[j - delta, j + delta] n [0, n - 1]|."""
    full = n * (2 * delta + 1) - delta * (delta + 1)  # n >= delta: each edge loses delta(delta+1)/2
    return full.where(n > delta, n * n)  # n <= delta: every band is the whole beam


def work_counts(fsmi, grid, p, d, chunk=32768):
    """(cells, Theorem-1 boundary terms n(n+1), terms the exact kernel evaluates, Approx band
    terms at Delta = 6) of one launch."""
    import torch

    cap = int(R_MAX * 1.5) + 4
    _, l, n = fsmi.trace_2d(grid.shape[1], grid.shape[0], p, d, R_MAX, cap)
    cs = float(torch.tensor(1.0 / (SIGMA * 1.4142135623730951), dtype=torch.float32) *
               torch.tensor(1.2011224087864498, dtype=torch.float32))
    cells = pairs = terms = band = 0.0
    col = torch.arange(cap + 1, device=l.device)
    for a in range(0, n.shape[0], chunk):
        nn = n[a:a + chunk].to(torch.int64)
        ll = l[a:a + chunk] * cs
        ll = torch.where(col[None, :] <= nn[:, None], ll, torch.full_like(ll, float("inf")))
        mu = 0.5 * (ll[:, :-1] + ll[:, 1:])
        valid = col[None, :-1] < nn[:, None]
        lo = torch.searchsorted(ll, mu - TAIL_CUT)
        hi = torch.searchsorted(ll, mu + TAIL_CUT)
        terms += float(torch.where(valid, hi - lo, torch.zeros_like(hi)).sum().item())
        n64 = nn.to(torch.float64)
        cells += float(n64.sum().item())
        pairs += float((n64 * (n64 + 1)).sum().item())
        band += float(band_terms(n64, 6).sum().item())
    return cells, pairs, terms, band


def rle_work_counts(fsmi, v, vp, vd, prm, cell_runlen, K, poses_per_chunk=8):
    """Algorithmic work of one fused 3D launch, from the (bit-exact) encoder: virtual-cell samples
    (a 4-byte gather each), runs, and the FP32 work of the path each ray takes. Cell-level form
    (rays with n < cell_runlen * n_r): 2K + 2 FMAs per cell (the 2K + 1 taps of the banded
    convolution and the product with P(e_j)); under Theorem 5 the taps of each cell's window of
    kept pairs (window_conv in csrc/evalrle.cuh) and the product. Run pairs (the other rays): the
    A/B terms of pair_AB (csrc/evalrle.cuh), 6 FP32 operations each (window difference, weighted
    window, two accumulations, the power of x)."""
    import torch

    thm5 = prm.variant == fsmi.APPROX and prm.approx_reading == 0
    D = prm.trunc_delta
    tot = {"rays": 0, "samples": 0, "runs": 0, "cell_rays": 0, "cell_cells": 0, "pair_rays": 0, "pair_terms": 0,
           "window_taps": 0}

    def terms(Lu, Lv, t):  # pair_AB iterations: j in [max(0, -K - t), min(Lu - 1, Lv - 1 + K - t)]
        lo = torch.clamp(-K - t, min=0)
        hi = torch.minimum(Lu - 1, Lv - 1 + K - t)
        return torch.clamp(hi - lo + 1, min=0)

    for a in range(0, vp.shape[0], poses_per_chunk):
        pp = vp[a:a + poses_per_chunk]
        nrays = pp.shape[0] * vd.shape[0]
        off, _, rl = fsmi.rle_encode_3d(v, pp, vd, prm, capacity=nrays * int(prm.max_range))
        off = off.to(torch.int64)
        L = rl.to(torch.int64)[:int(off[-1])]
        cum = torch.cat([torch.zeros(1, dtype=torch.int64, device=L.device), torch.cumsum(L, 0)])
        n = cum[off[1:]] - cum[off[:-1]]
        nr = off[1:] - off[:-1]
        tot["rays"] += nrays
        tot["samples"] += int(n.sum())
        tot["runs"] += int(nr.sum())
        cell = n < cell_runlen * nr
        tot["cell_rays"] += int(cell.sum())
        tot["cell_cells"] += int(n[cell].sum())
        pair = (~cell) & (nr > 0)
        tot["pair_rays"] += int(pair.sum())
        ray = torch.repeat_interleave(torch.arange(nrays, device=L.device), nr)
        S = cum[:-1] - cum[off[:-1]][ray]  # run start within its ray
        keep = pair[ray]
        if thm5 and bool(cell.any()):
            # each cell j of run u keeps the cells [lo_j, hi_j): lo_j = max(s of the run holding
            # j - D, s_u - D), hi_j = min(e_u + D, e of the run holding j + D); taps |k - j| <= K
            crun = torch.repeat_interleave(torch.arange(L.numel(), device=L.device), L)  # run of each cell
            cray = ray[crun]
            base = cum[off[:-1]][cray]  # the ray's first cell
            j = torch.arange(crun.numel(), device=L.device) - base
            nc = n[cray]
            ra = crun[base + torch.clamp(j - D, min=0)]
            rb = crun[base + torch.minimum(j + D, nc - 1)]
            lo = torch.maximum(S[ra], S[crun] - D)
            hi = torch.minimum(S[crun] + L[crun] + D, S[rb] + L[rb])
            taps = torch.clamp(torch.minimum(hi, j + K + 1) - torch.maximum(lo, j - K), min=0)
            tot["window_taps"] += int(taps[cell[cray]].sum())
            del crun, cray, base, j, nc, ra, rb, lo, hi, taps
        if thm5:
            tot["pair_terms"] += int(L[keep].sum())  # the diagonal blocks (theta, gamma): L_u terms
            for k in range(1, D + 2):  # runs within Delta of run u lie at most Delta + 1 runs away
                u, w = torch.arange(0, L.numel() - k, device=L.device), torch.arange(k, L.numel(), device=L.device)
                ok = keep[u] & (ray[u] == ray[w])
                su, Lu, sv, Lv = S[u], L[u], S[w], L[w]
                up = ok & (sv < su + Lu + D)  # u < v
                su2 = torch.maximum(su, sv - D)
                tot["pair_terms"] += int(torch.where(up, terms(su + Lu - su2, torch.minimum(Lv, su + Lu + D - sv),
                                                               su2 - sv), 0).sum())
                dn = ok & (su + Lu + D > sv)  # the same pair seen from v (v > u): sub-block below v
                # v as the first-hit run, u below it: Lu' = min(L_v, s_u + L_u + D - s_v), Lv' from s_v - D
                sv2 = torch.maximum(su, sv - D)
                tot["pair_terms"] += int(torch.where(dn, terms(torch.minimum(Lv, su + Lu + D - sv), su + Lu - sv2,
                                                               sv - sv2), 0).sum())
        elif bool(pair.any()):
            rid = torch.nonzero(pair).squeeze(1)
            m = int(nr[rid].max())
            idx = off[:-1][rid][:, None] + torch.arange(m, device=L.device)[None, :]
            valid = torch.arange(m, device=L.device)[None, :] < nr[rid][:, None]
            idx = torch.where(valid, idx, torch.zeros_like(idx))
            Sr, Lr = S[idx], L[idx]
            t = Sr[:, :, None] - Sr[:, None, :]
            c = terms(Lr[:, :, None], Lr[:, None, :], t)
            c = torch.where(valid[:, :, None] & valid[:, None, :], c, torch.zeros_like(c))
            tot["pair_terms"] += int(c.sum())
        del off, rl, L, cum
    if thm5:
        tot["fp32_ops"] = tot["window_taps"] + tot["cell_cells"] + 6 * tot["pair_terms"]
    else:
        tot["fp32_ops"] = tot["cell_cells"] * (2 * K + 2) + 6 * tot["pair_terms"]
    return tot


def rle_crossover_leg(dev):
    """The paper's run-length experiment (beams of 256 unit cells made of groups of L cells of equal
    occupancy; 100,000 beams rather than the paper's 1000, so that the GPU times throughput and not
    launch latency): exact FSMI on the cells (fsmi_eval_beams) against FSMI-RLE on the runs
    (fsmi_eval_rle, Gaussian mass of a unit cell, runs split at 64), same values."""
    import numpy as np
    import torch

    from paper_1905_02238_gb300 import fsmi

    rng = np.random.default_rng(15)
    nb, n = 100_000, 256
    prm_c = fsmi.Params(variant=fsmi.EXACT, sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP, max_range=float(n))
    prm_r = fsmi.Params(variant=fsmi.EXACT, sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP, max_range=float(n),
                        run_cap=64, g_kernel=fsmi.G_ERF)
    off = torch.arange(nb + 1, dtype=torch.int32, device=dev) * n
    l = torch.arange(n, dtype=torch.float32, device=dev).repeat(nb)
    lend = torch.full((nb,), float(n), dtype=torch.float32, device=dev)
    ws = torch.empty(fsmi.QUEUE_BYTES, dtype=torch.uint8, device=dev)
    # the paper's pairing (Table 2): Approx-FSMI (Delta = 3) on the cells vs Approx-FSMI-RLE on the runs
    prm_ac = fsmi.Params(variant=fsmi.APPROX, trunc_delta=3, sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP,
                         max_range=float(n))
    prm_ar = fsmi.Params(variant=fsmi.APPROX, trunc_delta=3, sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP,
                         max_range=float(n), run_cap=64, g_kernel=fsmi.G_ERF)
    paper_ratio = {1: 0.2, 2: 0.7, 4: 1.8, 8: 4.6, 16: 7.4, 32: 11.2, 64: 16.5, 128: 24.4}  # Table 2, one CPU core
    rows = []
    for L in (1, 2, 4, 8, 16, 32, 64, 128):
        ng = -(-n // L)
        og = rng.uniform(0.0, 1.0, (nb, ng)).astype(np.float32)
        o = torch.from_numpy(np.repeat(og, L, axis=1)[:, :n].reshape(-1).copy()).to(dev)
        lens = [min(L, n - k * L) for k in range(ng)]
        split = [(g, min(64, ln - s)) for g, ln in enumerate(lens) for s in range(0, ln, 64)]
        gi = np.array([g for g, _ in split])
        rl = torch.from_numpy(np.tile(np.array([x for _, x in split], np.uint8), nb)).to(dev)
        ro = torch.from_numpy(og[:, gi].reshape(-1).copy()).to(dev)
        roff = torch.arange(nb + 1, dtype=torch.int32, device=dev) * len(split)
        oc = torch.empty(nb, dtype=torch.float32, device=dev)
        orr = torch.empty(nb, dtype=torch.float32, device=dev)
        ms_c = _time_ms(lambda: fsmi.eval_beams(off, o, l, lend, prm_c, out=oc, ws=ws), reps=10)
        ms_auto = _time_ms(lambda: fsmi.eval_rle(roff, ro, rl, prm_r, out=orr, ws=ws), reps=10)
        saved = fsmi.get_schedule(fsmi.KIND_RLE)
        fsmi.set_schedule(fsmi.KIND_RLE, dataclasses.replace(saved, cell_runlen=1))  # run pairs always
        try:
            ms_r = _time_ms(lambda: fsmi.eval_rle(roff, ro, rl, prm_r, out=orr, ws=ws), reps=10)
        finally:
            fsmi.set_schedule(fsmi.KIND_RLE, saved)
        diff = float(((orr - oc).abs() / oc.abs().clamp_min(1e-30)).max().item())
        ms_ac = _time_ms(lambda: fsmi.eval_beams(off, o, l, lend, prm_ac, out=oc, ws=ws), reps=10)
        ms_ar = _time_ms(lambda: fsmi.eval_rle(roff, ro, rl, prm_ar, out=orr, ws=ws), reps=10)
        rows.append({"L": L, "runs_per_beam": len(split), "cells_ms": ms_c, "rle_run_pairs_ms": ms_r,
                     "rle_default_ms": ms_auto, "run_pairs_speedup": ms_c / ms_r, "max_rel_diff": diff,
                     "approx_cells_ms": ms_ac, "approx_rle_ms": ms_ar, "approx_rle_speedup": ms_ac / ms_ar,
                     "paper_approx_rle_speedup": paper_ratio[L]})
    faster = [r["L"] for r in rows if r["rle_run_pairs_ms"] < r["cells_ms"]]
    return {"workload": "100,000 beams x 256 unit cells in groups of L cells of equal U(0,1) occupancy; exact FSMI "
                        "per cell (fsmi_eval_beams) vs FSMI-RLE on the runs (fsmi_eval_rle, unit-cell Gaussian "
                        "mass; run pairs always, and with the default schedule that takes the cell form for "
                        "mean run lengths below 32); and the paper's pairing, Approx-FSMI (Delta = 3) per cell "
                        "vs Approx-FSMI-RLE (Theorem 5) on the runs, beside the paper's ratios (Table 2: "
                        "Xeon E5-2695, one core, 1000 beams)",
            "rows": rows, "run_pairs_faster_from_L": faster[0] if faster else None}


def _time_ms(fn, reps=5):
    import torch

    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def pipe_rates_leg(dev):
    """Measured denominators of the rooflines (fsmi_probe): SM clock, SFU ex2 / rcp and FP32 /
    packed-FP32 FMA issue rates per SM per clock, L2 read bandwidth (a 32 MB buffer, well inside
    the 126 MB L2, read 32 times per launch) and HBM read bandwidth (a 2 GB buffer read once)."""
    import torch

    from paper_1905_02238_gb300 import fsmi

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    cyc = torch.zeros(1, dtype=torch.int64, device=dev)
    sink = torch.zeros(4, dtype=torch.float32, device=dev)

    def mhz():
        ms = _time_ms(lambda: fsmi.probe(fsmi.PROBE_SPIN, 1 << 24, cyc), reps=1)
        return float(cyc.item()) / (ms * 1e3)

    f0 = mhz()
    rates = {}
    iters = 4096
    for name, kind in (("ex2", fsmi.PROBE_EX2), ("rcp", fsmi.PROBE_RCP), ("fma", fsmi.PROBE_FMA),
                       ("fma_f32x2_instructions", fsmi.PROBE_FMA2)):
        ms = _time_ms(lambda: fsmi.probe(kind, iters, sink), reps=2)
        rates[name] = fsmi.probe_threads(kind) * iters * 8 / (ms * 1e-3)  # lane operations per second
    f1 = mhz()
    f = 0.5 * (f0 + f1)
    per_clk = {k: v / sms / (f * 1e6) for k, v in rates.items()}
    l2buf = torch.ones((32 << 20) // 4, dtype=torch.float32, device=dev)
    ms_l2 = _time_ms(lambda: fsmi.probe(fsmi.PROBE_READ, 32, l2buf), reps=3)
    del l2buf
    hbuf = torch.ones((2 << 30) // 4, dtype=torch.float32, device=dev)
    ms_hbm = _time_ms(lambda: fsmi.probe(fsmi.PROBE_READ, 1, hbuf), reps=3)
    del hbuf
    return {"sm_mhz_before_after": [f0, f1], "per_sm_per_clock": per_clk,
            "l2_read_gbs": 32 * (32 << 20) / (ms_l2 * 1e-3) / 1e9, "hbm_read_gbs": (2 << 30) / (ms_hbm * 1e-3) / 1e9,
            "nominal_per_sm_per_clock": {"ex2": 32, "rcp": 16, "fma": 128, "fma_f32x2_instructions": 64},
            "how": "fsmi_probe kernels, CUDA events: 152 SMs x 8 blocks x 256 threads, 8 chains of 4096 dependent "
                   "operations per thread (rcp chains add one add.f32 each); reads cached in L2 only (ld.global.cg)"}


def _sched(s):
    return {"warps_per_block": s.warps_per_block, "blocks_per_sm": s.blocks_per_sm, "queue_chunk": s.queue_chunk,
            "cell_runlen": s.cell_runlen}


def roofline(bound, achieved, peak, unit, kernel, model, traffic=None, **extra):
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
            "traffic": traffic, "kernel": kernel, "model": model, **extra}


def other_variants(g, p, d, out, cells=None, terms=None, band=None, peak_terms=None, pipes=None,
                   sm_mhz=None):  # noqa: C901
    """Throughput of the other variants on the same devices (context; not the headline), each
    with its roofline. The 3D variants run as the 512x512x128 depth-camera batch in one persistent
    launch with an autotuned schedule, captured in a CUDA graph and timed by graph replays."""
    import numpy as np
    import torch

    from paper_1905_02238_gb300 import fsmi, synth

    res = {}
    sms = torch.cuda.get_device_properties(g.device).multi_processor_count
    f_hz = (sm_mhz or 2070.0) * 1e6
    l2_gbs = pipes["l2_read_gbs"] if pipes else None
    fma_peak = sms * FMA_LANES_PER_SM_CLK * f_hz  # FP32 lane operations per second
    nb = p.shape[0] * d.shape[0]
    gains_ws = torch.empty(fsmi.workspace_size(fsmi.FN_EVAL_2D, g.numel()), dtype=torch.uint8, device=g.device)
    for name, kw, nterms in (("exact_fsmi_full_sweep", dict(variant=fsmi.EXACT, flags=fsmi.FLAG_FULL_SWEEP), None),
                             ("exact_fsmi_full_window", dict(variant=fsmi.EXACT, flags=fsmi.FLAG_FULL_WINDOW), None),
                             ("approx_fsmi_delta6", dict(variant=fsmi.APPROX, trunc_delta=6), band),
                             ("uniform_fsmi_h4", dict(variant=fsmi.UNIFORM, uniform_h=4), None)):
        prm = fsmi.Params(sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP, max_range=R_MAX, **kw)
        traffic = TRAFFIC.get(name) if TRAFFIC["sources_sha1"] == kernel_sources_sha1() else None
        ms = _time_ms(lambda: fsmi.eval_2d(g, p, d, prm, out=out, ws=gains_ws))
        res[name] = {"beams_per_s": nb / (ms * 1e-3), "ms": ms}
        if cells:
            res[name]["cells_per_s"] = cells / (ms * 1e-3)
        if nterms:
            res[name]["band_terms_per_s"] = nterms / (ms * 1e-3)
            if peak_terms and cells:
                # Approx evaluates band + 1 boundary tails per first-hit cell (one ex2, one rcp each)
                res[name]["roofline_sfu_frac"] = (nterms + cells) / (ms * 1e-3) / peak_terms
                res[name]["roofline"] = roofline(
                    "alu", (nterms + cells) / (ms * 1e-3) / 1e12, peak_terms / 1e12, "T tail-terms/s (SFU)",
                    "k_eval_2d<APPROX,map>",
                    f"{nterms + cells:.4g} boundary tails per launch (sum over first-hit cells j of the band "
                    f"[j - 6, j + 6] clipped to the beam, plus one: its boundaries), one ex2 and one rcp each",
                    traffic=traffic)
        if name == "uniform_fsmi_h4" and cells and l2_gbs:
            # Algorithm 4 after the per-map-cell gains: per visited cell one 16-byte gather of
            # (o, f_occ, f_emp) from the L2-resident gains array, prefix sums and O(1) arithmetic
            res[name]["roofline"] = roofline(
                "l2", 16 * cells / (ms * 1e-3) / 1e9, l2_gbs, "GB/s", "k_eval_2d<UNIFORM,map>",
                f"{cells:.4g} visited cells per launch x 16 B gathered (per-map-cell gains, L2-resident) "
                "against the measured L2 read bandwidth (pipe_rates); the kernel is bound by issue "
                "(traversal, gathers, scans), not by either pipe", traffic=traffic)
    if terms:
        res["exact_fsmi_window_terms"] = terms
    # the 200x200 random grid (correctness workload, launch-latency bound): one pose x 360 beams, R = 64
    g1, p1, d1 = (torch.from_numpy(x).to(g.device) for x in synth.random_grid_200())
    o1 = torch.empty((1, 360), dtype=torch.float32, device=g.device)
    prm1 = fsmi.Params(variant=fsmi.EXACT, sigma=1.5, delta_occ=DOCC, delta_emp=DEMP, max_range=64.0)
    ws1 = torch.empty(fsmi.QUEUE_BYTES, dtype=torch.uint8, device=g.device)
    graph1 = fsmi.Graph(lambda: fsmi.eval_2d(g1, p1, d1, prm1, out=o1, ws=ws1))
    res["grid200_exact"] = {"us_per_launch_graph": 1e3 * _time_ms(graph1.replay, reps=200),
                            "us_per_call": 1e3 * _time_ms(lambda: fsmi.eval_2d(g1, p1, d1, prm1, out=o1, ws=ws1),
                                                          reps=200),
                            "workload": "200x200 grid, 1 pose x 360 beams, R = 64, sigma = 1.5; per call = "
                                        "through the Python binding (host launch overhead included)"}
    graph1.close()
    vox, vp, vd = synth.voxel_scene()
    v, vp, vd = (torch.from_numpy(x).to(g.device) for x in (vox, vp, vd))
    nr = vp.shape[0] * vd.shape[0]
    out3 = torch.empty((vp.shape[0], vd.shape[0]), dtype=torch.float32, device=g.device)
    ws3 = torch.empty(fsmi.QUEUE_BYTES, dtype=torch.uint8, device=g.device)
    saved = fsmi.get_schedule(fsmi.KIND_RLE)
    for name, kw in (("fsmi_rle_3d", dict(variant=fsmi.EXACT)), ("approx_fsmi_rle_3d_delta6", dict(variant=fsmi.APPROX)),
                     ("approx_fsmi_rle_3d_delta6_band", dict(variant=fsmi.APPROX, approx_reading=1)),
                     ("uniform_fsmi_rle_3d_h4", dict(variant=fsmi.UNIFORM))):
        prm = fsmi.Params(sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP, max_range=384.0, run_cap=64, trunc_delta=6,
                          uniform_h=4, **kw)
        fsmi.set_schedule(fsmi.KIND_RLE, saved)

        def call():
            fsmi.eval_3d(v, vp, vd, prm, out=out3, ws=ws3)

        ms_default = _time_ms(call)
        best, _, _ = fsmi.autotune(fsmi.KIND_RLE, call, reps=2)
        graph = fsmi.Graph(call)
        ms = _time_ms(graph.replay)
        graph.close()
        res[name] = {"rays_per_s": nr / (ms * 1e-3), "ms": ms, "ms_default_schedule_no_graph": ms_default,
                     "schedule": _sched(best),
                     "workload": "512x512x128 voxels, 64 poses x 128x128 rays, 384 virtual cells, fused sample+RLE+MI, "
                                 "autotuned schedule, CUDA-graph replay"}
        K = 4 if prm.variant == fsmi.UNIFORM else (6 if prm.approx_reading == 1 else int(np.ceil(7.45 * SIGMA)))
        wc = rle_work_counts(fsmi, v, vp, vd, prm, best.cell_runlen or 32, K)
        res[name]["work"] = wc
        sec = ms * 1e-3
        fr_fma = wc["fp32_ops"] / sec / fma_peak
        l2_bytes = 4 * wc["samples"] + 4 * nr
        if l2_gbs:
            fr_l2 = l2_bytes / sec / 1e9 / l2_gbs
            # the kernel's DRAM bytes per launch (ncu), whichever roofline binds
            traffic = TRAFFIC_3D.get(name) if TRAFFIC_3D.get("sources_sha1") == kernel_sources_sha1(
                KERNEL_SOURCES_3D) else None
            rl2 = roofline("l2", l2_bytes / sec / 1e9, l2_gbs, "GB/s", f"k_eval_3d ({name})",
                           f"{wc['samples']:.4g} virtual-cell samples x 4 B gathered + 4 B out per ray, against the "
                           "measured L2 read bandwidth (the 134 MB volume is mostly L2-served)", traffic=traffic)
            rfma = roofline("alu", wc["fp32_ops"] / sec / 1e12, fma_peak / 1e12, "T FP32 ops/s", f"k_eval_3d ({name})",
                            (f"{wc['cell_cells']:.4g} cells of cell-form rays: {wc['window_taps']:.4g} window taps "
                             f"(Theorem 5's kept pairs, |k - j| <= {K}) + 1 FMA each"
                             if wc["window_taps"] else
                             f"{wc['cell_cells']:.4g} cells of cell-form rays x {2 * K + 2} FMAs (banded convolution, "
                             f"K = {K})") + f" + {wc['pair_terms']:.4g} run-pair A/B terms x 6 FP32 ops",
                            traffic=traffic)
            res[name]["roofline"] = rl2 if fr_l2 >= fr_fma else rfma
            res[name]["roofline_other"] = rfma if fr_l2 >= fr_fma else rl2
    fsmi.set_schedule(fsmi.KIND_RLE, saved)
    return res


SURR_FLOPS_PER_BEAM = 2 * (128 * 32 * 6 + 64 * 32 * 96 + 32 * 32 * 96 + 1024 * 256 + 256)  # conv1-3, fc1, fc2


PRESCREEN_MIN_RANGE = 96.0  # shorter beams are cheap to evaluate exactly; the network's cost is per beam


def surrogate_leg(dev, steps: int = 2500):
    """Surrogate prescreen: train the surrogate on 10.3 M beams that exact FSMI labels (7 office maps x 4096
    poses x 360 beams), then select the best 10 of 4096 candidate poses on a held-out map by
    surrogate prescreen + exact rerank of the top 64, against exact FSMI of every beam. Both
    selections run as CUDA-graph replays. Returns (result, network)."""
    import numpy as np
    import torch

    from paper_1905_02238_gb300 import fsmi, synth
    from paper_1905_02238_gb300 import surrogate as sg

    d = torch.from_numpy(synth.beam_dirs_2d(360)).to(dev)
    prm = fsmi.Params(variant=fsmi.EXACT, sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP, max_range=R_MAX)
    t0 = time.perf_counter()
    maps = sg.label_maps(7, 4096, d, prm, seed=100)
    torch.cuda.synchronize()
    t_label = time.perf_counter() - t0
    lab = torch.cat([m.labels for m in maps])
    net = sg.Surrogate(seed=0, scale=float(lab.std()), shift=float(lab.mean()))
    t0 = time.perf_counter()
    losses = net.train(maps, d, steps=steps, batch=4096, lr=2e-3, log_every=steps // 4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    grid, poses, _ = synth.office_scene(n_poses=4096, seed=200, pose_seed=201)
    g, p = torch.from_numpy(grid).to(dev), torch.from_numpy(poses).to(dev)
    ex = sg.ExactAll(g, p, d, prm)
    pre = sg.Prescreen(net, g, p, d, prm, k=64)
    ex.run()
    found = pre.run()
    scores = ex.score.clone()
    truth = ex.best.clone()
    ex_graph, pre_graph = fsmi.Graph(ex.run), fsmi.Graph(pre.run)
    ms_exact = _time_ms(ex_graph.replay, reps=10)
    ms_pre = _time_ms(pre_graph.replay, reps=10)
    ms_pred = _time_ms(lambda: net.predict(g, p, d, out=pre.pred, ws=pre.ws_pred), reps=10)
    ex_graph.close()
    pre_graph.close()
    # frontier candidates: free cells 1-8 cells from unknown space, where the exact top 10 is
    # separated (no ties at 1e-5), so that strict recall discriminates
    fposes = synth.frontier_poses_2d(grid, 4096, seed=204, rmin=1.0, rmax=8.0)
    fp = torch.from_numpy(fposes).to(dev)
    fex = sg.ExactAll(g, fp, d, prm)
    fex.run()
    fpre = sg.Prescreen(net, g, fp, d, prm, k=64)
    ffound = fpre.run()
    fsc = fex.score.cpu().numpy().astype(np.float64)
    fsrt = np.sort(fsc)[::-1]
    frontier = {"workload": "the same held-out map, 4096 candidate poses at free cells 1-8 cells from unknown space",
                "tie_band_1e-4": sg.tie_band(fex.score, 10, 1e-4), "tie_band_1e-5": sg.tie_band(fex.score, 10, 1e-5),
                "gap_10th_11th_rel": float((fsrt[9] - fsrt[10]) / fsrt[9]),
                "recall_at_10_strict": sg.recall(ffound, fex.best),
                "recall_at_10_ties_1e-5": sg.recall_with_ties(ffound, fex.score, 10, 1e-5),
                "regret": sg.regret(ffound, fex.score),
                "ms": _time_ms(fpre.run, reps=10), "exact_all_ms": _time_ms(fex.run, reps=10)}
    frontier["poses_per_s"] = 4096 / (frontier["ms"] * 1e-3)
    frontier["speedup_vs_exact_all"] = frontier["exact_all_ms"] / frontier["ms"]
    del fex, fpre
    pred = pre.pred.cpu().numpy().astype(np.float64) * net.scale + net.shift
    exact = ex.mi.cpu().numpy().astype(np.float64).reshape(-1)
    rel = np.abs(pred - exact) / np.maximum(np.abs(exact), 1e-6)
    nb = p.shape[0] * d.shape[0]
    peaks = measured_peaks()
    tc = SURR_FLOPS_PER_BEAM * nb / (ms_pred * 1e-3) / 1e12
    return {
        "workload": "held-out 2048x2048 office map, 4096 candidate poses x 360 beams, R=256; surrogate "
                    "(1D conv 3x32 ch + MLP 256, BF16 weights) trained on 10.3 M exact-labelled beams "
                    "(7 maps x 4096 poses x 360); exact FSMI reranks the surrogate's top 64 poses",
        "poses_per_s": 4096 / (ms_pre * 1e-3), "ms": ms_pre,
        "exact_all_poses_per_s": 4096 / (ms_exact * 1e-3), "exact_all_ms": ms_exact,
        "speedup_vs_exact_all": ms_exact / ms_pre,
        "recall_at_10_ties_1e-4": sg.recall_with_ties(found, scores, 10, 1e-4),
        "recall_at_10_ties_1e-5": sg.recall_with_ties(found, scores, 10, 1e-5),
        "recall_at_10_strict": sg.recall(found, truth),
        "tie_band_1e-4": sg.tie_band(scores, 10, 1e-4), "tie_band_1e-5": sg.tie_band(scores, 10, 1e-5),
        "regret": sg.regret(found, scores),
        "frontier_candidates": frontier,
        "beam_mi_rel_err_median": float(np.median(rel)), "beam_mi_rel_err_p99": float(np.quantile(rel, 0.99)),
        "predict_ms": ms_pred,
        "tensor_cores": {"achieved_tflops": tc, "peak_tflops": peaks.get("bf16_tflops"), "unit": "TFLOP/s",
                         "frac": tc / peaks["bf16_tflops"] if peaks.get("bf16_tflops") else None,
                         "note": "mma.sync BF16 (conv stack + fc1), against the measured cuBLAS BF16 peak"},
        "training": {"label_s": t_label, "train_s": t_train, "steps": steps, "batch": 4096,
                     "loss_first_last": [losses[0], losses[-1]]},
    }, net


def surrogate_stream_leg(dev, net, k: int = 64, nsets: int = 32, seed: int = 5, pose_range=(16, 8192, 16, 512),
                         len_range=(8, 512, 8, 256)):
    """The mixed candidate-set stream with the surrogate: each 2D set of the stream whose range the network covers
    (R <= 256) and that has more than k poses selects its best 10 poses by surrogate prescreen
    (profiles cut at the set's range, which the network reads as the map ending there; it is
    trained at R = 256 only) + exact rerank of the top k, against exact FSMI of all its beams, and
    by a per-set choice of the two (prescreen from PRESCREEN_MIN_RANGE up). The sets run one after
    the other in stream order, all queued at time 0, so a set's latency is the sum of the service
    times up to it."""
    import numpy as np
    import torch

    from paper_1905_02238_gb300 import fsmi
    from paper_1905_02238_gb300 import surrogate as sg

    grid, poses2, dirs2, _, _, _, sets = stream_sets(nsets, seed, pose_range, len_range)
    g, p2, d2 = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (grid, poses2, dirs2))
    rows = []
    for s_ in sets:
        kind, po, npose, do, ndir, r = s_[:6]
        if kind != fsmi.SET_2D or r > fsmi.SURR_L or npose <= k:
            continue
        prm = fsmi.Params(variant=fsmi.EXACT, sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP, max_range=r)
        pg = p2[po:po + npose]
        ex = sg.ExactAll(g, pg, d2, prm)
        pre = sg.Prescreen(net, g, pg, d2, prm, k=k)
        ex.run()
        found = pre.run()
        scores = ex.score.clone()
        rows.append({"poses": npose, "range": r, "exact_ms": _time_ms(ex.run, reps=3),
                     "prescreen_ms": _time_ms(pre.run, reps=3),
                     "recall_at_10_ties_1e-4": sg.recall_with_ties(found, scores, 10, 1e-4),
                     "recall_at_10_strict": sg.recall(found, ex.best),
                     "tie_band_1e-4": sg.tie_band(scores, 10, 1e-4),
                     "regret": sg.regret(found, scores)})
        del ex, pre
    if not rows:
        return {"sets": 0}
    poses = sum(r_["poses"] for r_ in rows)

    for r_ in rows:
        use = r_["range"] >= PRESCREEN_MIN_RANGE
        r_["chosen_ms"] = r_["prescreen_ms"] if use else r_["exact_ms"]
        r_["chosen_recall"] = r_["recall_at_10_ties_1e-4"] if use else 1.0

    def summary(key):
        ms = np.array([r_[key] for r_ in rows])
        lat = np.cumsum(ms)
        return {"ms": float(ms.sum()), "poses_per_s": poses / (ms.sum() * 1e-3),
                "set_latency_ms_p50": float(np.percentile(lat, 50)), "set_latency_ms_p99": float(np.percentile(lat, 99))}

    rec = [r_["recall_at_10_ties_1e-4"] for r_ in rows]
    return {"workload": f"the 2D sets of the {nsets}-set stream (4096x4096 office map, 360 beams) with R <= "
                        f"{fsmi.SURR_L} and more than {k} poses; sets in stream order, all queued at t = 0",
            "sets": len(rows), "poses": poses, "exact_all": summary("exact_ms"),
            "prescreen_rerank": summary("prescreen_ms"),
            "speedup": sum(r_["exact_ms"] for r_ in rows) / sum(r_["prescreen_ms"] for r_ in rows),
            "recall_at_10_ties_1e-4": {"min": min(rec), "mean": float(np.mean(rec))},
            "per_set_choice": {**summary("chosen_ms"), "rule": f"prescreen when R >= {PRESCREEN_MIN_RANGE:g}, else exact",
                               "speedup": sum(r_["exact_ms"] for r_ in rows) / sum(r_["chosen_ms"] for r_ in rows),
                               "recall_at_10_min": min(r_["chosen_recall"] for r_ in rows)},
            "regret_max": max(r_["regret"] for r_ in rows), "rows": rows}


def stream_sets(nsets: int = 32, seed: int = 5, pose_range=(16, 8192, 16, 512), len_range=(8, 512, 8, 256)):
    """The mixed candidate-set stream: a 4096x4096 office map with 16384 free-cell poses and 360 beams, two
    256x256x64 voxel submaps with 512 poses each and 64x64 rays, and nsets candidate sets: 3 in 4
    are 2D (pose_range[0]-[1] poses, log-uniform; range len_range[0]-[1] cells), the rest 3D
    (pose_range[2]-[3] poses; len_range[2]-[3] virtual cells), as fsmi.make_sets tuples."""
    import numpy as np

    from paper_1905_02238_gb300 import fsmi, synth

    rng = np.random.default_rng(seed)
    grid = synth.office_grid(4096, n_obst=1600, seed=seed)
    poses2 = synth.free_cell_poses_2d(grid, 16384, seed=seed + 1)
    dirs2 = synth.beam_dirs_2d(360)
    vols = [synth.voxel_world(256, 256, 64, n_boxes=60, seed=seed + 10 + k, noise_seed=seed + 20 + k) for k in range(2)]
    poses3 = np.concatenate([synth.free_voxel_poses(v, 512, seed=seed + 30 + k, zlo=8, zhi=56)
                             for k, v in enumerate(vols)])
    dirs3 = synth.pinhole_dirs(64, 64, 90.0)
    sets = []
    for i in range(nsets):
        if rng.random() < 0.75:
            npose = int(np.exp(rng.uniform(np.log(pose_range[0]), np.log(pose_range[1]))))
            po = int(rng.integers(0, poses2.shape[0] - npose + 1))
            sets.append((fsmi.SET_2D, po, npose, 0, 360, float(rng.uniform(len_range[0], len_range[1]))))
        else:
            npose = int(np.exp(rng.uniform(np.log(pose_range[2]), np.log(pose_range[3]))))
            k = int(rng.integers(0, 2))
            sets.append((fsmi.SET_3D, 512 * k, npose, 0, 4096, float(rng.integers(len_range[2], len_range[3] + 1)), k))
    return grid, poses2, dirs2, vols, poses3, dirs3, sets


def mixed_leg(dev, nsets: int = 32, seed: int = 5, pose_range=(16, 8192, 16, 512), len_range=(8, 512, 8, 256)):
    """Mixed candidate sets: a stream of candidate sets on a 4096x4096 office map and two 256x256x64 voxel
    submaps, evaluated exactly (2D FSMI, sigma 2; 3D FSMI-RLE, sigma 2, run cap 64) in one
    persistent launch (fsmi_eval_mixed), against the same sets launched one after the other.
    Sets (default): 3 in 4 are 2D (16-8192 poses, log-uniform; 360 beams; range 8-512 cells), the
    rest 3D (16-512 poses; 64x64 rays; 8-256 virtual cells); pose_range and len_range give other
    streams. All sets are queued at time 0; a set's latency is the time until its last beam or ray
    is done."""
    import numpy as np
    import torch

    from paper_1905_02238_gb300 import fsmi, synth

    grid, poses2, dirs2, vols, poses3, dirs3, sets = stream_sets(nsets, seed, pose_range, len_range)
    g, p2, d2, p3, d3 = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (grid, poses2, dirs2, poses3, dirs3))
    vt = [torch.from_numpy(v).to(dev) for v in vols]
    vd = fsmi.make_volumes(vt, dev)
    st, n = fsmi.make_sets(sets, dev)
    prm2 = fsmi.Params(variant=fsmi.EXACT, sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP, max_range=float(len_range[1]))
    prm3 = fsmi.Params(variant=fsmi.EXACT, sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP, max_range=float(len_range[3]),
                       run_cap=64)
    out = torch.empty(n, dtype=torch.float32, device=dev)
    times = torch.zeros(n + 1, dtype=torch.int64, device=dev)
    # with room for the range-class plan: one launch per range class, in one call
    ws = torch.empty(fsmi.mixed_workspace_size(g.numel(), len(sets)), dtype=torch.uint8, device=dev)
    ws1 = torch.empty(fsmi.workspace_size(fsmi.FN_EVAL_2D, g.numel()), dtype=torch.uint8, device=dev)

    def mixed(w=ws):
        fsmi.eval_mixed(st, n, out=out, times=times, ws=w, grid=g, poses2=p2, dirs2=d2, prm2=prm2, volumes=vd,
                        poses3=p3, dirs3=d3, prm3=prm3)

    # the same sets, one launch each, in order
    seq_out = torch.empty(n, dtype=torch.float32, device=dev)
    ws3 = torch.empty(fsmi.QUEUE_BYTES, dtype=torch.uint8, device=dev)
    views, at = [], 0
    for s_ in sets:
        kind, po, npose, do, ndir, r = s_[:6]
        views.append((s_, seq_out[at:at + npose * ndir].view(npose, ndir)))
        at += npose * ndir
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(sets) + 1)]

    def sequential(record=False):
        if record:
            ev[0].record()
        for i, (s_, o) in enumerate(views):
            kind, po, npose, do, ndir, r = s_[:6]
            if npose:
                if kind == fsmi.SET_2D:
                    fsmi.eval_2d(g, p2[po:po + npose], d2[do:do + ndir], fsmi.Params(**{**prm2.__dict__, "max_range": r}),
                                 out=o, ws=ws)
                else:
                    fsmi.eval_3d(vt[s_[6]], p3[po:po + npose], d3[do:do + ndir],
                                 fsmi.Params(**{**prm3.__dict__, "max_range": r}), out=o, ws=ws3)
            if record:
                ev[i + 1].record()

    mixed(ws1)  # the single launch (no plan): every warp sized for the stream's longest beam or ray
    torch.cuda.synchronize()
    single_out = out.clone()
    ms_single = _time_ms(lambda: mixed(ws1), reps=3)
    mixed()
    sequential()
    torch.cuda.synchronize()
    ok = bool(torch.equal(out, seq_out)) and bool(torch.equal(single_out, seq_out))
    graph = fsmi.Graph(mixed)
    ms_mixed = _time_ms(graph.replay, reps=3)
    graph.replay()
    torch.cuda.synchronize()
    t = times.cpu().numpy().view(np.uint64).astype(np.float64)
    lat, at = [], 0
    for s_ in sets:
        m = s_[2] * s_[4]
        lat.append((t[1 + at:1 + at + m].max() - t[0]) * 1e-6 if m else 0.0)
        at += m
    ms_seq = _time_ms(sequential, reps=3)
    sequential(record=True)
    torch.cuda.synchronize()
    lat_seq = [ev[0].elapsed_time(ev[i + 1]) for i in range(len(sets))]
    graph.close()
    poses = sum(s_[2] for s_ in sets)
    n2 = sum(s_[2] * s_[4] for s_ in sets if s_[0] == fsmi.SET_2D)
    return {
        "workload": f"{nsets} candidate sets on a 4096x4096 office map ({sum(s_[0] == fsmi.SET_2D for s_ in sets)} 2D sets, "
                    f"{pose_range[0]}-{pose_range[1]} poses x 360 beams, R {len_range[0]}-{len_range[1]}) and two "
                    f"256x256x64 voxel submaps (3D sets, {pose_range[2]}-{pose_range[3]} poses x 64x64 rays, "
                    f"{len_range[2]}-{len_range[3]} virtual cells); exact FSMI / FSMI-RLE; all sets queued at t = 0",
        "items": n, "beams_2d": n2, "rays_3d": n - n2, "poses": poses,
        "one_launch": {"ms": ms_mixed, "poses_per_s": poses / (ms_mixed * 1e-3), "items_per_s": n / (ms_mixed * 1e-3),
                       "set_latency_ms_p50": float(np.percentile(lat, 50)),
                       "set_latency_ms_p99": float(np.percentile(lat, 99)),
                       "how": "one fsmi_eval_mixed call with the range-class plan (a launch per class), "
                              "captured in a CUDA graph"},
        "one_launch_without_plan_ms": ms_single,
        "launch_per_set": {"ms": ms_seq, "poses_per_s": poses / (ms_seq * 1e-3),
                           "set_latency_ms_p50": float(np.percentile(lat_seq, 50)),
                           "set_latency_ms_p99": float(np.percentile(lat_seq, 99))},
        "identical_results": ok,
    }


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle

    oracle.build()
    grid, poses, dirs = workload(0)
    prm = oracle.Params(variant=oracle.EXACT, sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP, max_range=R_MAX)
    threads = os.cpu_count() or 1
    per_step = 4  # poses per reference step (a bounded sample of the same batch)
    times = []
    for s in range(args.warmup + args.steps):
        sel = poses[(s * per_step) % N_POSES:(s * per_step) % N_POSES + per_step]
        t0 = time.perf_counter()
        oracle.eval_2d(grid, sel, dirs, prm, nthreads=threads)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    nb = per_step * dirs.shape[0]
    value = nb * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "beams/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": f"{per_step} poses x 360 beams"},
        "cpu_baseline": {"value": value, "unit": "beams/s", "cores": threads, "kind": "oracle",
                         "sample": f"{per_step} poses x {dirs.shape[0]} beams per step"},
        "e2e": {"value": value, "unit": "beams/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_fsmi(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_1905_02238_gb300 import build, fsmi

    build.build()
    fsmi.load()
    grid, poses, dirs = workload(rank, args.poses)
    g = torch.from_numpy(grid).to(dev)
    p = torch.from_numpy(poses).to(dev)
    d = torch.from_numpy(dirs).to(dev)
    P, B = poses.shape[0], dirs.shape[0]
    out = torch.empty((P, B), dtype=torch.float32, device=dev)
    prm = fsmi.Params(variant=fsmi.EXACT, sigma=SIGMA, delta_occ=DOCC, delta_emp=DEMP, max_range=R_MAX)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # algorithmic work of one launch, from the (bit-exact) traversal: Theorem 1 has n(n+1)
    # boundary terms per beam; the kernel evaluates those within its window
    cells, pairs, terms, band = work_counts(fsmi, grid, p, d)

    stream = torch.cuda.current_stream()

    gains_ws = torch.empty(fsmi.workspace_size(fsmi.FN_EVAL_2D, grid.size), dtype=torch.uint8, device=dev)

    def call():
        fsmi.eval_2d(g, p, d, prm, out=out, ws=gains_ws)

    # the step: the autotuned schedule (work queue, warps per block) captured once in a CUDA graph
    ms_default = _time_ms(call, reps=3)
    sched, cands, tune_ms = fsmi.autotune(fsmi.KIND_2D, call, reps=2)
    graph = fsmi.Graph(call)
    step = graph.replay

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        for i in range(args.steps):
            flush.fill_(float(i))  # evict the map from L2 between steps (untimed)
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    per = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = max_over_ranks(sum(per) / len(per), ws, dev)
    nbeams_all = P * B * ws
    value = whole_job_rate(P * B, ws, ms * 1e-3)

    # end to end through the public API with host buffers: every step copies its pinned inputs in
    # and its result out. fsmi.Pipeline2D overlaps one step's copies with the previous step's
    # evaluation; one synchronous fsmi.eval_2d call per step is reported beside it.
    hg, hp, hd = (torch.from_numpy(x).pin_memory() for x in (grid, poses, dirs))
    hres = [torch.empty((P, B), dtype=torch.float32).pin_memory() for _ in range(2)]
    pipe = fsmi.Pipeline2D(prm, grid.shape[1], grid.shape[0], P, B)
    for i in range(3):
        pipe.submit(hg, hp, hd, hres[i % 2])
    pipe.wait()
    for _ in range(2):
        fsmi.eval_2d(hg, hp, hd, prm)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    e2e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        pipe.submit(hg, hp, hd, hres[i % 2])
    pipe.wait()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, ws, dev)
    res = hres[(e2e_steps - 1) % 2]
    assert res.shape == (P, B) and bool(torch.isfinite(res).all())
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        res_sync = fsmi.eval_2d(hg, hp, hd, prm)
    torch.cuda.synchronize()
    e2e_sync_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, ws, dev)
    assert torch.equal(res_sync, res)
    h2d = grid.nbytes + poses.nbytes + dirs.nbytes
    d2h = P * B * 4

    if rank == 0:
        clocks = clk.summary()
        peaks = measured_peaks()
        sm_max = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak_ops = sms * FMA_LANES_PER_SM_CLK * sm_max * 1e6  # FMA-pipe ops/s at the maximum SM clock
        achieved_ops = terms * OPS_PER_TERM / (ms * 1e-3)
        peak_terms = sms * sm_max * 1e6 / SFU_CLK_PER_TERM  # tail terms/s the SFU allows
        achieved_terms = terms / (ms * 1e-3)
        traffic = TRAFFIC["bytes_per_launch"] if TRAFFIC["sources_sha1"] == kernel_sources_sha1() else None
        line = {
            "metric": METRIC, "value": value, "unit": "beams/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "poses_per_gpu": P, "beams_per_pose": B, "cells": cells,
                       "theorem1_terms": pairs, "evaluated_terms": terms,
                       "l2": "flushed between timed steps (512 MB write)",
                       "launch": "one CUDA-graph replay per step (queue reset, per-cell gains, beams)",
                       "schedule": _sched(sched), "ms_default_schedule_no_graph": ms_default,
                       "autotune_ms": {f"{c.warps_per_block}w/q{c.queue_chunk}": round(t, 4)
                                       for c, t in zip(cands, tune_ms)},
                       "parallelism": f"dp{ws} (poses sharded, map replicated)"},
            "roofline": {"bound": "alu", "achieved": achieved_terms / 1e12, "peak": peak_terms / 1e12,
                         "unit": "T tail-terms/s (SFU)", "frac": achieved_terms / peak_terms, "traffic": traffic,
                         "kernel": "k_eval_2d<EXACT,map>",
                         "fma_frac": achieved_ops / peak_ops,
                         "model": f"{terms:.4g} evaluated tail terms per launch, each one ex2 and one rcp on the "
                                  f"SFU ({EX2_PER_SM_CLK} and {RCP_PER_SM_CLK} per SM per clock: the binding pipe) "
                                  f"and {OPS_PER_TERM} FMA-pipe ops ({FMA_LANES_PER_SM_CLK} lanes per SM per clock; "
                                  f"fma_frac); peak = {sms} SMs x {sm_max:.0f} MHz"},
            "clocks": clocks,
            "e2e": {"value": whole_job_rate(P * B, ws, e2e_s), "unit": "beams/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "how": "fsmi.Pipeline2D: pinned inputs copied in and the result copied out every step, "
                           "one step's copies overlapped with the previous step's evaluation",
                    "one_call_per_step": whole_job_rate(P * B, ws, e2e_sync_s)},
            "gpu_launches": 2 * args.steps,  # per step: per-cell gains of the map, then the beams
        }
        if ws == 1 and not args.no_context:
            exact_out = out.cpu().numpy()  # the timed steps' result, before the context runs reuse `out`
            line["pipe_rates"] = pipe_rates_leg(dev)
            line["variants"] = other_variants(g, p, d, out, cells=cells, terms=terms, band=band,
                                              peak_terms=peak_terms, pipes=line["pipe_rates"], sm_mhz=sm_max)
            fw = line["variants"]["exact_fsmi_full_window"]
            # beside the headline: the same batch with every non-zero term of Theorem 1's n(n+1) sum,
            # bit-identical to the full sweep (FSMI_FLAG_FULL_WINDOW); 5 back-to-back calls, no graph
            line["full_window"] = {"value": fw["beams_per_s"], "unit": "beams/s", "ms": fw["ms"],
                                   "flag": "FSMI_FLAG_FULL_WINDOW"}
            line["rle_vs_cells"] = rle_crossover_leg(dev)
            net = None
            if not args.no_surrogate:
                line["surrogate_rerank"], net = surrogate_leg(dev)
            if not args.no_mixed:
                line["mixed_stream"] = mixed_leg(dev)
                line["mixed_stream_small_sets"] = mixed_leg(dev, nsets=256, seed=6, pose_range=(16, 128, 4, 16),
                                                            len_range=(8, 64, 8, 64))
                if net is not None:
                    line["mixed_stream_surrogate"] = surrogate_stream_leg(dev, net)
            line["cpu_baseline"] = cpu_baseline(grid, poses, dirs, gpu_out=exact_out)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def relaunch_cmd(n: int, argv: list[str], port: int) -> list[str]:
    """The torchrun command that runs this script as n local ranks (one per GPU) with argv."""
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
            "--master-addr", "127.0.0.1", f"--master-port={port}", os.path.abspath(__file__), *argv]


def free_port() -> int:
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def check_ranks() -> int:
    """--check-ranks: every rank joins a gloo group (no GPU work, nothing timed) and rank 0 prints
    how many joined: a self-check of the launcher, not a benchmark line."""
    import torch
    import torch.distributed as dist

    ws, rank, _ = dist_env()
    if ws > 1:
        dist.init_process_group("gloo")
        t = torch.ones(1)
        dist.all_reduce(t)
        joined = int(t.item())
        dist.destroy_process_group()
    else:
        joined = 1
    if rank == 0:
        print(json.dumps({"check": "ranks", "world_size": ws, "ranks_joined": joined}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["fsmi", "reference"], default="fsmi")
    ap.add_argument("--poses", type=int, default=N_POSES, help="poses per GPU (smaller for profiling cases)")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate leg (profiling runs)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed candidate-set stream leg")
    ap.add_argument("--no-context", action="store_true", help="only the timed steps (profiling runs)")
    ap.add_argument("--check-ranks", action="store_true", help="launcher self-check: join the ranks, report, exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws = int(os.environ.get("WORLD_SIZE", "0"))
    if args.gpus > 1 and ws == 0:
        # --gpus N without a launcher: start N local ranks (one process per GPU) and wait for them
        return subprocess.call(relaunch_cmd(args.gpus, sys.argv[1:], free_port()))
    if ws and ws != args.gpus:
        sys.stderr.write(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={ws}: the rank count must match\n")
        return 2
    if args.check_ranks:
        return check_ranks()
    if args.impl == "reference":
        return run_reference(args)
    return run_fsmi(args)


if __name__ == "__main__":
    sys.exit(main())
