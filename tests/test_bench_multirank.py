"""Host-side logic of bench.py's multi-GPU path, run as world_size-2 gloo ranks on CPU: each rank
gets its own poses (weak scaling, no data-path collective), the timing is the slowest rank's, and
the whole-job rate counts every rank's beams."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    assert bench.dist_env() == (ws, rank, rank)
    grid, poses, dirs = bench.workload(rank, n_poses=16)
    worst = bench.max_over_ranks(10.0 + rank, ws, torch.device("cpu"))
    rate = bench.whole_job_rate(poses.shape[0] * dirs.shape[0], ws, worst * 1e-3)
    q.put((rank, poses.copy(), worst, rate, float(grid.sum())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_poses_and_take_the_slowest_time():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, p0, w0, r0, g0), (_, p1, w1, r1, g1) = res
    assert not np.array_equal(p0, p1)  # each rank evaluates its own candidate poses
    assert g0 == g1  # on the same (replicated) map
    assert w0 == w1 == 11.0  # the job's time is the slowest rank's
    assert r0 == r1 == 2 * 16 * 360 / 11.0e-3


def test_gpus_flag_starts_that_many_ranks():
    # python bench.py --gpus 2 without a launcher re-launches itself as two torchrun ranks; the
    # launcher self-check joins them in a gloo group (no GPU work) and reports the count
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--check-ranks"],
                       capture_output=True, text=True, timeout=300, env=env, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert line == {"check": "ranks", "world_size": 2, "ranks_joined": 2}


def test_rank_count_mismatch_fails_loudly():
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, WORLD_SIZE="3", RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--check-ranks"],
                       capture_output=True, text=True, timeout=120, env=env, cwd=root)
    assert r.returncode == 2 and "WORLD_SIZE=3" in r.stderr
