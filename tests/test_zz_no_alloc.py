"""fsmi_rle_encode_3d_noalloc: the run-length encoder for callers that cannot allocate device
memory when they encode (a real-time planning loop with its memory reserved up front, or code
handed only input and output pointers). Its offset scan uses a library-owned array instead of a
caller workspace.

Called through the C ABI (ctypes), its runs must equal those of fsmi_rle_encode_3d (which takes a
caller workspace) bit for bit, on two calls in a row with different inputs, since every call
reuses the same library-owned array. Sizes beyond the array's limit are rejected before launch.
This file is collected last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


class _P(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("sigma", ctypes.c_float), ("delta_occ", ctypes.c_float),
                ("delta_emp", ctypes.c_float), ("trunc_delta", ctypes.c_int), ("uniform_h", ctypes.c_int),
                ("max_range", ctypes.c_float), ("run_cap", ctypes.c_int), ("g_kernel", ctypes.c_int),
                ("e0_mode", ctypes.c_int), ("approx_reading", ctypes.c_int), ("flags", ctypes.c_int)]


@pytest.fixture(scope="module")
def lib():
    from paper_1905_02238_gb300 import build

    path = build.build()
    torch.cuda.init()
    lib = ctypes.CDLL(path)
    vp, i = ctypes.c_void_p, ctypes.c_int
    lib.fsmi_rle_encode_3d.argtypes = [vp, i, i, i, vp, i, vp, i, ctypes.POINTER(_P), vp, vp, vp, i, vp,
                                       ctypes.c_size_t, vp]
    lib.fsmi_rle_encode_3d_noalloc.argtypes = [vp, i, i, i, vp, i, vp, i, ctypes.POINTER(_P), vp, vp, vp, i, vp]
    lib.fsmi_workspace_size.argtypes = [i, ctypes.c_longlong, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_size_t)]
    for f in (lib.fsmi_rle_encode_3d, lib.fsmi_rle_encode_3d_noalloc, lib.fsmi_workspace_size):
        f.restype = ctypes.c_int
    return lib


def _world(seed):
    from paper_1905_02238_gb300 import synth

    vox = synth.voxel_world(72, 56, 40, n_boxes=10, seed=seed, noise_seed=seed + 11, noise_frac=0.08)
    poses = synth.free_voxel_poses(vox, 5, seed=seed + 3, zlo=6, zhi=34)
    dirs = synth.pinhole_dirs(24, 20, 100.0)
    return (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (vox, poses, dirs))


def _encode(lib, noalloc, vox, poses, dirs, prm, capacity):
    Z, Y, X = vox.shape
    P, R = poses.shape[0], dirs.shape[0]
    off = torch.full((P * R + 1,), -7, dtype=torch.int32, device="cuda")
    ro = torch.full((capacity,), -1.0, dtype=torch.float32, device="cuda")
    rl = torch.zeros(capacity, dtype=torch.uint8, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = [ctypes.c_void_p(vox.data_ptr()), X, Y, Z, ctypes.c_void_p(poses.data_ptr()), P,
            ctypes.c_void_p(dirs.data_ptr()), R, ctypes.byref(prm), ctypes.c_void_p(off.data_ptr()),
            ctypes.c_void_p(ro.data_ptr()), ctypes.c_void_p(rl.data_ptr()), capacity]
    if noalloc:
        st = lib.fsmi_rle_encode_3d_noalloc(*args, s)
    else:
        need = ctypes.c_size_t(0)
        assert lib.fsmi_workspace_size(2, P * R, ctypes.byref(prm), ctypes.byref(need)) == 0
        ws = torch.empty(max(int(need.value), 4), dtype=torch.uint8, device="cuda")
        st = lib.fsmi_rle_encode_3d(*args, ctypes.c_void_p(ws.data_ptr()), ws.numel(), s)
    assert st == 0
    torch.cuda.synchronize()
    return off.cpu(), ro.cpu(), rl.cpu()


def test_noalloc_encoder_matches_workspace_encoder_on_consecutive_calls(lib):
    prm = _P(0, 2.0, 1.5, 0.67, 6, 4, 96.0, 16, 0, 0, 0, 0)
    for seed in (1, 5):  # two calls in a row, different worlds: the shared array must not leak state
        vox, poses, dirs = _world(seed)
        a_off, a_o, a_l = _encode(lib, True, vox, poses, dirs, prm, 240000)
        b_off, b_o, b_l = _encode(lib, False, vox, poses, dirs, prm, 240000)
        assert torch.equal(a_off, b_off)
        n = int(b_off[-1])
        assert 0 < n <= 240000
        assert torch.equal(a_o[:n].view(torch.int32), b_o[:n].view(torch.int32))
        assert torch.equal(a_l[:n], b_l[:n])


def test_noalloc_encoder_matches_workspace_encoder_past_one_scan_chunk(lib):
    # More than 1024 scan tiles of 4096 rays, so that the scan of the tile totals carries between
    # its chunks of 1024 entries; first the larger batch, then a smaller one, so that the second
    # call reads only entries it wrote itself.
    from paper_1905_02238_gb300 import synth

    vox = synth.voxel_world(64, 64, 32, n_boxes=6, seed=9, noise_seed=10, noise_frac=0.1)
    dirs = torch.from_numpy(synth.pinhole_dirs(64, 64, 90.0)).cuda()
    v = torch.from_numpy(vox).cuda()
    prm = _P(0, 2.0, 1.5, 0.67, 6, 4, 6.0, 2, 0, 0, 0, 0)  # 6 virtual cells per ray, runs of at most 2
    for npose, seed in ((1100, 21), (1030, 22)):
        poses = torch.from_numpy(synth.free_voxel_poses(vox, npose, seed=seed, zlo=4, zhi=28)).cuda()
        nrays = npose * dirs.shape[0]
        assert nrays > 1024 * 4096
        cap = 6 * nrays
        a_off, a_o, a_l = _encode(lib, True, v, poses, dirs, prm, cap)
        b_off, b_o, b_l = _encode(lib, False, v, poses, dirs, prm, cap)
        assert torch.equal(a_off, b_off)
        n = int(b_off[-1])
        assert nrays <= n <= cap
        assert torch.equal(a_o[:n].view(torch.int32), b_o[:n].view(torch.int32))
        assert torch.equal(a_l[:n], b_l[:n])
        del a_o, b_o, a_l, b_l


def test_noalloc_encoder_rejects_batches_beyond_its_array(lib):
    vox, poses, dirs = _world(1)
    prm = _P(0, 2.0, 1.5, 0.67, 6, 4, 96.0, 16, 0, 0, 0, 0)
    Z, Y, X = vox.shape
    big_P = (4096 * 4096) // dirs.shape[0] + 1  # P * R just above the limit
    # a poses buffer that really holds big_P poses: were the host check ever lost, the kernels
    # would still read only inside it
    big_poses = poses[torch.arange(big_P, device="cuda") % poses.shape[0]].contiguous()
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.fsmi_rle_encode_3d_noalloc(ctypes.c_void_p(vox.data_ptr()), X, Y, Z, ctypes.c_void_p(big_poses.data_ptr()),
                                        big_P, ctypes.c_void_p(dirs.data_ptr()), dirs.shape[0], ctypes.byref(prm),
                                        ctypes.c_void_p(out.data_ptr()), None, None, 0, s)
    assert st == 2  # FSMI_ERR_CAPACITY, checked on the host: nothing was launched
    torch.cuda.synchronize()
    assert torch.all(out == 0)
