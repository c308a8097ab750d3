"""FP64 CPU oracle of the learned surrogate (test infrastructure only).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs
may import this module. It shares no code with the CUDA library.

The surrogate is not part of the paper. It is a small network that predicts the FSMI of one 2D
beam from the beam's occupancy profile, used to prescreen candidate poses before exact FSMI
reranks the best of them. Architecture (fixed):

    input  x[256][2]: samples i = 0..255 of the beam at distance i + 1/2 cells; channel 0 = o of
           the cell holding the sample, channel 1 = 1 inside the map (0 and 0 beyond it)
    conv1  2 -> 32 channels, kernel 3, stride 2, zero padding 1, ReLU    (256 -> 128 positions)
    conv2  32 -> 32, kernel 3, stride 2, padding 1, ReLU                 (128 -> 64)
    conv3  32 -> 32, kernel 3, stride 2, padding 1, ReLU                 (64 -> 32)
    fc1    1024 -> 256 (input index t * 32 + c, position-major), ReLU
    fc2    256 -> 1

    conv: out[t][c] = b[c] + sum_{k < 3} sum_ci W[c][k][ci] in[2t + k - 1][ci]

Parameters form one flat float vector in the order of LAYOUT. Weights are used rounded to BF16
(round to nearest even) with accumulation in FP64 here; ``act_bf16`` also rounds the inputs of
the conv layers and of fc1 to BF16 (the tensor-core inference path feeds them to the tensor cores
in BF16; fc2 takes the fc1 activations in FP32).
"""
from __future__ import annotations

import numpy as np

L_IN, C_IN, CH, KS, HID = 256, 2, 32, 3, 256
LAYOUT = [("W1", (CH, KS, C_IN)), ("b1", (CH,)), ("W2", (CH, KS, CH)), ("b2", (CH,)), ("W3", (CH, KS, CH)),
          ("b3", (CH,)), ("W4", (HID, CH * (L_IN // 8))), ("b4", (HID,)), ("W5", (HID,)), ("b5", (1,))]
WEIGHTS = ("W1", "W2", "W3", "W4", "W5")


def n_params() -> int:
    return int(sum(np.prod(s) for _, s in LAYOUT))


def offsets() -> dict:
    out, o = {}, 0
    for name, shape in LAYOUT:
        n = int(np.prod(shape))
        out[name] = (o, shape)
        o += n
    return out


def unflatten(theta) -> dict:
    theta = np.asarray(theta, np.float64)
    return {name: theta[o:o + int(np.prod(s))].reshape(s) for name, (o, s) in offsets().items()}


def bf16_round(a) -> np.ndarray:
    """Round float32 values to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    return np.where(np.isnan(f), np.nan, out)


def init_params(seed: int) -> np.ndarray:
    """He-uniform weights, zero biases (float32 values)."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(n_params(), np.float32)
    for name, (o, shape) in offsets().items():
        n = int(np.prod(shape))
        if name.startswith("W"):
            fan_in = int(np.prod(shape[1:])) if len(shape) > 1 else shape[0]
            lim = np.sqrt(6.0 / fan_in)
            theta[o:o + n] = rng.uniform(-lim, lim, n)
    return theta


# ---- profile -------------------------------------------------------------------------------------

def profile_2d(grid, pose, u, L: int = L_IN, max_range: float = 0.0) -> np.ndarray:
    """Samples of one beam: sample i is the cell holding o + (i + 1/2) d (d the Q30 beam
    direction), i.e. the floor of the Q31 position (o << 15) + (2i + 1) d; x[i] = (o, 1) inside the
    map, (0, 0) outside, and (0, 0) too when the sample lies at or beyond max_range (i + 1/2 >=
    max_range, max_range > 0): a beam cut at range R sees the cells of a map that ends at R. Exact
    integer arithmetic."""
    H, W = grid.shape
    c, s = int(pose[2]), int(pose[3])
    ux, uy = int(u[0]), int(u[1])
    dx = (c * ux - s * uy + (1 << 29)) >> 30
    dy = (s * ux + c * uy + (1 << 29)) >> 30
    x = np.zeros((L, 2), np.float64)
    for i in range(L):
        if max_range > 0 and i + 0.5 >= max_range:
            continue
        px = ((int(pose[0]) << 15) + (2 * i + 1) * dx) >> 31
        py = ((int(pose[1]) << 15) + (2 * i + 1) * dy) >> 31
        if 0 <= px < W and 0 <= py < H:
            x[i, 0] = float(grid[py, px])
            x[i, 1] = 1.0
    return x


def profiles_2d(grid, poses, dirs, L: int = L_IN, max_range: float = 0.0) -> np.ndarray:
    out = np.zeros((poses.shape[0] * dirs.shape[0], L, 2))
    for p in range(poses.shape[0]):
        for b in range(dirs.shape[0]):
            out[p * dirs.shape[0] + b] = profile_2d(grid, poses[p], dirs[b], L, max_range)
    return out


# ---- forward / backward --------------------------------------------------------------------------

def conv(x, W, b):
    """x [N][Lin][Cin], W [Cout][3][Cin], b [Cout] -> [N][Lin/2][Cout] (stride 2, zero pad 1)."""
    N, Lin, Cin = x.shape
    Lout = Lin // 2
    xp = np.zeros((N, Lin + 2, Cin))
    xp[:, 1:Lin + 1] = x
    out = np.broadcast_to(b, (N, Lout, W.shape[0])).copy()
    for k in range(KS):
        # input position 2t + k - 1 = padded index 2t + k
        out += np.einsum("ntc,oc->nto", xp[:, k:k + 2 * Lout:2], W[:, k, :])
    return out


def conv_backward(x, W, dout):
    """Gradients of conv(): (dx, dW, db)."""
    N, Lin, Cin = x.shape
    Lout = Lin // 2
    xp = np.zeros((N, Lin + 2, Cin))
    xp[:, 1:Lin + 1] = x
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for k in range(KS):
        dW[:, k, :] = np.einsum("nto,ntc->oc", dout, xp[:, k:k + 2 * Lout:2])
        dxp[:, k:k + 2 * Lout:2] += np.einsum("nto,oc->ntc", dout, W[:, k, :])
    return dxp[:, 1:Lin + 1], dW, dout.sum(axis=(0, 1))


def weights_bf16(theta) -> dict:
    p = unflatten(np.asarray(theta, np.float32).astype(np.float64))
    for w in WEIGHTS:
        p[w] = bf16_round(p[w])
    return p


def forward(theta, x, act_bf16: bool = False, bf16_weights: bool = True):
    """Predictions [N] and the cache for backward(). x [N][256][2]. bf16_weights=False uses the
    parameters as given (FP64), for differentiating numerically."""
    p = weights_bf16(theta) if bf16_weights else unflatten(theta)
    rnd = bf16_round if act_bf16 else (lambda a: np.asarray(a, np.float64))
    a0 = rnd(x)
    z1 = conv(a0, p["W1"], p["b1"])
    a1 = rnd(np.maximum(z1, 0.0))
    z2 = conv(a1, p["W2"], p["b2"])
    a2 = rnd(np.maximum(z2, 0.0))
    z3 = conv(a2, p["W3"], p["b3"])
    a3 = rnd(np.maximum(z3, 0.0))
    h0 = a3.reshape(a3.shape[0], -1)  # index t * 32 + c
    z4 = h0 @ p["W4"].T + p["b4"]
    a4 = np.maximum(z4, 0.0)  # fc2 reads the fc1 activations in FP32 in both modes
    pred = a4 @ p["W5"] + p["b5"][0]
    return pred, dict(p=p, a0=a0, z1=z1, a1=a1, z2=z2, a2=a2, z3=z3, a3=a3, h0=h0, z4=z4, a4=a4)


def mse(pred, y):
    """Loss mean((pred - y)^2) and its gradient with respect to pred."""
    d = np.asarray(pred, np.float64) - np.asarray(y, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(cache, dpred) -> np.ndarray:
    """Gradient of sum(dpred * pred) with respect to the flat parameters (through the BF16-rounded
    weights, i.e. straight through the rounding)."""
    p = cache["p"]
    g = {}
    g["W5"] = cache["a4"].T @ dpred
    g["b5"] = np.array([dpred.sum()])
    dz4 = np.outer(dpred, p["W5"]) * (cache["z4"] > 0)
    g["W4"] = dz4.T @ cache["h0"]
    g["b4"] = dz4.sum(axis=0)
    dz3 = (dz4 @ p["W4"]).reshape(cache["a3"].shape) * (cache["z3"] > 0)
    da2, g["W3"], g["b3"] = conv_backward(cache["a2"], p["W3"], dz3)
    dz2 = da2 * (cache["z2"] > 0)
    da1, g["W2"], g["b2"] = conv_backward(cache["a1"], p["W2"], dz2)
    dz1 = da1 * (cache["z1"] > 0)
    _, g["W1"], g["b1"] = conv_backward(cache["a0"], p["W1"], dz1)
    return np.concatenate([g[name].reshape(-1) for name, _ in LAYOUT])


def loss_and_grad(theta, x, y):
    pred, cache = forward(theta, x)
    loss, dpred = mse(pred, y)
    return loss, backward(cache, dpred)


def adam(theta, m, v, g, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam step (Kingma and Ba, Algorithm 1) with bias correction; returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
