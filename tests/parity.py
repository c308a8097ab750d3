"""Parity tolerance for FP32 GPU results against the FP64 oracle.

Per-beam mutual information: |gpu - oracle| <= REL * |oracle| + ABS, with REL = 1e-4 (the
required per-beam relative error) and ABS = 1e-7 nats as an absolute floor for beams whose MI is
at the level of FP32 rounding of their own terms (e.g. nearly known maps).
Integer work (cell lists, run decompositions) is compared bit for bit.
"""
import numpy as np

REL = 1e-4
ABS = 1e-7


def assert_mi_close(gpu, ref, what=""):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    assert np.all(np.isfinite(gpu)), f"{what}: non-finite GPU values"
    err = np.abs(gpu - ref)
    bad = err > REL * np.abs(ref) + ABS
    if bad.any():
        i = np.flatnonzero(bad.reshape(-1))[:5]
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} beams out of tolerance; "
                             f"first: gpu={gpu.reshape(-1)[i]}, oracle={ref.reshape(-1)[i]}")
    rel = err / np.maximum(np.abs(ref), 1e-30)
    return float(rel.max()), float(np.median(rel))
