"""The Gaussian-tail constants in csrc/gauss_tail.cuh meet their stated bound when evaluated in
FP32 (emulated here on the CPU): |T - 0.5 erfc(z)| <= 3e-6 T + 5e-8 and <= 2.5e-7 everywhere."""
import os
import re

import numpy as np
from scipy.special import erfc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _constants():
    src = open(os.path.join(ROOT, "paper_1905_02238_gb300", "csrc", "gauss_tail.cuh")).read()
    vals = dict(re.findall(r"constexpr float (kTail\w+) = ([-0-9.e]+)f;", src))
    p = np.float32(float(vals["kTailP"]))
    ncoef = len([k for k in vals if k.startswith("kTailC")])
    coef = [np.float32(float(vals[f"kTailC{i}"])) for i in range(ncoef)]
    return p, coef


def test_tail_constants_fp32_error():
    p, coef = _constants()
    k = np.sqrt(np.log2(np.e))
    s = np.concatenate([np.linspace(0, 8, 800001), np.linspace(8, 200, 20001)]).astype(np.float32)
    ref = 0.5 * erfc(s.astype(np.float64) / k)
    t = (np.float32(1) / (np.float32(1) + p * s)).astype(np.float32)
    q = coef[-1]
    for c in coef[-2::-1]:
        q = (q * t + c).astype(np.float32)
    e = (2.0 ** (-(s * s).astype(np.float64))).astype(np.float32)
    T = ((e * t).astype(np.float32) * q).astype(np.float32)
    err = np.abs(T.astype(np.float64) - ref)
    assert err.max() <= 2.5e-7
    assert np.all(err <= 3e-6 * ref + 5e-8)
