"""The fused 3D kernel (csrc/evalrle.cuh sample_encode_ray) splits runs every `cap` cells with a
remainder taken from a rounded FP32 quotient: rel - rint(float(rel) * (1.0f / cap)) * cap == 0
stands for rel % cap == 0. Checked here exhaustively in IEEE FP32 (correctly rounded division and
product, round-half-even conversion, as the kernel's 1.0f / cap, FP32 multiply and
__float2int_rn) for every cap the ABI accepts (1..255) and every rel below 2^20 (a ray has at
most 1024 virtual cells)."""
import numpy as np


def test_rounded_quotient_gives_the_remainder_test():
    rel = np.arange(1 << 20, dtype=np.int64)
    relf = rel.astype(np.float32)
    for cap in range(1, 256):
        inv = np.float32(1.0) / np.float32(cap)
        q = np.rint(relf * inv).astype(np.int64)  # float32 product, rounded half to even
        np.testing.assert_array_equal(rel - q * cap == 0, rel % cap == 0, err_msg=f"cap {cap}")
