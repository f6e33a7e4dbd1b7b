"""The error bound behind the GEMM tile's tensor-core path, checked on the
CPU: a float32 x split as x_hi = bf16(x), x_lo = bf16(x - x_hi), both rounded
to nearest even, represents x to within 2^-17 |x|, x - x_hi is exact in
float32, and the four products of two split operands form a b to within
2^-15 |a b| -- inside the 1e-4 sum_k |a b| bound of the GEMM body with room
for the float32 accumulation.  (The GPU tests check the kernel itself against
the oracle.)"""
import numpy as np


def bf16_rne(x: np.ndarray) -> np.ndarray:
    """float32 -> nearest bf16 (ties to even), returned as float32."""
    u = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def test_two_part_bf16_split_bounds():
    rng = np.random.default_rng(2310)
    n = 1 << 20
    x = (rng.standard_normal(n) * 2.0 ** rng.integers(-30, 30, n)).astype(np.float32)
    hi = bf16_rne(x)
    r = (x - hi).astype(np.float32)
    assert np.array_equal(r.astype(np.float64), x.astype(np.float64) - hi.astype(np.float64))   # exact
    lo = bf16_rne(r)
    x64 = x.astype(np.float64)
    rep = np.abs(hi.astype(np.float64) + lo.astype(np.float64) - x64)
    assert np.all(rep <= 2.0 ** -17 * np.abs(x64))
    a, b = x64[: n // 2], x64[n // 2:]
    ah, al, bh, bl = (v.astype(np.float64) for v in (hi[: n // 2], lo[: n // 2], hi[n // 2:], lo[n // 2:]))
    prod = ah * bh + ah * bl + al * bh + al * bl        # each bf16 x bf16 product is exact in float32
    assert np.all(np.abs(prod - a * b) <= 2.0 ** -15 * np.abs(a * b))
    # a single bf16 product per pair would miss the GEMM bound
    assert np.max(np.abs(ah * bh - a * b) / np.abs(a * b)) > 1e-4
