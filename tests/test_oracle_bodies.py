"""Pins for the oracle's work bodies: closed forms, invariants, and special
cases that reduce to library routines (numpy, math.fsum).  CPU only."""
import math

import numpy as np
import pytest

from paper_2310_01212_gb300 import synth


def test_add_closed_forms(oracle_lib):
    o = oracle_lib
    n = 10007
    a = np.arange(n, dtype=np.int32)
    assert np.all(o.add_i32(a, -a) == 0)
    assert np.all(o.add_i32(a, (n - 1 - a).astype(np.int32)) == n - 1)
    # operand order matters for neither side, but a dropped or shifted operand does
    b = np.arange(n, dtype=np.int32) * 3
    assert np.array_equal(o.add_i32(a, b), (np.arange(n) * 4).astype(np.int32))


def test_add_wraps_mod_2_32(oracle_lib):
    o = oracle_lib
    a = np.array([2**31 - 1, -(2**31), -1, 2**31 - 1], dtype=np.int32)
    b = np.array([1, -1, 1, 2**31 - 1], dtype=np.int32)
    assert o.add_i32(a, b).tolist() == [-(2**31), 2**31 - 1, 0, -2]


def test_add_matches_python_integers_mod_2_32(oracle_lib):
    a = synth.int32_uniform(1, 1, 5000, -(2**31), 2**31 - 1)
    b = synth.int32_uniform(1, 2, 5000, -(2**31), 2**31 - 1)
    got = oracle_lib.add_i32(a, b)
    want = [((int(x) + int(y) + 2**31) % 2**32) - 2**31 for x, y in zip(a, b)]
    assert got.tolist() == want


def test_copy_identity(oracle_lib):
    x = synth.int32_uniform(2, 1, 4099, -(2**31), 2**31 - 1)
    assert np.array_equal(oracle_lib.copy_i32(x), x)
    assert oracle_lib.copy_i32(np.zeros(0, np.int32)).size == 0


def test_hist_closed_forms(oracle_lib):
    o = oracle_lib
    n = 256 * 41
    x = (np.arange(n) % 256).astype(np.uint8)
    assert np.all(o.hist_u8(x) == 41)
    h = o.hist_u8(np.full(1000, 7, np.uint8))
    assert h[7] == 1000 and h.sum() == 1000
    # value v appears v+1 times: an off-by-one bin index cannot pass
    x = np.concatenate([np.full(v + 1, v, np.uint8) for v in range(256)])
    x = x[synth.permutation(3, 1, x.size)]
    assert np.array_equal(o.hist_u8(x), np.arange(1, 257))
    assert np.all(o.hist_u8(np.zeros(0, np.uint8)) == 0)


def test_hist_matches_bincount(oracle_lib):
    x = synth.bytes_uniform(4, 1, (1 << 20) + 13)
    h = oracle_lib.hist_u8(x)
    assert np.array_equal(h, np.bincount(x, minlength=256))
    assert h.sum() == x.size


@pytest.mark.parametrize("n", [0, 1, 7, 8, 9, 1000, 65536, (1 << 20) + 3])
def test_sum_arange_exact(oracle_lib, n):
    x = np.arange(n, dtype=np.float32)   # exact in binary32 below 2^24
    assert oracle_lib.sum_f32(x) == n * (n - 1) / 2


def test_sum_periodic_closed_form(oracle_lib):
    n = 100003
    x = ((np.arange(n) % 7) - 3).astype(np.float32)
    full, rem = divmod(n, 7)
    want = full * 0 + sum(r - 3 for r in range(rem))
    assert oracle_lib.sum_f32(x) == want


def test_sum_within_bound_of_correctly_rounded(oracle_lib):
    x = synth.normal_f32(5, 1, (1 << 20) + 5)
    s = oracle_lib.sum_f32(x)
    exact = math.fsum(float(v) for v in x)
    bound = 21 * 2.0**-53 * float(np.abs(x.astype(np.float64)).sum())
    assert abs(s - exact) <= bound
    assert oracle_lib.abs_sum_f32(x) == pytest.approx(float(np.abs(x.astype(np.float64)).sum()), rel=1e-12)


def test_sum_sign_matters(oracle_lib):
    x = np.array([1.0, -2.0, 3.0, -4.0, 5.0], dtype=np.float32)
    assert oracle_lib.sum_f32(x) == 3.0
    assert oracle_lib.abs_sum_f32(x) == 15.0


def _tiles(t):
    return np.zeros((t, 64, 64), np.float32)


def test_gemm_identity_and_ones(oracle_lib):
    o = oracle_lib
    B = synth.normal_f32(6, 1, 3 * 4096).reshape(3, 64, 64)
    I = np.broadcast_to(np.eye(64, dtype=np.float32), (3, 64, 64)).copy()
    assert np.array_equal(o.gemm64_f32(I, B), B.astype(np.float64))
    ones = np.ones((2, 64, 64), np.float32)
    assert np.all(o.gemm64_f32(ones, ones) == 64.0)


def test_gemm_diag_scales_rows(oracle_lib):
    d = np.arange(1, 65, dtype=np.float32)
    A = np.diag(d)[None].astype(np.float32)
    B = synth.int32_uniform(7, 1, 4096, -50, 50).astype(np.float32).reshape(1, 64, 64)
    assert np.array_equal(oracle_lib.gemm64_f32(A, B)[0], d[:, None].astype(np.float64) * B[0])


def test_gemm_integer_matrices_match_numpy_exactly(oracle_lib):
    # non-symmetric integer tiles: a transposed operand or swapped index fails
    A = synth.int32_uniform(8, 1, 4 * 4096, -100, 100).reshape(4, 64, 64)
    B = synth.int32_uniform(8, 2, 4 * 4096, -100, 100).reshape(4, 64, 64)
    C = oracle_lib.gemm64_f32(A.astype(np.float32), B.astype(np.float32))
    want = np.matmul(A.astype(np.int64), B.astype(np.int64))
    assert np.array_equal(C, want.astype(np.float64))


# ---- the per-element GEMM bound sum_k |a_ik b_kj| -------------------------------------
# Pinned by values the mathematics fixes, not by a second copy of the formula:
# each case below fails a bound that takes |sum_k a b| instead of sum_k |a b|,
# drops the absolute value of one operand, or transposes an operand.

def test_gemm_abs_bound_all_ones_is_64(oracle_lib):
    ones = np.ones((2, 64, 64), np.float32)
    assert np.all(oracle_lib.gemm64_abs_bound(ones, ones) == 64.0)
    # negated operands: the products are all +1 or all -1, the bound stays 64
    assert np.all(oracle_lib.gemm64_abs_bound(-ones, ones) == 64.0)


def test_gemm_abs_bound_identity_is_abs_b(oracle_lib):
    B = synth.normal_f32(9, 2, 3 * 4096).reshape(3, 64, 64)
    I = np.broadcast_to(np.eye(64, dtype=np.float32), (3, 64, 64)).copy()
    assert np.array_equal(oracle_lib.gemm64_abs_bound(I, B), np.abs(B).astype(np.float64))
    # B = I: the bound is |A| (a transposed operand would give |A|^T)
    A = synth.normal_f32(9, 3, 3 * 4096).reshape(3, 64, 64)
    assert np.array_equal(oracle_lib.gemm64_abs_bound(A, I), np.abs(A).astype(np.float64))


def test_gemm_abs_bound_signed_diagonal(oracle_lib):
    # A = diag(d) with signs: bound[i][j] = |d_i| |b_ij| exactly (one product per sum)
    d = synth.normal_f32(9, 4, 64)
    A = np.diag(d)[None].astype(np.float32)
    B = synth.normal_f32(9, 5, 4096).reshape(1, 64, 64)
    want = np.abs(d.astype(np.float64))[:, None] * np.abs(B[0].astype(np.float64))
    assert np.array_equal(oracle_lib.gemm64_abs_bound(A, B)[0], want)


def test_gemm_abs_bound_signed_integers_exact(oracle_lib):
    # signed integer tiles: sum_k |a||b| is an exact integer, computed in int64;
    # |sum_k a b| (an easy slip) differs from it almost everywhere
    A = synth.int32_uniform(9, 6, 4 * 4096, -1000, 1000).reshape(4, 64, 64)
    B = synth.int32_uniform(9, 7, 4 * 4096, -1000, 1000).reshape(4, 64, 64)
    want = np.matmul(np.abs(A.astype(np.int64)), np.abs(B.astype(np.int64)))
    got = oracle_lib.gemm64_abs_bound(A.astype(np.float32), B.astype(np.float32))
    assert np.array_equal(got, want.astype(np.float64))
    signed = np.abs(np.matmul(A.astype(np.int64), B.astype(np.int64)))
    assert np.count_nonzero(signed != want) > 0.99 * want.size


def test_gemm_abs_bound_cancelling_row(oracle_lib):
    # row 0 of A = (1, -1, 0, ...), B all ones: C[0][j] = 0, bound[0][j] = 2
    A = np.zeros((1, 64, 64), np.float32)
    A[0, 0, 0], A[0, 0, 1] = 1.0, -1.0
    B = np.ones((1, 64, 64), np.float32)
    assert np.all(oracle_lib.gemm64_f32(A, B)[0, 0] == 0.0)
    assert np.all(oracle_lib.gemm64_abs_bound(A, B)[0, 0] == 2.0)
    assert np.all(oracle_lib.gemm64_abs_bound(A, B)[0, 1:] == 0.0)


def test_gemm_abs_bound_dominates_the_product(oracle_lib):
    A = synth.normal_f32(9, 1, 4096).reshape(1, 64, 64)
    B = synth.normal_f32(9, 2, 4096).reshape(1, 64, 64)
    assert np.all(oracle_lib.gemm64_abs_bound(A, B) >= np.abs(oracle_lib.gemm64_f32(A, B)))


# ---- the compute-bound loop (Sec. III) ----------------------------------------------
@pytest.mark.parametrize("x0", [0, 1, 12345, 2**31 + 7, 2**32 - 1])
@pytest.mark.parametrize("iters", [0, 1, 2, 3, 17, 1000, 20000, 65537])
def test_lcg_jump_ahead_equals_the_loop(oracle_lib, x0, iters):
    assert oracle_lib.lcg_jump(x0, iters) == oracle_lib.lcg_brute(x0, iters)


def test_lcg_matches_python_integers(oracle_lib):
    x = 99
    for _ in range(50):
        x = (1664525 * x + 1013904223) % 2**32
    assert oracle_lib.lcg_jump(99, 50) == x


def test_lcg_full_period_of_the_map(oracle_lib):
    # Hull-Dobell: c odd and a - 1 divisible by 4 give period 2^32, so the map
    # returns to its start after 2^32 steps and not after 2^31
    assert oracle_lib.lcg_jump(5, 2**32) == 5
    assert oracle_lib.lcg_jump(5, 2**31) != 5


def test_spin_xor_is_xor_of_threads(oracle_lib):
    want = 0
    for t in range(7):
        want ^= oracle_lib.lcg_brute(65536 * 3 + t + 1, 100)
    assert oracle_lib.spin_xor(3, 7, 100) == want
