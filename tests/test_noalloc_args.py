"""Argument checks of lk_launch_noalloc, through the C ABI itself (the Python
binding's own size checks are bypassed).  Every case here is refused before
any CUDA call, so these run without a GPU: the checks are lk_submit's
(shared code), plus the entry point's own CTA and thread limits."""
import ctypes

import pytest

from paper_2310_01212_gb300 import lk

A, B, O = 0x10000, 0x20000, 0x30000   # 16-byte aligned stand-ins; never dereferenced


def call(op, n, ins, out, ctas=4, threads=256, flags=0, device=0, desc=True):
    lib = lk.load()
    d = lk.lk_desc(op, flags, n, 0)
    arr = (ctypes.c_void_p * max(1, len(ins)))(*ins) if ins else None
    return lib.lk_launch_noalloc(device, ctypes.byref(d) if desc else None, arr, len(ins), out, ctas, threads, None)


@pytest.fixture(scope="module", autouse=True)
def _built(native_built):
    return native_built


@pytest.mark.parametrize("op", [lk.LK_OP_COMBINE_SUM, lk.LK_OP_COMBINE_HIST])
def test_combine_needs_an_output_even_when_empty(op):
    # the combine bodies store to out[0] (out[0..255]) whatever n is
    assert call(op, 0, [None], None) == lk.LK_EINVAL
    assert call(op, 3, [A], None) == lk.LK_EINVAL


@pytest.mark.parametrize("op", [lk.LK_OP_COMBINE_SUM, lk.LK_OP_COMBINE_HIST])
def test_combine_length_cap(op):
    assert call(op, (1 << 20) + 1, [A], O) == lk.LK_EINVAL


def test_spin_length_cap():
    # n dependent steps per thread: 2^32 is the cap, as for lk_submit
    assert call(lk.LK_OP_SPIN, (1 << 32) + 1, [], None) == lk.LK_EINVAL


@pytest.mark.parametrize("op", [lk.LK_OP_BATCH, 10, 99, 2**31])
def test_unknown_op(op):
    assert call(op, 16, [A], O) == lk.LK_EINVAL


def test_sum_and_hist_always_write_out():
    assert call(lk.LK_OP_SUM_F32, 0, [None], None) == lk.LK_EINVAL
    assert call(lk.LK_OP_HIST_U8, 0, [None], None) == lk.LK_EINVAL


def test_size_limits():
    assert call(lk.LK_OP_ADD_I32, (1 << 40) + 1, [A, B], O) == lk.LK_EINVAL
    assert call(lk.LK_OP_HIST_U8, 1 << 31, [A], O) == lk.LK_EINVAL
    assert call(lk.LK_OP_GEMM64_F32, (1 << 28) + 1, [A, B], O) == lk.LK_EINVAL


def test_inputs_alignment_and_count():
    assert call(lk.LK_OP_ADD_I32, 16, [A], O) == lk.LK_EINVAL          # needs two inputs
    assert call(lk.LK_OP_ADD_I32, 16, [A + 4, B], O) == lk.LK_EINVAL   # misaligned
    assert call(lk.LK_OP_ADD_I32, 16, [A, None], O) == lk.LK_EINVAL    # missing
    assert call(lk.LK_OP_COPY_I32, 16, [A], O + 8) == lk.LK_EINVAL     # misaligned out
    assert call(lk.LK_OP_COPY_I32, 16, [A], None) == lk.LK_EINVAL      # missing out
    assert call(lk.LK_OP_COPY_I32, 16, [1 << 49], O) == lk.LK_EINVAL   # above 2^48


def test_flags_descriptor_and_device():
    assert call(lk.LK_OP_SUM_F32, 16, [A], O, flags=1) == lk.LK_EINVAL
    assert call(lk.LK_OP_SUM_F32, 16, [A], O, desc=False) == lk.LK_EINVAL
    assert call(lk.LK_OP_SUM_F32, 16, [A], O, device=-1) == lk.LK_EINVAL
    assert call(lk.LK_OP_SUM_F32, 16, [A], O, device=256) == lk.LK_EINVAL


@pytest.mark.parametrize("ctas", [0, -1, 1025])
def test_cta_limit_of_the_static_array(ctas):
    assert call(lk.LK_OP_SUM_F32, 16, [A], O, ctas=ctas) == lk.LK_EINVAL


@pytest.mark.parametrize("threads", [0, 32, 48, 100, 1056])
def test_thread_limits(threads):
    assert call(lk.LK_OP_SUM_F32, 16, [A], O, threads=threads) == lk.LK_EINVAL
