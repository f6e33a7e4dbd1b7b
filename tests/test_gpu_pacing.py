"""Load-rate caps (lk_set_rate, lk_desc.aux) on the GPU: paced bodies give
the oracle's results and take at least the time their input bytes need at
the cap; unpaced ones are unaffected."""
import time

import numpy as np
import pytest

from gpu_util import gemm_ok, host, need_gpu, sum_ok, to_dev
from paper_2310_01212_gb300 import lk, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_ready(native_built):
    return need_gpu()


def submit(c, *args, **kw):
    """lk_submit that names the device-side reason when the context stopped."""
    try:
        return lk.lk_submit(c, *args, **kw)
    except lk.LkError as e:
        raise AssertionError(f"{e}: device error {lk.lk_device_error(c)}, status {lk.lk_status(c, 0)}") from e


def timed_wait(c, h):
    t0 = time.perf_counter()
    assert lk.lk_wait(c, h, timeout_ns=30_000_000_000) == lk.LK_OK
    return time.perf_counter() - t0


def test_paced_copy_takes_the_paced_time(torch_ready, oracle_lib):
    torch = torch_ready
    n = 1 << 26                                    # 256 MiB of int32 loaded
    a = torch.randint(-1000, 1000, (n,), dtype=torch.int32, device="cuda",
                      generator=torch.Generator(device="cuda").manual_seed(5))
    # every output exists before the context starts: an allocation while the
    # persistent kernel runs may wait for the whole device
    outs = [torch.zeros_like(a) for _ in range(3)]
    torch.cuda.current_stream().synchronize()
    rate = 50_000                                  # bytes/us over the cluster = 50 GB/s
    with lk.lk_init([16], idle_lease_ns=5_000_000_000) as c:
        fast = timed_wait(c, submit(c, 0, lk.LK_OP_COPY_I32, n, (a,), outs[0]))
        lk.lk_set_rate(c, 0, rate)
        paced = timed_wait(c, submit(c, 0, lk.LK_OP_COPY_I32, n, (a,), outs[1]))
        # a per-descriptor cap overrides the cluster's default
        lk.lk_set_rate(c, 0, 0)
        paced2 = timed_wait(c, submit(c, 0, lk.LK_OP_COPY_I32, n, (a,), outs[2], aux=2 * rate))
    for o in outs:
        assert torch.equal(o, a)
    want = 4.0 * n / (rate * 1e6)                  # seconds at the cap
    burst = 16 * 4 * 32768 / (rate * 1e6)          # the bucket: 4 stages per CTA
    print(f"\ncopy 256 MiB: unpaced {fast * 1e3:.2f} ms, paced {paced * 1e3:.2f} ms (cap {want * 1e3:.2f} ms), "
          f"per-descriptor x2 {paced2 * 1e3:.2f} ms")
    assert paced >= want - burst - 1e-4 and paced < 2.0 * want
    assert paced2 >= want / 2 - burst - 1e-4 and paced2 < paced
    assert fast < want / 4


def test_paced_histogram_takes_the_paced_time(torch_ready, oracle_lib):
    """Large histogram shares stream through one ring per warp; the cap is
    split evenly over the warps and still bounds the whole CTA's loads."""
    torch = torch_ready
    n = 1 << 26                                    # 64 MiB of bytes: 4 MiB per CTA
    hb = synth.bytes_uniform(33, 0, n)
    dh = to_dev(hb)
    outs = [torch.zeros(256, dtype=torch.int32, device="cuda") for _ in range(2)]
    torch.cuda.current_stream().synchronize()
    rate = 20_000                                  # bytes/us over the cluster = 20 GB/s
    with lk.lk_init([16], idle_lease_ns=5_000_000_000) as c:
        fast = timed_wait(c, submit(c, 0, lk.LK_OP_HIST_U8, n, (dh,), outs[0]))
        paced = timed_wait(c, submit(c, 0, lk.LK_OP_HIST_U8, n, (dh,), outs[1], aux=rate))
    want = n / (rate * 1e6)
    burst = 16 * 4 * 32768 / (rate * 1e6)          # the buckets: each warp's four stages
    print(f"\nhistogram 64 MiB: unpaced {fast * 1e3:.2f} ms, paced {paced * 1e3:.2f} ms (cap {want * 1e3:.2f} ms)")
    for o in outs:
        assert np.array_equal(host(o).astype(np.int64), oracle_lib.hist_u8(hb))
    assert paced >= want - burst - 1e-4 and paced < 2.0 * want
    assert fast < want / 4


def test_paced_bodies_match_oracle(torch_ready, oracle_lib):
    torch = torch_ready
    n = (1 << 20) + 13
    x = synth.normal_f32(31, 1, n)
    a = synth.int32_uniform(31, 2, n, -(2**31), 2**31 - 1)
    b = synth.int32_uniform(31, 3, n, -(2**31), 2**31 - 1)
    hb = synth.bytes_uniform(31, 4, 3 * n)
    t = 37
    A = synth.normal_f32(31, 5, t * 4096).reshape(t, 64, 64)
    B = synth.normal_f32(31, 6, t * 4096).reshape(t, 64, 64)
    dx, da, db, dh, dA, dB = map(to_dev, (x, a, b, hb, A, B))
    o_sum = torch.zeros(4, device="cuda")
    o_add = torch.zeros(n, dtype=torch.int32, device="cuda")
    o_hist = torch.zeros(256, dtype=torch.int32, device="cuda")
    o_gemm = torch.zeros((t, 64, 64), device="cuda")
    torch.cuda.current_stream().synchronize()
    for per_sm in (1, 2):
        with lk.lk_init([8], idle_lease_ns=5_000_000_000, ctas_per_sm=per_sm) as c:
            lk.lk_set_rate(c, 0, 20_000)
            hs = [lk.lk_submit(c, 0, lk.LK_OP_SUM_F32, n, (dx,), o_sum),
                  lk.lk_submit(c, 0, lk.LK_OP_ADD_I32, n, (da, db), o_add),
                  lk.lk_submit(c, 0, lk.LK_OP_HIST_U8, hb.size, (dh,), o_hist),
                  lk.lk_submit(c, 0, lk.LK_OP_GEMM64_F32, t, (dA, dB), o_gemm)]
            for h in hs:
                assert lk.lk_wait(c, h, timeout_ns=30_000_000_000) == lk.LK_OK
        assert sum_ok(float(host(o_sum)[0]), x, oracle_lib)
        assert np.array_equal(host(o_add), oracle_lib.add_i32(a, b))
        assert np.array_equal(host(o_hist).astype(np.int64), oracle_lib.hist_u8(hb))
        assert gemm_ok(host(o_gemm), A, B, oracle_lib)


def test_paced_batch(torch_ready, oracle_lib):
    torch = torch_ready
    n = 1 << 22
    xs = [synth.normal_f32(32, i, n) for i in range(4)]
    dxs = [to_dev(x) for x in xs]
    outs = torch.zeros((4, 4), device="cuda")
    torch.cuda.current_stream().synchronize()
    items = np.zeros(4, dtype=lk.BATCH_ITEM_DTYPE)
    items["op"] = lk.LK_OP_SUM_F32
    items["n"] = n
    items["in0"] = [d.data_ptr() for d in dxs]
    items["out"] = [outs[i].data_ptr() for i in range(4)]
    with lk.lk_init([8], idle_lease_ns=5_000_000_000) as c:
        lk.lk_set_rate(c, 0, 10_000)                    # 64 MiB at 10 GB/s: >= 6.7 ms
        h = lk.lk_submit_batch(c, 0, items)
        dt = timed_wait(c, h)
    got = host(outs)[:, 0]
    for i in range(4):
        assert sum_ok(float(got[i]), xs[i], oracle_lib)
    assert dt >= 4 * 4.0 * n / 10_000e6 * 0.9
