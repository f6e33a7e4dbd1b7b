"""lk_launch_noalloc: one ordinary launch whose combine scratch is a static
device array, for callers that cannot allocate (a real-time loop that must
not pay an allocator's unbounded latency after start-up, or a thread sharing
the GPU with a running persistent context, where an allocation or free can
block until that kernel returns).

On two calls in a row (the second finds the array exactly as the first left
it) every output is checked against the oracle -- integer bodies bit-exact,
the sum within 1e-4 sum|x| of the binary64 sum, the GEMM per element within
1e-4 sum_k |a b| -- and against the existing allocating entry point,
lk_baseline_run_trace: the same kernel with the same CTAs and threads, so
even the float32 results must be bit-identical (a stale or misordered
partial left in the shared array would show there).  This file is collected
last so that a stop at the first failure has already run every other test.
The argument checks, which need no GPU, are in test_noalloc_args.py."""
import numpy as np
import pytest

from gpu_util import gemm_ok, host, need_gpu, sum_ok, to_dev
from paper_2310_01212_gb300 import lk, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_ready(native_built):
    return need_gpu()


def _cases(torch):
    n = 65536 + 3
    x = synth.normal_f32(31, 1, n)
    hb = synth.bytes_uniform(31, 2, (1 << 20) + 5)
    a = synth.int32_uniform(31, 3, 100003, -(1 << 20), 1 << 20)
    b = synth.int32_uniform(31, 4, 100003, -(1 << 20), 1 << 20)
    A = synth.normal_f32(31, 5, 5 * 4096).reshape(5, 64, 64)
    B = synth.normal_f32(31, 6, 5 * 4096).reshape(5, 64, 64)
    dx, dh, da, db, dA, dB = map(to_dev, (x, hb, a, b, A, B))
    # (op, n, device inputs, host inputs, output maker, kind)
    return [
        (lk.LK_OP_SUM_F32, n, (dx,), (x,), lambda: torch.full((4,), 7.0, device="cuda"), "sum"),
        (lk.LK_OP_HIST_U8, hb.size, (dh,), (hb,), lambda: torch.full((256,), -1, dtype=torch.int32, device="cuda"),
         "hist"),
        (lk.LK_OP_ADD_I32, a.size, (da, db), (a, b), lambda: torch.zeros(a.size, dtype=torch.int32, device="cuda"),
         "add"),
        (lk.LK_OP_GEMM64_F32, 5, (dA, dB), (A, B), lambda: torch.zeros((5, 64, 64), device="cuda"), "gemm"),
    ]


def _oracle_ok(kind, got, hin, oracle):
    if kind == "add":
        return np.array_equal(got, oracle.add_i32(*hin))
    if kind == "hist":
        return np.array_equal(got.astype(np.int64), oracle.hist_u8(*hin))
    if kind == "sum":
        return sum_ok(got[0], hin[0], oracle)
    return gemm_ok(got, hin[0], hin[1], oracle)


@pytest.mark.parametrize("ctas,threads", [(37, 256), (148, 512), (1, 128)])
def test_noalloc_matches_oracle_and_allocating_entry_point(torch_ready, oracle_lib, ctas, threads):
    torch = torch_ready
    cases = _cases(torch)
    # the existing entry point: same kernel, scratch from cudaMalloc
    ref_outs = [c[4]() for c in cases]
    items = np.zeros(len(cases), dtype=lk.TRACE_ITEM_DTYPE)
    for i, (op, n, ins, _, _, _) in enumerate(cases):
        items[i]["op"], items[i]["n"] = op, n
        items[i]["in0"] = ins[0].data_ptr()
        items[i]["in1"] = ins[1].data_ptr() if len(ins) > 1 else 0
        items[i]["out"] = ref_outs[i].data_ptr()
    torch.cuda.current_stream().synchronize()
    rc, _ = lk.lk_baseline_run_trace(items, [ctas], threads=threads, n_threads=1)
    assert rc == lk.LK_OK
    ref = [host(o) for o in ref_outs]
    for (_, _, _, hin, _, kind), r in zip(cases, ref):
        assert _oracle_ok(kind, r, hin, oracle_lib), ("allocating path", kind)

    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):   # two calls in a row share the array
        outs = [c[4]() for c in cases]
        for (op, n, ins, _, _, _), o in zip(cases, outs):
            assert lk.lk_launch_noalloc(op, n, ins, o, ctas=ctas, threads=threads, stream=stream) == lk.LK_OK
        got = [host(o) for o in outs]
        for (_, _, _, hin, _, kind), g, r in zip(cases, got, ref):
            assert _oracle_ok(kind, g, hin, oracle_lib), (call, kind)
            assert np.array_equal(g, r), (call, kind)   # same kernel, same split: bit-identical
