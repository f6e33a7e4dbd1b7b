"""GPU parity of batches (lk_submit_batch): every item of a batch against the
oracle, split and unsplit, mixed with single descriptors; a sum split into
p parts is bit-identical to the same sum on a cluster of p CTAs; the CUDA
graph baseline computes the same outputs."""
import numpy as np
import pytest

from gpu_util import gemm_ok, host, need_gpu, sum_ok, to_dev
from paper_2310_01212_gb300 import lk, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_ready(native_built):
    return need_gpu()


def _make(torch, seed, sizes_ops):
    """items with host copies of their inputs; outputs zeroed on the device."""
    rows, refs = [], []
    for i, (op, n, parts) in enumerate(sizes_ops):
        if op == lk.LK_OP_ADD_I32:
            a = synth.int32_uniform(seed, 2 * i, n, -(1 << 20), 1 << 20)
            b = synth.int32_uniform(seed, 2 * i + 1, n, -(1 << 20), 1 << 20)
            out = torch.zeros(max(n, 4), dtype=torch.int32, device="cuda")
            rows.append((op, n, (to_dev(a), to_dev(b)), out, parts))
            refs.append((a, b))
        elif op == lk.LK_OP_COPY_I32:
            a = synth.int32_uniform(seed, 2 * i, n, -(2**31), 2**31 - 1)
            out = torch.zeros(max(n, 4), dtype=torch.int32, device="cuda")
            rows.append((op, n, (to_dev(a),), out, parts))
            refs.append((a,))
        elif op == lk.LK_OP_SUM_F32:
            x = synth.normal_f32(seed, 2 * i, n)
            out = torch.full((4,), 7.0, device="cuda")
            rows.append((op, n, (to_dev(x) if n else torch.zeros(4, device="cuda"),), out, parts))
            refs.append((x,))
        elif op == lk.LK_OP_HIST_U8:
            x = synth.bytes_uniform(seed, 2 * i, n)
            out = torch.full((256,), -1, dtype=torch.int32, device="cuda")
            rows.append((op, n, (to_dev(x) if n else torch.zeros(16, dtype=torch.uint8, device="cuda"),), out, parts))
            refs.append((x,))
        else:
            A = synth.normal_f32(seed, 2 * i, n * 4096).reshape(n, 64, 64)
            B = synth.normal_f32(seed, 2 * i + 1, n * 4096).reshape(n, 64, 64)
            out = torch.zeros((n, 64, 64), device="cuda")
            rows.append((op, n, (to_dev(A), to_dev(B)), out, parts))
            refs.append((A, B))
    return rows, refs


def _check(oracle, rows, refs):
    for (op, n, ins, out, parts), ref in zip(rows, refs):
        got = host(out)
        if op == lk.LK_OP_ADD_I32:
            assert np.array_equal(got[:n], oracle.add_i32(*ref)), (op, n, parts)
        elif op == lk.LK_OP_COPY_I32:
            assert np.array_equal(got[:n], ref[0]), (op, n, parts)
        elif op == lk.LK_OP_SUM_F32:
            assert sum_ok(got[0], ref[0], oracle), (n, parts, got[0], oracle.sum_f32(ref[0]))
        elif op == lk.LK_OP_HIST_U8:
            assert np.array_equal(got.astype(np.int64), oracle.hist_u8(ref[0])), (n, parts)
        else:
            assert gemm_ok(got, *ref, oracle), (n, parts)


MIX = [(lk.LK_OP_ADD_I32, 1000, 0), (lk.LK_OP_ADD_I32, 3_000_001, 0), (lk.LK_OP_ADD_I32, 65536, 5),
       (lk.LK_OP_SUM_F32, 1027, 0), (lk.LK_OP_SUM_F32, 2_000_003, 0), (lk.LK_OP_SUM_F32, 262144, 8),
       (lk.LK_OP_SUM_F32, 0, 0), (lk.LK_OP_HIST_U8, 1 << 20, 0), (lk.LK_OP_HIST_U8, (1 << 22) + 7, 4),
       (lk.LK_OP_HIST_U8, 100, 3), (lk.LK_OP_COPY_I32, 777_777, 0), (lk.LK_OP_COPY_I32, 5, 2),
       (lk.LK_OP_GEMM64_F32, 1, 0), (lk.LK_OP_GEMM64_F32, 3, 8), (lk.LK_OP_GEMM64_F32, 40, 2), (lk.LK_OP_NOP, 0, 1)]


@pytest.mark.parametrize("part_bytes", [1 << 20, 16 << 20])
def test_batch_items_match_oracle(torch_ready, oracle_lib, part_bytes):
    torch = torch_ready
    rows, refs = _make(torch, 41, MIX)
    items = lk.batch_items(rows)
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([37], idle_lease_ns=5_000_000_000, exec_log_cap=64) as c:
        h = lk.lk_submit_batch(c, 0, items, part_bytes=part_bytes)
        assert lk.lk_wait(c, h) == lk.LK_OK
        log, _ = lk.lk_exec_log(c)
        assert len(log) == 37 and set(log["op"].tolist()) == {lk.LK_OP_BATCH}
    _check(oracle_lib, rows, refs)


def test_batches_mixed_with_single_descriptors(torch_ready, oracle_lib):
    torch = torch_ready
    rows1, refs1 = _make(torch, 42, MIX[:8])
    rows2, refs2 = _make(torch, 43, MIX[8:])
    x = synth.normal_f32(44, 1, 100_003)
    dx = to_dev(x)
    outs = [torch.zeros(4, device="cuda") for _ in range(3)]
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([16, 16], idle_lease_ns=5_000_000_000) as c:
        hs = [lk.lk_submit(c, 0, lk.LK_OP_SUM_F32, x.size, (dx,), outs[0]),
              lk.lk_submit_batch(c, 0, lk.batch_items(rows1)),
              lk.lk_submit(c, 0, lk.LK_OP_SUM_F32, x.size, (dx,), outs[1]),
              lk.lk_submit_batch(c, 0, lk.batch_items(rows2)),
              lk.lk_submit_batch(c, 1, lk.batch_items([])),
              lk.lk_submit(c, 0, lk.LK_OP_SUM_F32, x.size, (dx,), outs[2])]
        for h in hs:
            assert h is not None and lk.lk_wait(c, h) == lk.LK_OK
    _check(oracle_lib, rows1, refs1)
    _check(oracle_lib, rows2, refs2)
    v = [host(o)[0] for o in outs]
    assert v[0] == v[1] == v[2] and sum_ok(v[0], x, oracle_lib)


@pytest.mark.parametrize("p", [1, 3, 8])
def test_split_sum_equals_cluster_of_that_size(torch_ready, p):
    torch = torch_ready
    x = synth.normal_f32(45, p, 1_000_003)
    dx = to_dev(x)
    ob, oc = torch.zeros(4, device="cuda"), torch.zeros(4, device="cuda")
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([8], idle_lease_ns=5_000_000_000) as c:
        assert lk.lk_wait(c, lk.lk_submit_batch(c, 0, lk.batch_items([(lk.LK_OP_SUM_F32, x.size, (dx,), ob, p)]))) == 0
    with lk.lk_init([p], idle_lease_ns=5_000_000_000) as c:
        assert lk.lk_wait(c, lk.lk_submit(c, 0, lk.LK_OP_SUM_F32, x.size, (dx,), oc)) == lk.LK_OK
    assert host(ob)[0] == host(oc)[0]


def test_many_batches_back_to_back(torch_ready, oracle_lib):
    torch = torch_ready
    rows, refs = _make(torch, 46, [(lk.LK_OP_ADD_I32, 4096 + i, 0) for i in range(64)])
    items = lk.batch_items(rows)
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([37], idle_lease_ns=5_000_000_000) as c:
        hs = []
        for _ in range(40):
            while True:
                h = lk.lk_submit_batch(c, 0, items)
                if h is not None:
                    break
            hs.append(h)
        for h in hs:
            assert lk.lk_wait(c, h) == lk.LK_OK
    _check(oracle_lib, rows, refs)


def test_graph_baseline_same_outputs(torch_ready, oracle_lib):
    torch = torch_ready
    rows, refs = _make(torch, 47, MIX)
    items = lk.batch_items(rows)
    torch.cuda.current_stream().synchronize()
    ms = lk.lk_baseline_graph(items, max_ctas=148, threads=256, reps=2)
    assert ms.size == 2 and np.all(ms > 0)
    _check(oracle_lib, rows, refs)
