"""The full-chip mixed workload (4 clusters x 37 SMs, the four bodies in
equal shuffled shares, Poisson arrivals at 20,000/s): one whole step of
10,000 items, every item's output checked against the oracle, and the
persistent kernel's execution log against the oracle checker."""
import numpy as np
import pytest

from gpu_util import need_gpu
from paper_2310_01212_gb300 import lk, workloads as wl

pytestmark = pytest.mark.gpu


def test_every_item_of_a_full_chip_step(native_built, oracle_lib):
    torch = need_gpu()
    import oracle

    cfg = wl.FULL_CHIP
    pools = wl.Pools.create(cfg["seed"])
    items = 10_000
    it, meta = wl.full_chip_trace(pools, cfg["seed"], 0, items, cfg)
    # one output slot per item of each op: nothing is overwritten in the step
    for op in wl.OPS4:
        assert np.sum(meta["op"] == op) <= pools.slots
    torch.cuda.synchronize()
    sizes = cfg["sizes"]
    with lk.lk_init(sizes, threads_per_cta=cfg["threads"], exec_log_cap=items, idle_lease_ns=5_000_000_000) as c:
        rc, res = lk.lk_run_trace(c, it, n_threads=len(sizes))
        assert rc == lk.LK_OK and np.all(res["status"] == lk.LK_OK)
        log, dropped = lk.lk_exec_log(c)
        pinned = sum((lk.lk_cluster_info(c, k) for k in range(len(sizes))), [])
    assert dropped == 0
    order = np.arange(items)
    n_posted = [int(np.sum(order % len(sizes) == k)) for k in range(len(sizes))]
    posted_op = np.concatenate([meta["op"][order % len(sizes) == k] for k in range(len(sizes))])
    verdict = oracle.check_exec_log(log["seq"], log["cluster"], log["rank"], log["smid"], log["op"], log["order"],
                                    sizes, n_posted, pinned_smid=pinned, posted_op=posted_op)
    assert verdict["violations"] == 0, verdict

    i32, u8, f32 = pools.i32.cpu().numpy(), pools.u8.cpu().numpy(), pools.f32.cpu().numpy()
    out_add, out_hist = pools.out_add.cpu().numpy(), pools.out_hist.cpu().numpy()
    out_sum, out_gemm = pools.out_sum.cpu().numpy(), pools.out_gemm.cpu().numpy()
    bad = {op: 0 for op in wl.OPS4}
    for i in range(items):
        op, n, s = int(meta["op"][i]), int(meta["n"][i]), int(meta["slot"][i])
        o0, o1 = int(meta["off0"][i]), int(meta["off1"][i])
        if op == lk.LK_OP_ADD_I32:
            ok = np.array_equal(out_add[s, :n], oracle.add_i32(i32[o0:o0 + n], i32[o1:o1 + n]))
        elif op == lk.LK_OP_HIST_U8:
            ok = np.array_equal(out_hist[s].astype(np.int64), oracle.hist_u8(u8[o0:o0 + n]))
        elif op == lk.LK_OP_SUM_F32:
            x = f32[o0:o0 + n]
            ok = abs(float(out_sum[s, 0]) - oracle.sum_f32(x)) <= 1e-4 * oracle.abs_sum_f32(x)
        else:
            A = f32[o0:o0 + 4096 * n].reshape(n, 64, 64)
            B = f32[o1:o1 + 4096 * n].reshape(n, 64, 64)
            got = out_gemm[s].reshape(n, 64, 64).astype(np.float64)
            ok = bool(np.all(np.abs(got - oracle.gemm64_f32(A, B)) <= 1e-4 * oracle.gemm64_abs_bound(A, B)))
        bad[op] += 0 if ok else 1
    assert sum(bad.values()) == 0, bad
