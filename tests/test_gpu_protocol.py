"""GPU parity of the dispatch protocol: the persistent kernel's own execution
log must satisfy the oracle checker (every descriptor exactly once on every
CTA of its cluster, per-cluster FIFO, CTAs pinned to the SMs they booted on,
completion only after every share), and every output must match the oracle."""
import threading
import time

import numpy as np
import pytest

from gpu_util import check_log, host, need_gpu, sum_ok, to_dev
from paper_2310_01212_gb300 import lk, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_ready(native_built):
    return need_gpu()


@pytest.mark.parametrize("flags", [0, lk.LK_INIT_DIRECT, lk.LK_INIT_MAILBOX])
def test_config_small_closed_loop(torch_ready, oracle_lib, flags):
    """4 SMs as 2 clusters of 2, 256 threads; 10,000 closed-loop int32 adds of
    4096 elements, values uniform in [-2^20, 2^20], seed 0, round-robin."""
    torch = torch_ready
    N, n = 10000, 4096
    a = synth.int32_uniform(0, 1, N * n, -(1 << 20), 1 << 20).reshape(N, n)
    b = synth.int32_uniform(0, 2, N * n, -(1 << 20), 1 << 20).reshape(N, n)
    da, db = to_dev(a), to_dev(b)
    out = torch.zeros((N, n), dtype=torch.int32, device="cuda")
    items = np.zeros(N, dtype=lk.TRACE_ITEM_DTYPE)
    items["cluster"] = np.arange(N) % 2
    items["op"] = lk.LK_OP_ADD_I32
    items["n"] = n
    row = n * 4
    items["in0"] = da.data_ptr() + np.arange(N, dtype=np.uint64) * row
    items["in1"] = db.data_ptr() + np.arange(N, dtype=np.uint64) * row
    items["out"] = out.data_ptr() + np.arange(N, dtype=np.uint64) * row
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([2, 2], threads_per_cta=256, exec_log_cap=N, idle_lease_ns=5_000_000_000, flags=flags) as c:
        rc, res = lk.lk_run_trace(c, items, n_threads=1, closed_loop=True)
        assert rc == lk.LK_OK and np.all(res["status"] == lk.LK_OK)
        log, dropped = lk.lk_exec_log(c)
        assert dropped == 0
        verdict, pinned = check_log(oracle_lib, c, log, [2, 2], [N // 2, N // 2],
                                    posted_op=[lk.LK_OP_ADD_I32] * N)
        assert verdict["violations"] == 0, verdict
        assert len(set(pinned)) == 4          # one CTA per SM
    assert np.array_equal(host(out), oracle_lib.add_i32(a, b))
    lat = (res["t_complete_ns"] - res["t_submit_ns"]) / 1000.0
    print(f"\nconfig small closed loop (flags {flags}): p50 {np.percentile(lat, 50):.2f} us  p99 {np.percentile(lat, 99):.2f} us  "
          f"max {lat.max():.2f} us")


def test_smids_recorded_stay_on_boot_sms(torch_ready, oracle_lib):
    with lk.lk_init([37, 37, 37, 37], exec_log_cap=64, idle_lease_ns=5_000_000_000) as c:
        hs = [lk.lk_submit(c, i % 4, lk.LK_OP_NOP, 0) for i in range(200)]
        for h in hs:
            assert lk.lk_wait(c, h) == lk.LK_OK
        log, _ = lk.lk_exec_log(c)
        verdict, pinned = check_log(oracle_lib, c, log, [37] * 4, [50] * 4, posted_op=[0] * 200)
        assert verdict["violations"] == 0, verdict
        assert len(set(pinned)) == 148
        # clusters are contiguous ranges of the sorted SM ids
        flat = [s for cl in range(4) for s in lk.lk_cluster_info(c, cl)]
        assert flat == sorted(flat)


def test_explicit_smid_lists(torch_ready, oracle_lib):
    torch = torch_ready
    props = torch.cuda.get_device_properties(0)
    last = props.multi_processor_count - 1
    lists = [[0, 1, 2], [last, last - 1]]
    with lk.lk_init([3, 2], smids=lists[0] + lists[1], exec_log_cap=64, idle_lease_ns=5_000_000_000) as c:
        assert lk.lk_cluster_info(c, 0) == lists[0]
        assert lk.lk_cluster_info(c, 1) == lists[1]
        hs = [lk.lk_submit(c, i % 2, lk.LK_OP_NOP, 0) for i in range(20)]
        for h in hs:
            assert lk.lk_wait(c, h) == lk.LK_OK
        log, _ = lk.lk_exec_log(c)
        verdict, _ = check_log(oracle_lib, c, log, [3, 2], [10, 10])
        assert verdict["violations"] == 0, verdict
        for r in log:
            assert r["smid"] == lists[r["cluster"]][r["rank"]]


@pytest.mark.parametrize("roles", [False, True], ids=["no_roles", "critical_and_yield"])
@pytest.mark.parametrize("flags", [0, lk.LK_INIT_DIRECT, lk.LK_INIT_MAILBOX])
def test_many_producers_mixed_bodies(torch_ready, oracle_lib, flags, roles):
    torch = torch_ready
    sizes = [8, 8, 8, 8]
    n = 65536
    x = synth.normal_f32(21, 1, n)
    a = synth.int32_uniform(21, 2, n, -(1 << 20), 1 << 20)
    hb = synth.bytes_uniform(21, 3, 1 << 20)
    dx, da, dh = to_dev(x), to_dev(a), to_dev(hb)
    P, J = 4, 200
    outs_sum = torch.zeros((P, J, 4), device="cuda")
    outs_add = torch.zeros((P, J, n), dtype=torch.int32, device="cuda")
    outs_hist = torch.zeros((P, J, 256), dtype=torch.int32, device="cuda")
    torch.cuda.current_stream().synchronize()
    posted = {}
    lock = threading.Lock()
    with lk.lk_init(sizes, exec_log_cap=1024, idle_lease_ns=5_000_000_000, flags=flags) as c:
        if roles:   # the role bits ride on every descriptor; the protocol and results stay the same
            lk.lk_set_role(c, 0, lk.LK_ROLE_CRITICAL)
            for k in (1, 2, 3):
                lk.lk_set_role(c, k, lk.LK_ROLE_YIELD)

        def producer(p):
            for j in range(J):
                cl = (p + j) % 4
                kind = j % 3
                if kind == 0:
                    args = (lk.LK_OP_SUM_F32, n, (dx,), outs_sum[p, j])
                elif kind == 1:
                    args = (lk.LK_OP_ADD_I32, n, (da, da), outs_add[p, j])
                else:
                    args = (lk.LK_OP_HIST_U8, hb.size, (dh,), outs_hist[p, j])
                while True:
                    h = lk.lk_submit(c, cl, *args)
                    if h is not None:
                        break
                with lock:
                    posted[(h >> 48, h & 0xffffffffffff)] = args[0]

        th = [threading.Thread(target=producer, args=(p,)) for p in range(P)]
        [t.start() for t in th]
        [t.join() for t in th]
        assert lk.lk_sync(c) == lk.LK_OK
        log, dropped = lk.lk_exec_log(c)
        n_posted = [sum(1 for (cl, _) in posted if cl == k) for k in range(4)]
        posted_op = [posted[(k, s)] for k in range(4) for s in range(1, n_posted[k] + 1)]
        verdict, _ = check_log(oracle_lib, c, log, sizes, n_posted, posted_op=posted_op)
        assert verdict["violations"] == 0, verdict
    s_out = host(outs_sum)[:, :, 0]
    ref_add = oracle_lib.add_i32(a, a)
    ref_h = oracle_lib.hist_u8(hb)
    add_out, hist_out = host(outs_add), host(outs_hist)
    for p in range(P):
        for j in range(J):
            if j % 3 == 0:
                assert s_out[p, j] == s_out[0, 0]        # same input, same cluster size: same bits
            elif j % 3 == 1:
                assert np.array_equal(add_out[p, j], ref_add)
            else:
                assert np.array_equal(hist_out[p, j].astype(np.int64), ref_h)
    assert sum_ok(s_out[0, 0], x, oracle_lib)


def test_idle_lease_returns_the_kernel(torch_ready):
    c = lk.lk_init([2], idle_lease_ns=200_000_000)
    h = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
    assert lk.lk_wait(c, h) == lk.LK_OK
    time.sleep(1.0)
    assert lk.lk_device_error(c) == lk.LK_DERR_LEASE
    assert lk.lk_status(c, 0) == lk.LK_ST_ERROR
    with pytest.raises(lk.LkError):
        lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
    assert c.dispose() == lk.LK_OK


def test_dispose_drains_queued_work(torch_ready, oracle_lib):
    torch = torch_ready
    n = 1 << 22
    a = synth.int32_uniform(22, 1, n, -5, 5)
    da = to_dev(a)
    outs = [torch.zeros(n, dtype=torch.int32, device="cuda") for _ in range(8)]
    torch.cuda.current_stream().synchronize()
    c = lk.lk_init([4], idle_lease_ns=5_000_000_000)
    for o in outs:
        lk.lk_submit(c, 0, lk.LK_OP_COPY_I32, n, (da,), o)
    assert c.dispose() == lk.LK_OK      # EXIT queues behind the copies
    for o in outs:
        assert np.array_equal(host(o), a)


def test_status_words_follow_table1(torch_ready):
    with lk.lk_init([1, 1], idle_lease_ns=5_000_000_000) as c:
        assert lk.lk_status(c, 0) == lk.LK_ST_INIT
        lk.lk_wait(c, lk.lk_submit(c, 0, lk.LK_OP_NOP, 0))
        assert lk.lk_status(c, 0) == lk.LK_ST_FINISHED
        assert lk.lk_status(c, 1) == lk.LK_ST_INIT


def test_two_ctas_per_sm_share_every_sm(torch_ready, oracle_lib):
    """ctas_per_sm = 2: both slots of every SM join clusters; slot-major order
    puts cluster 0 (all first CTAs) and cluster 1 (all second CTAs) on the
    same SMs, and every descriptor runs once on the CTAs it was pinned to."""
    torch = torch_ready
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    with lk.lk_init([nsm, nsm], ctas_per_sm=2, exec_log_cap=64, idle_lease_ns=5_000_000_000) as c:
        a, b = lk.lk_cluster_info(c, 0), lk.lk_cluster_info(c, 1)
        assert a == b == sorted(a) and len(set(a)) == nsm
        hs = [lk.lk_submit(c, i % 2, lk.LK_OP_NOP, 0) for i in range(40)]
        assert all(lk.lk_wait(c, h) == lk.LK_OK for h in hs)
        log, _ = lk.lk_exec_log(c)
        verdict, _ = check_log(oracle_lib, c, log, [nsm, nsm], [20, 20], posted_op=[0] * 40)
        assert verdict["violations"] == 0, verdict


def test_two_ctas_per_sm_pinned_lists(torch_ready, oracle_lib):
    lists = [[0, 1, 2], [2, 1], [0]]    # SM 0, 1, 2 each hold two CTAs of different clusters
    with lk.lk_init([3, 2, 1], smids=sum(lists, []), ctas_per_sm=2, exec_log_cap=64,
                    idle_lease_ns=5_000_000_000) as c:
        for k in range(3):
            assert lk.lk_cluster_info(c, k) == lists[k]
        hs = [lk.lk_submit(c, i % 3, lk.LK_OP_NOP, 0) for i in range(30)]
        assert all(lk.lk_wait(c, h) == lk.LK_OK for h in hs)
        log, _ = lk.lk_exec_log(c)
        verdict, _ = check_log(oracle_lib, c, log, [3, 2, 1], [10, 10, 10], posted_op=[0] * 30)
        assert verdict["violations"] == 0, verdict
        for r in log:
            assert r["smid"] == lists[r["cluster"]][r["rank"]]


def test_mailbox_status_words_follow_table1(torch_ready):
    """One-deep mailbox: INIT, WORKING/FINISHED around a descriptor, then the
    master's NOP acknowledgement of the host's re-arm (Table 1)."""
    with lk.lk_init([1, 1], idle_lease_ns=5_000_000_000, flags=lk.LK_INIT_MAILBOX) as c:
        assert lk.lk_status(c, 0) == lk.LK_ST_INIT
        h = lk.lk_submit(c, 0, lk.LK_OP_SPIN, 1 << 20)     # ~2.5 ms of work
        assert lk.lk_submit(c, 0, lk.LK_OP_NOP, 0) is None   # one deep
        t0 = time.monotonic()
        while lk.lk_status(c, 0) != lk.LK_ST_WORKING:
            assert time.monotonic() - t0 < 2.0
        assert lk.lk_wait(c, h) == lk.LK_OK
        t0 = time.monotonic()
        while lk.lk_status(c, 0) != lk.LK_ST_NOP:
            assert time.monotonic() - t0 < 2.0
        assert lk.lk_status(c, 1) == lk.LK_ST_INIT
        assert lk.lk_wait(c, lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)) == lk.LK_OK


def test_baseline_launches_and_pingpong(torch_ready, oracle_lib):
    torch = torch_ready
    n = 65536 + 3
    a = synth.int32_uniform(23, 1, n, -(1 << 20), 1 << 20)
    x = synth.normal_f32(23, 2, n)
    hb = synth.bytes_uniform(23, 3, 1 << 20)
    da, dx, dh = to_dev(a), to_dev(x), to_dev(hb)
    oa = torch.zeros(n, dtype=torch.int32, device="cuda")
    os_ = torch.zeros(4, device="cuda")
    oh = torch.zeros(256, dtype=torch.int32, device="cuda")
    torch.cuda.current_stream().synchronize()
    items = np.zeros(3, dtype=lk.TRACE_ITEM_DTYPE)
    items["cluster"] = [0, 1, 0]
    items["op"] = [lk.LK_OP_ADD_I32, lk.LK_OP_SUM_F32, lk.LK_OP_HIST_U8]
    items["n"] = [n, n, hb.size]
    items["in0"] = [da.data_ptr(), dx.data_ptr(), dh.data_ptr()]
    items["in1"] = [da.data_ptr(), 0, 0]
    items["out"] = [oa.data_ptr(), os_.data_ptr(), oh.data_ptr()]
    rc, res = lk.lk_baseline_run_trace(items, [37, 37], threads=256, n_threads=2)
    assert rc == lk.LK_OK
    assert np.array_equal(host(oa), oracle_lib.add_i32(a, a))
    assert sum_ok(host(os_)[0], x, oracle_lib)
    assert np.array_equal(host(oh).astype(np.int64), oracle_lib.hist_u8(hb))
    rtt = lk.lk_pingpong(2000)
    assert rtt.min() > 0
