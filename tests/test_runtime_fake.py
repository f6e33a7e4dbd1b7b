"""Host runtime (liblk_fake.so: the real lk_runtime.cpp over a host-thread
stand-in for the GPU).  Tickets, FIFO handles, ring-full refusals, argument
checks, waits and timeouts, device-side errors, the idle lease, dispose and
the execution log, all without a GPU.  Faults are injected on the host."""
import os
import threading
import time

import numpy as np
import pytest

from paper_2310_01212_gb300 import lk


@pytest.fixture
def fake_env(native_built):
    saved = {k: os.environ.get(k) for k in ("LK_FAKE_SMS", "LK_FAKE_STALL_US", "LK_FAKE_DROP_AFTER",
                                            "LK_FAKE_FAIL_AFTER", "LK_FAKE_NO_BOOT")}
    for k in saved:
        os.environ.pop(k, None)
    yield os.environ
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


def ctx_(sizes=(2, 3), **kw):
    kw.setdefault("exec_log_cap", 256)
    return lk.lk_init(list(sizes), fake=True, **kw)


A = 0x10000   # any 16-byte-aligned "device" address: the fake runs no bodies


def test_boot_clusters_cut_from_sorted_smids(fake_env):
    with ctx_() as c:
        # fake SMs: CTA g on (5g+3) mod 16 -> 3, 8, 13, 2, 7 ; sorted 2,3 | 7,8,13
        assert lk.lk_cluster_info(c, 0) == [2, 3]
        assert lk.lk_cluster_info(c, 1) == [7, 8, 13]
        assert lk.lk_status(c, 0) == lk.LK_ST_INIT
        assert lk.lk_num_ctas(c) == 5 and lk.lk_num_sms(c) == 16


def test_explicit_smid_lists(fake_env):
    with ctx_(sizes=(2, 1), smids=[8, 3, 13]) as c:
        assert lk.lk_cluster_info(c, 0) == [8, 3]
        assert lk.lk_cluster_info(c, 1) == [13]
        h = lk.lk_submit(c, 1, lk.LK_OP_NOP, 0)
        assert lk.lk_wait(c, h) == lk.LK_OK


def test_submit_wait_handles_fifo(fake_env):
    with ctx_() as c:
        hs = [lk.lk_submit(c, i % 2, lk.LK_OP_NOP, 0) for i in range(10)]
        for i, h in enumerate(hs):
            assert h >> 48 == i % 2 and h & ((1 << 48) - 1) == i // 2 + 1
        for h in hs:
            assert lk.lk_wait(c, h) == lk.LK_OK
            assert lk.lk_poll(c, h) == lk.LK_OK
        assert lk.lk_status(c, 0) == lk.LK_ST_FINISHED
        assert lk.lk_sync(c) == lk.LK_OK


@pytest.mark.parametrize("op,ins,out,n", [
    (lk.LK_OP_ADD_I32, (A, A + 8), A, 16),       # misaligned input
    (lk.LK_OP_ADD_I32, (A,), A, 16),             # wrong input count
    (lk.LK_OP_SUM_F32, (A,), None, 16),          # sum needs an output
    (lk.LK_OP_HIST_U8, (A,), A, 1 << 31),        # int32 bins cannot count 2^31
    (lk.LK_OP_COPY_I32, (A,), A + 4, 16),        # misaligned output
    (lk.LK_OP_ADD_I32, (0, A), A, 16),           # null input with n > 0
    (99, (), None, 0),                           # unknown op
])
def test_argument_checks(fake_env, op, ins, out, n):
    with ctx_() as c:
        with pytest.raises(lk.LkError) as e:
            lk.lk_submit(c, 0, op, n, ins, out)
        assert e.value.code == lk.LK_EINVAL


def test_bad_cluster_and_handle(fake_env):
    with ctx_() as c:
        with pytest.raises(lk.LkError):
            lk.lk_submit(c, 2, lk.LK_OP_NOP, 0)
        with pytest.raises(lk.LkError):
            lk.lk_poll(c, 0)
        with pytest.raises(lk.LkError):
            lk.lk_poll(c, (0 << 48) | 5)    # never issued


def test_zero_length_items_allowed(fake_env):
    with ctx_() as c:
        h1 = lk.lk_submit(c, 0, lk.LK_OP_ADD_I32, 0, (0, 0), None)
        h2 = lk.lk_submit(c, 0, lk.LK_OP_SUM_F32, 0, (0,), A)
        assert lk.lk_wait(c, h1) == lk.LK_OK and lk.lk_wait(c, h2) == lk.LK_OK


def test_ring_full_is_refused(fake_env):
    fake_env["LK_FAKE_STALL_US"] = "300000"
    with ctx_(ring_depth=2) as c:
        h0 = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
        h1 = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
        assert lk.lk_submit(c, 0, lk.LK_OP_NOP, 0) is None    # LK_EAGAIN: nothing posted
        assert lk.lk_submit(c, 1, lk.LK_OP_NOP, 0) is not None   # other cluster unaffected
        assert lk.lk_wait(c, h0) == lk.LK_OK
        h2 = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
        assert h2 is not None and h2 & 0xffff == 3
        assert lk.lk_wait(c, h1) == lk.LK_OK and lk.lk_wait(c, h2) == lk.LK_OK


def test_lost_completion_times_out(fake_env):
    fake_env["LK_FAKE_DROP_AFTER"] = "1"
    with ctx_() as c:
        h1 = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
        h2 = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
        assert lk.lk_wait(c, h1) == lk.LK_OK
        t0 = time.monotonic()
        assert lk.lk_wait(c, h2, timeout_ns=50_000_000) == lk.LK_ETIMEDOUT
        assert 0.04 < time.monotonic() - t0 < 2.0
        assert lk.lk_poll(c, h2) == lk.LK_PENDING


def test_device_error_surfaces(fake_env):
    fake_env["LK_FAKE_FAIL_AFTER"] = "1"
    c = ctx_()
    h1 = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
    h2 = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
    assert lk.lk_wait(c, h1) == lk.LK_OK
    with pytest.raises(lk.LkError) as e:
        lk.lk_wait(c, h2)
    assert e.value.code == lk.LK_EDEVICE
    assert lk.lk_device_error(c) == lk.LK_DERR_BADDESC
    assert lk.lk_status(c, 0) == lk.LK_ST_ERROR
    with pytest.raises(lk.LkError) as e:
        lk.lk_submit(c, 1, lk.LK_OP_NOP, 0)
    assert e.value.code == lk.LK_ESTATE
    assert c.dispose() == lk.LK_EDEVICE


def test_bounds_violation_surfaces_as_a_device_error(fake_env):
    """A descriptor that the bounds-checking build stops (LK_DERR_BOUNDS)
    fails its wait with LK_EDEVICE and names the reason, like any device error."""
    fake_env["LK_FAKE_FAIL_AFTER"] = "0"
    fake_env["LK_FAKE_FAIL_CODE"] = str(lk.LK_DERR_BOUNDS)
    c = ctx_([4])
    h = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
    with pytest.raises(lk.LkError) as e:
        lk.lk_wait(c, h)
    assert e.value.code == lk.LK_EDEVICE
    assert lk.lk_device_error(c) == lk.LK_DERR_BOUNDS
    assert c.dispose() == lk.LK_EDEVICE


def test_idle_lease_expires_and_heartbeat_extends(fake_env):
    c = ctx_(idle_lease_ns=300_000_000)
    for _ in range(6):              # 0.6 s of beats: stays up
        time.sleep(0.1)
        assert lk.lk_heartbeat(c) == lk.LK_OK
    h = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
    assert lk.lk_wait(c, h) == lk.LK_OK
    time.sleep(1.0)                 # silence: the lease runs out
    assert lk.lk_device_error(c) == lk.LK_DERR_LEASE
    with pytest.raises(lk.LkError) as e:
        lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
    assert e.value.code == lk.LK_ESTATE
    assert lk.lk_poll(c, h) == lk.LK_OK      # finished work stays finished
    assert c.dispose() == lk.LK_OK


def test_boot_timeout(fake_env):
    fake_env["LK_FAKE_NO_BOOT"] = "1"
    with pytest.raises(lk.LkError) as e:
        ctx_(boot_timeout_ns=100_000_000)
    assert e.value.code == lk.LK_ETIMEDOUT


def test_dispose_aborts_a_stuck_device(fake_env):
    fake_env["LK_FAKE_STALL_US"] = "1500000"
    c = ctx_()
    lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
    time.sleep(0.05)
    t0 = time.monotonic()
    rc = c.dispose(timeout_ns=100_000_000)
    assert rc in (lk.LK_ETIMEDOUT, lk.LK_OK)
    assert time.monotonic() - t0 < 5


@pytest.mark.parametrize("sizes,bad", [((20,), "too many CTAs"), ((0, 2), "empty cluster")])
def test_init_rejects_bad_partitions(fake_env, sizes, bad):
    with pytest.raises(lk.LkError) as e:
        ctx_(sizes=sizes)
    assert e.value.code == lk.LK_EINVAL, bad


@pytest.mark.parametrize("kw", [dict(threads_per_cta=48), dict(ring_depth=3), dict(smids=[1, 1, 2, 3, 4]),
                                dict(smids=[1, 2, 3, 4, 99]), dict(flags=8)])
def test_init_rejects_bad_params(fake_env, kw):
    with pytest.raises(lk.LkError) as e:
        ctx_(**kw)
    assert e.value.code == lk.LK_EINVAL


def test_multi_producer_exec_log_passes_checker(fake_env, oracle_lib):
    import oracle

    sizes = (2, 3, 1)
    c = ctx_(sizes=sizes, exec_log_cap=1024)
    posted = {}
    lock = threading.Lock()

    def producer(p):
        for j in range(150):
            cl = (p + j) % 3
            op = (lk.LK_OP_NOP, lk.LK_OP_ADD_I32, lk.LK_OP_COPY_I32)[j % 3]
            ins = {lk.LK_OP_NOP: (), lk.LK_OP_ADD_I32: (A, A), lk.LK_OP_COPY_I32: (A,)}[op]
            while True:
                h = lk.lk_submit(c, cl, op, 64 if op else 0, ins, A if op else None)
                if h is not None:
                    break
            with lock:
                posted[(h >> 48, h & 0xffffffffffff)] = op

    th = [threading.Thread(target=producer, args=(p,)) for p in range(4)]
    [t.start() for t in th]
    [t.join() for t in th]
    assert lk.lk_sync(c) == lk.LK_OK
    log, dropped = lk.lk_exec_log(c)
    assert dropped == 0
    n_posted = [sum(1 for (cl, _) in posted if cl == k) for k in range(3)]
    posted_op = [posted[(k, s)] for k in range(3) for s in range(1, n_posted[k] + 1)]
    pinned = sum((lk.lk_cluster_info(c, k) for k in range(3)), [])
    res = oracle.check_exec_log(log["seq"], log["cluster"], log["rank"], log["smid"], log["op"], log["order"],
                                sizes, n_posted, pinned_smid=pinned, posted_op=posted_op)
    assert res["violations"] == 0, res
    assert len(log) == sum(n_posted[k] * sizes[k] for k in range(3))
    assert c.dispose() == lk.LK_OK


def test_stress_trace_full_chip_passes_checker(fake_env, oracle_lib):
    """100,000 NOPs from four native producer threads over eight clusters of
    very different sizes covering 152 fake SMs; the whole log is checked."""
    import oracle

    fake_env["LK_FAKE_SMS"] = "152"
    sizes = [1, 3, 4, 8, 16, 24, 32, 64]
    total, C = 100_000, 8
    items = np.zeros(total, dtype=lk.TRACE_ITEM_DTYPE)
    items["cluster"] = np.arange(total) % C
    n_posted = [total // C] * C
    with ctx_(sizes=sizes, exec_log_cap=total // C) as c:
        rc, res = lk.lk_run_trace(c, items, n_threads=4, timeout_ns=60_000_000_000)
        assert rc == lk.LK_OK and np.all(res["status"] == lk.LK_OK)
        log, dropped = lk.lk_exec_log(c)
        assert dropped == 0 and len(log) == sum(sizes) * total // C
        pinned = sum((lk.lk_cluster_info(c, k) for k in range(C)), [])
        assert sorted(pinned) == list(range(152))
        res = oracle.check_exec_log(log["seq"], log["cluster"], log["rank"], log["smid"], log["op"], log["order"],
                                    sizes, n_posted, pinned_smid=pinned, posted_op=np.zeros(total, np.int32))
        assert res["violations"] == 0, res


class _DevBuf:
    """Stands in for a CUDA tensor: what the binding's size check reads."""

    def __init__(self, nbytes, addr=A, is_cuda=True, contiguous=True):
        self.nbytes, self.addr, self.is_cuda, self.contiguous = nbytes, addr, is_cuda, contiguous

    def numel(self):
        return self.nbytes

    def element_size(self):
        return 1

    def is_contiguous(self):
        return self.contiguous

    def data_ptr(self):
        return self.addr


def test_op_bytes_follow_the_operation_definitions():
    n = 1000
    assert lk.op_bytes(lk.LK_OP_NOP, n) == (0, 0, 0)
    assert lk.op_bytes(lk.LK_OP_ADD_I32, n) == (4000, 4000, 4000)
    assert lk.op_bytes(lk.LK_OP_HIST_U8, n) == (1000, 0, 1024)
    assert lk.op_bytes(lk.LK_OP_SUM_F32, n) == (4000, 0, 4)
    assert lk.op_bytes(lk.LK_OP_GEMM64_F32, 3) == (3 * 64 * 64 * 4,) * 3
    assert lk.op_bytes(lk.LK_OP_COPY_I32, n) == (4000, 0, 4000)
    assert lk.op_bytes(lk.LK_OP_COMBINE_SUM, 5) == (16 * 4 + 4, 0, 4)
    assert lk.op_bytes(lk.LK_OP_COMBINE_SUM, 0) == (0, 0, 4)
    assert lk.op_bytes(lk.LK_OP_COMBINE_HIST, 3) == (3 * 1024, 0, 1024)
    assert lk.op_bytes(lk.LK_OP_SPIN, 20000, ctas=7) == (0, 0, 28)


def test_binding_checks_tensor_sizes_before_the_call(fake_env):
    torch = pytest.importorskip("torch")
    with ctx_(sizes=(3,)) as c:
        n = 256
        ok = _DevBuf(4 * n)
        h = lk.lk_submit(c, 0, lk.LK_OP_ADD_I32, n, (ok, ok), ok)
        assert lk.lk_wait(c, h) == lk.LK_OK
        for bad in [(_DevBuf(4 * n - 1), ok, ok), (ok, _DevBuf(4 * n - 4), ok), (ok, ok, _DevBuf(16)),
                    (ok, ok, _DevBuf(4 * n, contiguous=False)), (ok, _DevBuf(4 * n, is_cuda=False), ok)]:
            with pytest.raises(lk.LkError) as e:
                lk.lk_submit(c, 0, lk.LK_OP_ADD_I32, n, bad[:2], bad[2])
            assert e.value.code == lk.LK_EINVAL
        # a host tensor is never a device operand
        with pytest.raises(lk.LkError, match="not a CUDA tensor"):
            lk.lk_submit(c, 0, lk.LK_OP_COPY_I32, 4, (torch.zeros(4, dtype=torch.int32),), ok)
        # spin writes one uint32 per CTA of the cluster
        assert lk.lk_wait(c, lk.lk_submit(c, 0, lk.LK_OP_SPIN, 10, (), _DevBuf(12))) == lk.LK_OK
        with pytest.raises(lk.LkError):
            lk.lk_submit(c, 0, lk.LK_OP_SPIN, 10, (), _DevBuf(8))
        # histogram bins and batch items are checked the same way
        with pytest.raises(lk.LkError):
            lk.lk_submit(c, 0, lk.LK_OP_HIST_U8, 64, (_DevBuf(64),), _DevBuf(1020))
        with pytest.raises(lk.LkError):
            lk.batch_items([(lk.LK_OP_COPY_I32, n, (ok,), _DevBuf(4 * n - 16))])
        # plain ints pass through unchecked (the library checks alignment)
        assert lk.lk_wait(c, lk.lk_submit(c, 0, lk.LK_OP_COPY_I32, n, (A,), A)) == lk.LK_OK
        assert lk.lk_sync(c) == lk.LK_OK


def test_exec_log_ring_keeps_latest(fake_env):
    with ctx_(sizes=(1,), exec_log_cap=4) as c:
        for _ in range(10):
            lk.lk_wait(c, lk.lk_submit(c, 0, lk.LK_OP_NOP, 0))
        log, dropped = lk.lk_exec_log(c, cap=100)
        assert dropped == 6 and log["seq"].tolist() == [7, 8, 9, 10] and log["order"].tolist() == [6, 7, 8, 9]


def test_trace_runner_open_and_closed_loop(fake_env):
    with ctx_(sizes=(1, 1, 1, 1)) as c:
        n = 400
        items = np.zeros(n, dtype=lk.TRACE_ITEM_DTYPE)
        items["t_arrival_ns"] = np.arange(n) * 20_000
        items["cluster"] = np.arange(n) % 4
        items["op"] = lk.LK_OP_NOP
        for closed in (False, True):
            rc, res = lk.lk_run_trace(c, items, n_threads=2, closed_loop=closed)
            assert rc == lk.LK_OK
            assert np.all(res["status"] == lk.LK_OK)
            assert np.all(res["t_complete_ns"] >= res["t_submit_ns"])
            assert np.all(res["t_submit_ns"] >= items["t_arrival_ns"])


def test_trace_runner_reports_device_error(fake_env):
    fake_env["LK_FAKE_FAIL_AFTER"] = "3"
    c = ctx_(sizes=(1,))
    items = np.zeros(10, dtype=lk.TRACE_ITEM_DTYPE)
    items["op"] = lk.LK_OP_NOP
    rc, res = lk.lk_run_trace(c, items, n_threads=1, timeout_ns=5_000_000_000)
    assert rc == lk.LK_EDEVICE
    assert np.sum(res["status"] == lk.LK_OK) == 3
    c.dispose()


def test_finite_mode_runs_the_list(fake_env):
    descs = [(lk.LK_OP_NOP, 0)] * 7
    ms, log = lk.lk_run_finite([2, 1], descs, [0, 1, 0, 0, 1, 0, 1], fake=True, log_cap=64)
    assert ms >= 0
    assert sorted(log[log["cluster"] == 0]["seq"].tolist()) == [1, 1, 2, 2, 3, 3, 4, 4]
    assert sorted(log[log["cluster"] == 1]["seq"].tolist()) == [1, 2, 3]


# ---- batches -------------------------------------------------------------------------
def test_batch_posts_one_descriptor(fake_env):
    with ctx_(sizes=(4,), exec_log_cap=16) as c:
        items = lk.batch_items([(lk.LK_OP_ADD_I32, 1 << 20, (A, A), A), (lk.LK_OP_SUM_F32, 1000, (A,), A),
                                (lk.LK_OP_NOP, 0, (), None)])
        h = lk.lk_submit_batch(c, 0, items)
        assert h is not None and lk.lk_wait(c, h) == lk.LK_OK
        log, _ = lk.lk_exec_log(c)
        assert set(log["op"].tolist()) == {lk.LK_OP_BATCH} and len(log) == 4
        assert lk.lk_wait(c, lk.lk_submit_batch(c, 0, lk.batch_items([]))) == lk.LK_OK   # empty batch


@pytest.mark.parametrize("bad", [
    (lk.LK_OP_ADD_I32, 16, (A, A + 4), A),      # misaligned
    (lk.LK_OP_SUM_F32, 16, (A,), None),         # sum needs an output
    (9, 16, (A,), A),                           # unknown op
    (lk.LK_OP_COPY_I32, 16, (A,), A, 9),        # more than 8 parts
])
def test_batch_item_checks(fake_env, bad):
    with ctx_() as c:
        with pytest.raises(lk.LkError) as e:
            lk.lk_submit_batch(c, 0, lk.batch_items([bad]))
        assert e.value.code == lk.LK_EINVAL


def test_batch_unit_capacity(fake_env):
    with ctx_(sizes=(8,), max_batch_units=64) as c:
        ok = lk.batch_items([(lk.LK_OP_COPY_I32, 1 << 24, (A,), A, 8)] * 8)      # 64 units
        assert lk.lk_wait(c, lk.lk_submit_batch(c, 0, ok)) == lk.LK_OK
        with pytest.raises(lk.LkError):
            lk.lk_submit_batch(c, 0, lk.batch_items([(lk.LK_OP_COPY_I32, 1 << 24, (A,), A, 8)] * 9))


def test_batch_tables_busy_is_refused(fake_env):
    fake_env["LK_FAKE_STALL_US"] = "300000"
    with ctx_(sizes=(2,)) as c:
        items = lk.batch_items([(lk.LK_OP_NOP, 0, (), None)])
        h1 = lk.lk_submit_batch(c, 0, items)
        h2 = lk.lk_submit_batch(c, 0, items)
        assert h1 and h2
        assert lk.lk_submit_batch(c, 0, items) is None     # both unit tables still in use
        assert lk.lk_wait(c, h1) == lk.LK_OK
        h3 = lk.lk_submit_batch(c, 0, items)
        assert h3 is not None
        assert lk.lk_wait(c, h3) == lk.LK_OK


def test_split_rule_counts_units(fake_env):
    # parts = ceil(input bytes / part_bytes) capped by max_parts and the cluster size
    with ctx_(sizes=(4,), max_batch_units=10) as c:
        items = lk.batch_items([(lk.LK_OP_SUM_F32, 1 << 20, (A,), A)] * 2)      # 4 MiB each
        assert lk.lk_wait(c, lk.lk_submit_batch(c, 0, items, part_bytes=1 << 20)) == lk.LK_OK   # 4 + 4 units
        with pytest.raises(lk.LkError):   # 3 items x 4 parts = 12 > 10
            lk.lk_submit_batch(c, 0, lk.batch_items([(lk.LK_OP_SUM_F32, 1 << 20, (A,), A)] * 3), part_bytes=1 << 20)
        assert lk.lk_wait(c, lk.lk_submit_batch(c, 0, lk.batch_items([(lk.LK_OP_SUM_F32, 1 << 20, (A,), A)] * 3),
                                                max_parts=2, part_bytes=1 << 20)) == lk.LK_OK


# ---- serving ---------------------------------------------------------------------------
def _reqs(n, ops, sizes, producers=4, gap_ns=20_000, out=None):
    r = np.zeros(n, dtype=lk.REQUEST_DTYPE)
    r["t_arrival_ns"] = np.arange(n) * gap_ns
    r["op"] = [ops[i % len(ops)] for i in range(n)]
    r["producer"] = np.arange(n) % producers
    r["n"] = [sizes[i % len(sizes)] for i in range(n)]
    r["in0"] = A
    r["in1"] = A
    r["out"] = 0 if out is None else out
    return r


def test_serve_admits_chunks_and_combines(fake_env):
    with ctx_(sizes=(2, 2, 2), exec_log_cap=4096) as c:
        reqs = _reqs(60, [lk.LK_OP_ADD_I32, lk.LK_OP_SUM_F32, lk.LK_OP_HIST_U8, lk.LK_OP_GEMM64_F32],
                     [1 << 10, 5 << 20, 3 << 20, 40])
        rc, res = lk.lk_serve(c, reqs, n_producers=4, budget_bytes=1 << 34, arena=1 << 20, arena_bytes=1 << 34,
                              chunk_bytes=1 << 20)
        assert rc == lk.LK_OK and np.all(res["status"] == lk.LK_OK)
        assert np.all(res["t_complete_ns"] >= res["t_admit_ns"])
        assert np.all(res["t_admit_ns"] >= reqs["t_arrival_ns"])
        # chunks: ceil(input bytes / 1 MiB) in whole alignment units
        want = {lk.LK_OP_ADD_I32: 1, lk.LK_OP_SUM_F32: 20, lk.LK_OP_HIST_U8: 3, lk.LK_OP_GEMM64_F32: 2}
        for r, q in zip(reqs, res):
            assert q["chunks"] == want[int(r["op"])], (int(r["op"]), q["chunks"])
        log, _ = lk.lk_exec_log(c, cap=1 << 16)
        ops = log["op"]
        # 15 split sums and 15 split histograms, each finished by one combine (2 ranks log each)
        assert np.sum(ops == lk.LK_OP_COMBINE_SUM) == 2 * 15 and np.sum(ops == lk.LK_OP_COMBINE_HIST) == 2 * 15
        # arena outputs were handed out and given back: all 256-byte aligned
        assert np.all(res["out"] % 256 == 0)


def test_serve_coalesces_small_requests(fake_env):
    """Requests of at most coalesce_bytes go out many to a batch post: fewer
    posts than requests, every request finished, larger ones still chunked."""
    fake_env["LK_FAKE_STALL_US"] = "200"
    with ctx_(sizes=(2, 2), exec_log_cap=4096) as c:
        reqs = _reqs(200, [lk.LK_OP_ADD_I32, lk.LK_OP_SUM_F32, lk.LK_OP_HIST_U8], [1 << 10, 1 << 12, 1 << 14],
                     gap_ns=0)
        big = _reqs(4, [lk.LK_OP_SUM_F32], [5 << 20], gap_ns=0)
        allr = np.concatenate([reqs, big])
        rc, res = lk.lk_serve(c, allr, n_producers=4, budget_bytes=1 << 34, arena=1 << 20, arena_bytes=1 << 34,
                              chunk_bytes=1 << 20, coalesce_bytes=1 << 16, coalesce_max=64)
        assert rc == lk.LK_OK and np.all(res["status"] == lk.LK_OK)
        assert np.all(res["chunks"][:200] == 1) and np.all(res["chunks"][200:] == 20)
        log, _ = lk.lk_exec_log(c, cap=1 << 16)
        batches = int(np.sum(log["op"] == lk.LK_OP_BATCH)) // 2       # two ranks log each post
        assert 4 <= batches < 200
        assert np.sum(log["op"] == lk.LK_OP_COMBINE_SUM) == 2 * 4


@pytest.mark.parametrize("units,kw", [(8192, dict(coalesce_bytes=2 << 20, chunk_bytes=1 << 20)),   # > chunk
                                      (8192, dict(coalesce_max=300)),                            # > 256
                                      (1024, dict())])                     # 256 items x 8 parts > table
def test_serve_coalesce_checks(fake_env, units, kw):
    with ctx_(sizes=(1,), max_batch_units=units) as c:
        kw.setdefault("coalesce_bytes", 1 << 16)
        kw.setdefault("chunk_bytes", 1 << 20)
        rc, _ = lk.lk_serve(c, _reqs(1, [lk.LK_OP_COPY_I32], [16]), n_producers=4, budget_bytes=1 << 30,
                            arena=1 << 20, arena_bytes=1 << 30, **kw)
        assert rc == lk.LK_EINVAL


def test_serve_budget_limits_admission(fake_env):
    fake_env["LK_FAKE_STALL_US"] = "2000"
    with ctx_(sizes=(1, 1)) as c:
        reqs = _reqs(8, [lk.LK_OP_COPY_I32], [1 << 20], producers=2, gap_ns=0)   # 8 MiB held each
        rc, res = lk.lk_serve(c, reqs, n_producers=2, budget_bytes=8 << 20, arena=1 << 20, arena_bytes=1 << 30)
        assert rc == lk.LK_OK
        # one request fits the budget at a time: admissions are serialised
        order = np.argsort(res["t_admit_ns"])
        adm, comp = res["t_admit_ns"][order], res["t_complete_ns"][order]
        assert np.all(adm[1:] >= comp[:-1])


def test_serve_rejects_requests_larger_than_the_budget(fake_env):
    with ctx_(sizes=(1,)) as c:
        reqs = _reqs(1, [lk.LK_OP_COPY_I32], [1 << 20])
        rc, _ = lk.lk_serve(c, reqs, n_producers=4, budget_bytes=1 << 20, arena=1 << 20, arena_bytes=1 << 30)
        assert rc == lk.LK_ENOMEM


def test_serve_needs_equal_clusters(fake_env):
    with ctx_(sizes=(1, 2)) as c:
        rc, _ = lk.lk_serve(c, _reqs(1, [lk.LK_OP_NOP + 1], [16]), n_producers=4, budget_bytes=1 << 30,
                            arena=1 << 20, arena_bytes=1 << 30)
        assert rc == lk.LK_EINVAL


def test_phase_run_on_fake(fake_env):
    res = lk.lk_phase_run(sms=2, iters=100, runs=5, fake=True)
    assert res.size == 5
    for f in ("init_ns", "trigger_ns", "wait_ns", "dispose_ns"):
        assert np.all(res[f] > 0)


# ---- the paper's one-deep mailbox (LK_INIT_MAILBOX, Sec. II.D, Table 1) ----------
def test_mailbox_four_phase_handshake(fake_env):
    fake_env["LK_FAKE_STALL_US"] = "200000"
    with ctx_(sizes=(2, 1), flags=lk.LK_INIT_MAILBOX) as c:
        assert lk.lk_status(c, 0) == lk.LK_ST_INIT
        h1 = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
        assert h1 is not None and h1 & 0xffff == 1
        time.sleep(0.05)
        assert lk.lk_status(c, 0) == lk.LK_ST_WORKING          # master answered
        assert lk.lk_submit(c, 0, lk.LK_OP_NOP, 0) is None    # one deep: EAGAIN
        assert lk.lk_submit(c, 1, lk.LK_OP_NOP, 0) is not None   # other mailbox unaffected
        assert lk.lk_poll(c, h1) == lk.LK_PENDING
        assert lk.lk_wait(c, h1) == lk.LK_OK                   # saw FINISHED, re-armed
        # the master acknowledges the re-arm with from_GPU = THREAD_NOP
        t0 = time.monotonic()
        while lk.lk_status(c, 0) != lk.LK_ST_NOP:
            assert time.monotonic() - t0 < 2.0
        h2 = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
        assert h2 is not None and h2 & 0xffff == 2
        assert lk.lk_wait(c, h2) == lk.LK_OK
        assert lk.lk_sync(c) == lk.LK_OK


def test_mailbox_rejects_direct(fake_env):
    with pytest.raises(lk.LkError) as e:
        ctx_(flags=lk.LK_INIT_MAILBOX | lk.LK_INIT_DIRECT)
    assert e.value.code == lk.LK_EINVAL


def test_mailbox_multi_producer_exec_log_passes_checker(fake_env, oracle_lib):
    """Racing producers drive the handshake themselves (a refused post
    re-arms a FINISHED mailbox); every descriptor runs once, in order."""
    import oracle

    sizes = (2, 3)
    c = ctx_(sizes=sizes, exec_log_cap=1024, flags=lk.LK_INIT_MAILBOX)
    posted = {}
    lock = threading.Lock()

    def producer(p):
        for j in range(60):
            cl = (p + j) % 2
            op = (lk.LK_OP_NOP, lk.LK_OP_COPY_I32)[j % 2]
            while True:
                h = lk.lk_submit(c, cl, op, 64 if op else 0, (A,) if op else (), A if op else None)
                if h is not None:
                    break
            with lock:
                posted[(h >> 48, h & 0xffffffffffff)] = op

    th = [threading.Thread(target=producer, args=(p,)) for p in range(3)]
    [t.start() for t in th]
    [t.join() for t in th]
    assert lk.lk_sync(c) == lk.LK_OK
    log, dropped = lk.lk_exec_log(c)
    assert dropped == 0
    n_posted = [sum(1 for (cl, _) in posted if cl == k) for k in range(2)]
    assert sum(n_posted) == 180
    posted_op = [posted[(k, s)] for k in range(2) for s in range(1, n_posted[k] + 1)]
    pinned = sum((lk.lk_cluster_info(c, k) for k in range(2)), [])
    res = oracle.check_exec_log(log["seq"], log["cluster"], log["rank"], log["smid"], log["op"], log["order"],
                                sizes, n_posted, pinned_smid=pinned, posted_op=posted_op)
    assert res["violations"] == 0, res
    assert c.dispose() == lk.LK_OK


def test_mailbox_trace_runner_and_dispose(fake_env):
    with ctx_(sizes=(1, 2), flags=lk.LK_INIT_MAILBOX) as c:
        n = 200
        items = np.zeros(n, dtype=lk.TRACE_ITEM_DTYPE)
        items["cluster"] = np.arange(n) % 2
        items["op"] = lk.LK_OP_NOP
        for closed in (True, False):
            rc, res = lk.lk_run_trace(c, items, n_threads=2, closed_loop=closed)
            assert rc == lk.LK_OK and np.all(res["status"] == lk.LK_OK)


def test_mailbox_lost_completion_and_lease(fake_env):
    fake_env["LK_FAKE_DROP_AFTER"] = "1"
    c = ctx_(sizes=(1,), flags=lk.LK_INIT_MAILBOX, idle_lease_ns=200_000_000)
    h1 = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
    assert lk.lk_wait(c, h1) == lk.LK_OK
    t0 = time.monotonic()
    while (h2 := lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)) is None:
        assert time.monotonic() - t0 < 2.0
    assert lk.lk_wait(c, h2, timeout_ns=50_000_000) == lk.LK_ETIMEDOUT   # FINISHED never comes
    assert lk.lk_submit(c, 0, lk.LK_OP_NOP, 0) is None                   # still one deep
    time.sleep(0.8)                                                      # no heartbeat: the lease ends
    assert lk.lk_device_error(c) == lk.LK_DERR_LEASE
    assert lk.lk_poll(c, h1) == lk.LK_OK
    assert c.dispose() == lk.LK_OK


# ---- two persistent CTAs per SM (ctas_per_sm = 2) ---------------------------------
def test_two_ctas_per_sm_slot_major_clusters(fake_env):
    """16 fake SMs x 2: every SM's first CTA (by SM id) before any second CTA,
    so clusters 0 and 1 below sit on the same eight SMs."""
    with ctx_(sizes=(8, 8, 8, 8), ctas_per_sm=2) as c:
        info = [lk.lk_cluster_info(c, k) for k in range(4)]
        assert info[0] == list(range(8)) and info[1] == list(range(8, 16))
        assert info[2] == list(range(8)) and info[3] == list(range(8, 16))
        hs = [lk.lk_submit(c, i % 4, lk.LK_OP_NOP, 0) for i in range(40)]
        assert all(lk.lk_wait(c, h) == lk.LK_OK for h in hs)


def test_two_ctas_per_sm_pinned_lists(fake_env, oracle_lib):
    import oracle

    # SM 3 appears twice: its first CTA joins cluster 0, its second cluster 1
    lists = [[3, 5], [3, 9, 5]]
    with ctx_(sizes=(2, 3), smids=lists[0] + lists[1], ctas_per_sm=2, exec_log_cap=64) as c:
        assert lk.lk_cluster_info(c, 0) == lists[0] and lk.lk_cluster_info(c, 1) == lists[1]
        hs = [lk.lk_submit(c, i % 2, lk.LK_OP_NOP, 0) for i in range(10)]
        assert all(lk.lk_wait(c, h) == lk.LK_OK for h in hs)
        log, _ = lk.lk_exec_log(c)
        res = oracle.check_exec_log(log["seq"], log["cluster"], log["rank"], log["smid"], log["op"], log["order"],
                                    [2, 3], [5, 5], pinned_smid=lists[0] + lists[1], posted_op=[0] * 10)
        assert res["violations"] == 0, res


@pytest.mark.parametrize("kw", [dict(sizes=(8,), ctas_per_sm=3),                      # one or two only
                                dict(sizes=(17, 16), ctas_per_sm=2),                  # > 2 x 16 CTAs
                                dict(sizes=(2,), ctas_per_sm=2, threads_per_cta=512),  # registers
                                dict(sizes=(3,), smids=[4, 4, 4], ctas_per_sm=2),     # an SM thrice
                                dict(sizes=(2,), smids=[4, 4])])                      # twice, one per SM
def test_two_ctas_per_sm_rejects(fake_env, kw):
    sizes = kw.pop("sizes")
    with pytest.raises(lk.LkError) as e:
        ctx_(sizes=sizes, **kw)
    assert e.value.code == lk.LK_EINVAL


# ---- load-rate caps (lk_set_rate, lk_desc.aux) --------------------------------------
def test_rate_caps_are_checked(fake_env):
    with ctx_() as c:
        lk.lk_set_rate(c, 0, 0)
        lk.lk_set_rate(c, 1, lk.LK_RATE_MIN)
        for bad in (1, lk.LK_RATE_MIN - 1, 1 << 40):
            with pytest.raises(lk.LkError) as e:
                lk.lk_set_rate(c, 0, bad)
            assert e.value.code == lk.LK_EINVAL
        with pytest.raises(lk.LkError) as e:
            lk.lk_set_rate(c, 2, 5000)       # no such cluster
        assert e.value.code == lk.LK_EINVAL
        with pytest.raises(lk.LkError) as e:
            lk.lk_submit(c, 0, lk.LK_OP_COPY_I32, 64, (A,), A, aux=999)
        assert e.value.code == lk.LK_EINVAL
        h = lk.lk_submit(c, 0, lk.LK_OP_COPY_I32, 64, (A,), A, aux=5000)
        assert lk.lk_wait(c, h) == lk.LK_OK


# ---- load yielding (lk_set_role) -----------------------------------------------------
def test_roles_are_checked(fake_env):
    with ctx_() as c:
        for cl, role in ((0, lk.LK_ROLE_CRITICAL), (1, lk.LK_ROLE_YIELD), (1, lk.LK_ROLE_NONE)):
            lk.lk_set_role(c, cl, role)
        for cl, role in ((0, 3), (0, -1), (2, lk.LK_ROLE_YIELD), (-1, lk.LK_ROLE_CRITICAL)):
            with pytest.raises(lk.LkError) as e:
                lk.lk_set_role(c, cl, role)
            assert e.value.code == lk.LK_EINVAL


@pytest.mark.parametrize("flags", [0, lk.LK_INIT_DIRECT, lk.LK_INIT_MAILBOX])
def test_role_bits_ride_the_wire(fake_env, flags):
    """The role travels as flag bits of the posted descriptor next to a rate
    cap: every delivery mode still carries and completes such descriptors,
    batches included."""
    with ctx_(flags=flags) as c:
        lk.lk_set_role(c, 0, lk.LK_ROLE_CRITICAL)
        lk.lk_set_role(c, 1, lk.LK_ROLE_YIELD)
        lk.lk_set_rate(c, 1, 5000)
        for i in range(12):   # one at a time: the mailbox holds one descriptor per cluster
            assert lk.lk_wait(c, lk.lk_submit(c, i % 2, lk.LK_OP_COPY_I32, 64, (A,), A)) == lk.LK_OK
        for cl in (0, 1):
            items = lk.batch_items([(lk.LK_OP_COPY_I32, 64, (A,), A)] * 3)
            assert lk.lk_wait(c, lk.lk_submit_batch(c, cl, items)) == lk.LK_OK


def test_gemm_ffma_flag_accepted(fake_env):
    with ctx_(flags=lk.LK_INIT_GEMM_FFMA | lk.LK_INIT_MAILBOX) as c:
        assert lk.lk_wait(c, lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)) == lk.LK_OK


# ---- serving through the device-resident queue (LK_SERVE_QUEUE) --------------------------
def _queue_arena(extra=1 << 20, max_inflight=64):
    """A real host buffer stands in for the arena (the fake's device memory
    is host memory): the queue's state lives at its start."""
    n = lk.lk_serve_queue_state_bytes(max_inflight) + extra
    buf = np.zeros(n + 256, dtype=np.uint8)
    base = (buf.ctypes.data + 255) // 256 * 256
    return buf, base, n


def _serve_q(c, reqs, **kw):
    buf, base, n = _queue_arena(max_inflight=kw.get("max_inflight", 64))
    kw.setdefault("max_inflight", 64)
    kw.setdefault("part_bytes", 1 << 20)
    kw.setdefault("min_part_bytes", kw["part_bytes"])   # no spreading unless a test asks for it
    rc, res = lk.lk_serve(c, reqs, n_producers=4, budget_bytes=kw.pop("budget_bytes", 1 << 34), arena=base,
                          arena_bytes=n, mode=lk.LK_SERVE_QUEUE, **kw)
    del buf
    return rc, res


def test_queue_serves_every_request_with_its_units(fake_env):
    with ctx_(sizes=(2, 2, 2)) as c:
        reqs = _reqs(80, [lk.LK_OP_ADD_I32, lk.LK_OP_SUM_F32, lk.LK_OP_HIST_U8, lk.LK_OP_GEMM64_F32, lk.LK_OP_COPY_I32],
                     [1 << 10, 5 << 20, 3 << 20, 40, 0])
        rc, res = _serve_q(c, reqs)
        assert rc == lk.LK_OK and np.all(res["status"] == lk.LK_OK)
        assert np.all(res["t_complete_ns"] >= res["t_admit_ns"])
        assert np.all(res["t_admit_ns"] >= reqs["t_arrival_ns"])
        # units: ceil(input bytes / 1 MiB), at least one
        want = {lk.LK_OP_ADD_I32: 1, lk.LK_OP_SUM_F32: 20, lk.LK_OP_HIST_U8: 3, lk.LK_OP_GEMM64_F32: 2,
                lk.LK_OP_COPY_I32: 1}
        for r, q in zip(reqs, res):
            assert q["chunks"] == want[int(r["op"])], (int(r["op"]), q["chunks"])
        assert np.all(res["out"] % 256 == 0)
        # the context serves ordinary descriptors again afterwards
        assert lk.lk_wait(c, lk.lk_submit(c, 1, lk.LK_OP_NOP, 0)) == lk.LK_OK


def test_serve_parts_rule():
    """The exported split rule, host-only, at the defaults (8 MiB parts, 128 KiB
    minimum, so 1 MiB units while not saturated) on 148 CTAs."""
    MiB = 1 << 20
    P = lk.lk_serve_parts
    # add of 512 MiB input: 1 MiB units unless the backlog saturates the queue
    assert P(lk.LK_OP_ADD_I32, 64 * MiB, 148) == 512
    assert P(lk.LK_OP_ADD_I32, 64 * MiB, 148, 10, 148 * 8 * MiB) == 138        # saturated: max(64, 138 idle)
    assert P(lk.LK_OP_ADD_I32, 64 * MiB, 148, 500, 148 * 8 * MiB) == 64        # and no idle CTA
    assert P(lk.LK_OP_ADD_I32, 64 * MiB, 148, 500, 148 * 8 * MiB - 1) == 512   # just below saturation
    # a sum's width ignores the backlog: max(ceil(B / 8 MiB), min(148, ceil(B / 128 KiB)))
    for bu, bb in ((0, 0), (500, 1 << 40)):
        assert P(lk.LK_OP_SUM_F32, 1 << 20, 148, bu, bb) == 32
        assert P(lk.LK_OP_SUM_F32, 1 << 26, 148, bu, bb) == 148
        assert P(lk.LK_OP_SUM_F32, 1 << 30, 148, bu, bb) == 512
    # a 1 MiB histogram behind 200 queued units: one unit
    assert P(lk.LK_OP_HIST_U8, MiB, 148, 200, 0) == 1
    # GEMM: whole tiles
    assert P(lk.LK_OP_GEMM64_F32, 3, 148) == 1
    assert P(lk.LK_OP_GEMM64_F32, 1000, 148) == 148
    assert P(lk.LK_OP_GEMM64_F32, 1000, 148, 140, 0) == 32
    # refused
    for args in ((lk.LK_OP_NOP, 1, 148), (lk.LK_OP_SPIN, 1, 148), (lk.LK_OP_ADD_I32, 1, 0)):
        assert P(*args) == 0
    assert P(lk.LK_OP_ADD_I32, 1, 148, 0, 0, 8 * MiB, 1000) == 0
    assert P(lk.LK_OP_ADD_I32, 1, 148, 0, 0, (1 << 40) + 1, 0) == 0


def test_queue_split_rule(fake_env):
    """A sum gets exactly max(ceil(B / part), min(CTAs, ceil(B / min_part)))
    units, whatever else runs; another op spreads over the CTAs no unclaimed
    unit waits for (here all six: nothing else is queued at once), and with
    the queue not saturated never takes units above max(min_part, part / 8)."""
    with ctx_(sizes=(2, 2, 2)) as c:
        ops = [lk.LK_OP_SUM_F32, lk.LK_OP_SUM_F32, lk.LK_OP_SUM_F32, lk.LK_OP_COPY_I32, lk.LK_OP_COPY_I32,
               lk.LK_OP_HIST_U8, lk.LK_OP_GEMM64_F32]
        ns = [1 << 10, 1 << 18, 9 << 20, 1 << 18, 9 << 20, 1 << 20, 3]
        reqs = _reqs(len(ops), ops, ns, gap_ns=3_000_000, out=A)
        rc, res = _serve_q(c, reqs, part_bytes=4 << 20, min_part_bytes=64 << 10)
        assert rc == lk.LK_OK
        got = res["chunks"].tolist()
        # sums (6 CTAs): 4 KiB -> 1; 1 MiB -> min(6, 16) = 6; 36 MiB -> max(9, 6) = 9
        # copy 1 MiB -> max(2, min(6 idle, 16)) = 6; copy 36 MiB -> units of at
        # most 512 KiB (part / 8): max(72, min(6, 576)) = 72
        # hist 1 MiB -> 6; gemm 3 tiles (96 KiB) -> min(6, 2, 3 tiles) = 2
        assert got == [1, 6, 9, 6, 72, 6, 2], got
        # lk_serve_parts states the same rule
        assert got == [lk.lk_serve_parts(o, n, 6, 0, 0, 4 << 20, 64 << 10) for o, n in zip(ops, ns)]


def test_queue_serves_twice_and_empty(fake_env):
    with ctx_(sizes=(1, 1)) as c:
        for k in range(3):
            reqs = _reqs(0 if k == 1 else 30, [lk.LK_OP_SUM_F32, lk.LK_OP_COPY_I32], [3 << 20, 1 << 12])
            rc, res = _serve_q(c, reqs)
            assert rc == lk.LK_OK and np.all(res["status"] == lk.LK_OK)


def test_queue_interleaves_a_late_small_request(fake_env):
    """A small request that arrives while a large one is still being
    published is not queued behind all of its units: round-robin publication
    with a bounded window lets it finish first."""
    fake_env["LK_FAKE_STALL_US"] = "300"
    with ctx_(sizes=(1, 1)) as c:
        big = _reqs(1, [lk.LK_OP_COPY_I32], [256 << 20], gap_ns=0, out=A)   # 1024 units of 1 MiB
        small = _reqs(1, [lk.LK_OP_COPY_I32], [1 << 10], gap_ns=0, out=A)
        small["t_arrival_ns"] = 5_000_000
        rc, res = _serve_q(c, np.concatenate([big, small]), window=2)
        assert rc == lk.LK_OK and res["chunks"][0] == 1024
        assert res["t_complete_ns"][1] < res["t_complete_ns"][0]
        assert res["t_complete_ns"][1] - res["t_admit_ns"][1] < 50_000_000


def test_queue_budget_limits_admission(fake_env):
    fake_env["LK_FAKE_STALL_US"] = "1000"
    with ctx_(sizes=(1, 1)) as c:
        reqs = _reqs(6, [lk.LK_OP_COPY_I32], [1 << 20], producers=2, gap_ns=0, out=A)   # 8 MiB held each
        rc, res = _serve_q(c, reqs, budget_bytes=8 << 20)
        assert rc == lk.LK_OK
        order = np.argsort(res["t_admit_ns"])
        assert np.all(res["t_admit_ns"][order][1:] >= res["t_complete_ns"][order][:-1])


def test_queue_slots_limit_admission(fake_env):
    fake_env["LK_FAKE_STALL_US"] = "500"
    with ctx_(sizes=(2,)) as c:
        reqs = _reqs(12, [lk.LK_OP_SUM_F32], [1 << 10], gap_ns=0)
        rc, res = _serve_q(c, reqs, max_inflight=2)
        assert rc == lk.LK_OK and np.all(res["status"] == lk.LK_OK)
        # never more than two admitted and unfinished at once
        ev = sorted([(t, 1) for t in res["t_admit_ns"]] + [(t, -1) for t in res["t_complete_ns"]],
                    key=lambda e: (e[0], e[1]))
        live = np.cumsum([e[1] for e in ev])
        assert live.max() <= 2


@pytest.mark.parametrize("kw", [dict(part_bytes=1 << 12), dict(max_inflight=1 << 20), dict(mode=7)])
def test_queue_argument_checks(fake_env, kw):
    with ctx_(sizes=(1,)) as c:
        buf, base, n = _queue_arena()
        mode = kw.pop("mode", lk.LK_SERVE_QUEUE)
        rc, _ = lk.lk_serve(c, _reqs(1, [lk.LK_OP_COPY_I32], [16]), n_producers=4, budget_bytes=1 << 30,
                            arena=base, arena_bytes=n, mode=mode, **kw)
        assert rc == lk.LK_EINVAL


def test_queue_needs_arena_for_its_state(fake_env):
    with ctx_(sizes=(1,)) as c:
        buf, base, n = _queue_arena()
        rc, _ = lk.lk_serve(c, _reqs(1, [lk.LK_OP_COPY_I32], [16]), n_producers=4, budget_bytes=1 << 30,
                            arena=base, arena_bytes=1024, mode=lk.LK_SERVE_QUEUE)
        assert rc == lk.LK_ENOMEM


def test_queue_device_error_ends_the_call(fake_env):
    fake_env["LK_FAKE_FAIL_AFTER"] = "0"
    with ctx_(sizes=(1,)) as c:
        rc, res = _serve_q(c, _reqs(5, [lk.LK_OP_COPY_I32], [16]))
        assert rc != lk.LK_OK
