"""Protocol stress on the GPU (Sec. II.C, Fig. 2): a million NOP descriptors
through a full-chip context, released by several native producer threads,
then checked record by record with the oracle's execution-log checker
(every descriptor exactly once on every CTA of its cluster, per-cluster
FIFO, CTAs on the SMs they booted on, completion after every share).  A
second test has Python producer threads race on the same clusters, so the
ticket path of lk_submit is contended, and checks that the tickets each
cluster handed out are dense and unique.  Every wait has a deadline."""
import threading
import time

import numpy as np
import pytest

from gpu_util import check_log, need_gpu
from paper_2310_01212_gb300 import lk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_ready(native_built):
    return need_gpu()


def full_chip_sizes(torch):
    """Eight clusters of very different sizes that cover every SM."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    head = [1, 3, 4, 8, 16, 24, 32]
    assert sms > sum(head)
    return head + [sms - sum(head)]


@pytest.mark.parametrize("flags,total", [(0, 1_000_000), (lk.LK_INIT_DIRECT, 1_000_000),
                                         (lk.LK_INIT_MAILBOX, 200_000)])
def test_million_nops_native_producers(torch_ready, oracle_lib, flags, total):
    torch = torch_ready
    sizes = full_chip_sizes(torch)
    C = len(sizes)
    items = np.zeros(total, dtype=lk.TRACE_ITEM_DTYPE)
    items["cluster"] = np.arange(total) % C
    items["op"] = lk.LK_OP_NOP
    n_posted = [int(np.count_nonzero(items["cluster"] == c)) for c in range(C)]
    t0 = time.monotonic()
    with lk.lk_init(sizes, exec_log_cap=max(n_posted), idle_lease_ns=30_000_000_000, flags=flags) as c:
        # open loop: four threads, each owning two clusters, release as fast as the rings take them
        rc, res = lk.lk_run_trace(c, items, n_threads=4, closed_loop=False, timeout_ns=120_000_000_000)
        assert rc == lk.LK_OK, lk.lk_strerror(rc)
        assert np.all(res["status"] == lk.LK_OK)
        assert lk.lk_device_error(c) == 0
        # each cluster's completions are observed in its FIFO order
        for k in range(C):
            tc = res["t_complete_ns"][items["cluster"] == k]
            assert np.all(np.diff(tc.astype(np.int64)) >= 0)
        log, dropped = lk.lk_exec_log(c)
        assert dropped == 0
        assert len(log) == sum(s * n for s, n in zip(sizes, n_posted))
        verdict, pinned = check_log(oracle_lib, c, log, sizes, n_posted, posted_op=np.zeros(total, np.int32))
        assert verdict["violations"] == 0, verdict
        assert len(set(pinned)) == sum(sizes)       # every SM exactly once
    wall = time.monotonic() - t0
    span = (res["t_complete_ns"].max() - res["t_submit_ns"].min()) / 1e9
    print(f"\nstress flags {flags}: {total} NOPs over {C} clusters {sizes} in {span:.2f} s "
          f"({total / span / 1e3:.0f} k descriptors/s; {wall:.1f} s with setup and checks)")


@pytest.mark.parametrize("flags,per_thread", [(0, 50_000), (lk.LK_INIT_MAILBOX, 5_000)])
def test_contended_tickets_python_producers(torch_ready, oracle_lib, flags, per_thread):
    torch = torch_ready
    sizes = full_chip_sizes(torch)
    C, P = len(sizes), 4
    got = [[] for _ in range(P)]
    errors = []
    deadline = time.monotonic() + 120.0
    with lk.lk_init(sizes, exec_log_cap=P * per_thread, idle_lease_ns=30_000_000_000, flags=flags) as c:
        def producer(p):
            rng = np.random.default_rng(1000 + p)
            targets = rng.integers(0, C, per_thread)
            try:
                for cl in targets:
                    while True:
                        h = lk.lk_submit(c, int(cl), lk.LK_OP_NOP, 0)
                        if h is not None:
                            break
                        if time.monotonic() > deadline:
                            raise TimeoutError("ring stayed full")
                    got[p].append(h)
            except Exception as e:          # surfaced below, after the join
                errors.append(e)

        th = [threading.Thread(target=producer, args=(p,)) for p in range(P)]
        [t.start() for t in th]
        [t.join() for t in th]
        assert not errors, errors
        assert lk.lk_sync(c, timeout_ns=60_000_000_000) == lk.LK_OK
        assert lk.lk_device_error(c) == 0
        h = np.array(sum(got, []), dtype=np.uint64)
        cl = (h >> np.uint64(48)).astype(np.int64)
        seq = (h & np.uint64((1 << 48) - 1)).astype(np.int64)
        n_posted = [int(np.count_nonzero(cl == k)) for k in range(C)]
        # tickets per cluster: exactly 1..n, each once, whichever thread took them
        for k in range(C):
            assert np.array_equal(np.sort(seq[cl == k]), np.arange(1, n_posted[k] + 1))
        # per producer thread, its own tickets on one cluster increase
        for p in range(P):
            hp = np.array(got[p], dtype=np.uint64)
            for k in range(C):
                s = (hp[(hp >> np.uint64(48)) == k] & np.uint64((1 << 48) - 1)).astype(np.int64)
                assert np.all(np.diff(s) > 0)
        log, dropped = lk.lk_exec_log(c)
        assert dropped == 0
        verdict, _ = check_log(oracle_lib, c, log, sizes, n_posted, posted_op=np.zeros(len(h), np.int32))
        assert verdict["violations"] == 0, verdict
