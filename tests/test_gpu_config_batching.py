"""A batch of the batching stream (50/50 sum / add items, n log-uniform on
[1024, 2^24] elements, inputs at random offsets of device pools larger than
L2), run as one post on every SM with the tuned split, its outputs remapped to
disjoint buffers: every item of at most 1 MB of input is checked against the
oracle, and a seeded 1 % sample (at least four) of the larger ones."""
import json
import os

import numpy as np
import pytest

from gpu_util import need_gpu
from paper_2310_01212_gb300 import lk, synth, workloads as wl

pytestmark = pytest.mark.gpu


def test_stream_batch_items(native_built, oracle_lib):
    torch = need_gpu()
    import oracle

    seed = wl.BATCHING["seed"]
    pools = wl.Pools.create(seed)
    it, meta = wl.batching_batch(pools, seed, 5)          # 1,457 items
    ops, n = meta["op"], meta["n"].astype(np.int64)
    add = ops == lk.LK_OP_ADD_I32
    # disjoint outputs: adds back to back in one buffer, sums one row each
    offs = np.zeros(ops.size, dtype=np.int64)
    offs[add] = np.concatenate([[0], np.cumsum((n[add] + 3) // 4 * 4)[:-1]])
    add_out = torch.zeros(int(((n[add] + 3) // 4 * 4).sum()) + 4, dtype=torch.int32, device="cuda")
    sum_out = torch.zeros((ops.size, 4), dtype=torch.float32, device="cuda")
    it = it.copy()
    it["out"][add] = add_out.data_ptr() + 4 * offs[add].astype(np.uint64)
    it["out"][~add] = sum_out.data_ptr() + 16 * np.arange(ops.size, dtype=np.uint64)[~add]
    tuned = json.load(open(os.path.join(os.path.dirname(lk.__file__), "autotune_gb300.json")))["best"]
    torch.cuda.synchronize()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    with lk.lk_init([sms], threads_per_cta=tuned["threads"], max_batch_units=1 << 16,
                    idle_lease_ns=5_000_000_000) as c:
        h = lk.lk_submit_batch(c, 0, it, max_parts=tuned["max_parts"], part_bytes=tuned["part_bytes"])
        assert lk.lk_wait(c, h, timeout_ns=30_000_000_000) == lk.LK_OK
    in_bytes = np.where(add, 8 * n, 4 * n)
    small = np.flatnonzero(in_bytes <= (1 << 20))
    large = np.flatnonzero(in_bytes > (1 << 20))
    pick = large[synth.choice(seed, 4242, max(4, large.size // 100), large.size)] if large.size else large
    check = np.unique(np.concatenate([small, pick]))
    assert small.size > 100 and pick.size >= 4
    bad = 0
    for i in check:
        k = int(n[i])
        if add[i]:
            a = pools.i32[int(meta["off0"][i]):int(meta["off0"][i]) + k].cpu().numpy()
            b = pools.i32[int(meta["off1"][i]):int(meta["off1"][i]) + k].cpu().numpy()
            got = add_out[int(offs[i]):int(offs[i]) + k].cpu().numpy()
            bad += 0 if np.array_equal(got, oracle.add_i32(a, b)) else 1
        else:
            x = pools.f32[int(meta["off0"][i]):int(meta["off0"][i]) + k].cpu().numpy()
            got = float(sum_out[i, 0].cpu())
            bad += 0 if abs(got - oracle.sum_f32(x)) <= 1e-4 * oracle.abs_sum_f32(x) else 1
    assert bad == 0, (bad, check.size)
