"""Synthetic workloads of the dispatch configurations: partitions, body mixes,
sizes, value distributions and arrival processes.  Numbers are drawn with
``synth``; nothing here computes a work body or the dispatch protocol.

Configurations (all seeded):
  small      4 SMs as 2 clusters of 2, 256 threads; 10,000 closed-loop int32
             adds of 4096 elements, values uniform on [-2^20, 2^20],
             round-robin over the clusters.
  full_chip  148 SMs as 4 clusters of 37, 256 threads; the four bodies in
             equal shares, shuffled: int32 add of 65,536 elements, histogram
             of 1 MiB of uniform bytes, float32 sum of 65,536 N(0,1) values,
             one 64x64x64 float32 GEMM tile of N(0,1) values; Poisson
             arrivals at 20,000 per second; round-robin clusters; one host
             submitter thread per cluster.
  batching   batches of int-log-uniform 1..4096 items, item sizes
             log-uniform 1,024..16,777,216 elements, float32 sum / int32 add
             50/50, one post per batch to a cluster of every SM; a seeded
             prefix of the 1,000,000-descriptor stream.
  serving    8 host producer threads, open-loop Poisson arrivals at 5k..200k
             requests/s, request sizes log-uniform 4 KB..256 MB over the four
             bodies (a GEMM request of S bytes is floor(S / 48 KB) >= 1 tiles),
             admission by a 64 GB budget, 148 SMs as 4 clusters of 37; the
             device-resident queue splits requests into units of at most 8 MiB, spread
             over idle CTAs down to 128 KiB units.
  isolation  a critical cluster of 16 SMs releases an FP32 sum over 1 MB
             (262,144 N(0,1) values) every 1 ms, waiting for each; a
             best-effort cluster of 132 SMs runs int32 copies of 4 GiB and
             histograms of 256 MiB back to back; the critical latencies are
             measured alone and under that load.
Inputs of full_chip items are slices of device pools much larger than L2
(129 MB on GB300) at random 16-byte-aligned offsets, so every item reads
from HBM.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import lk, synth

SMALL = dict(sizes=[2, 2], threads=256, items=10_000, n=4096, lo=-(1 << 20), hi=1 << 20, seed=0)
FULL_CHIP = dict(sizes=[37, 37, 37, 37], threads=256, rate_per_s=20_000.0, n_add=65_536, n_hist=1 << 20,
                 n_sum=65_536, gemm_tiles=1, seed=0)
BATCHING = dict(max_count=4096, n_lo=1024, n_hi=16_777_216, seed=0)
SERVING = dict(sizes=[37, 37, 37, 37], threads=256, producers=8, rates=(5_000, 10_000, 20_000, 50_000, 100_000, 200_000),
               s_lo=4096, s_hi=256 << 20, budget_bytes=64 << 30, arena_bytes=24 << 30, chunk_bytes=64 << 20, window=2,
               coalesce_bytes=4 << 20, coalesce_part_bytes=256 << 10, part_bytes=8 << 20, min_part_bytes=128 << 10,
               queue_window=2,
               seed=0)
ISOLATION = dict(sizes=[16, 132], threads=256, period_ns=1_000_000, crit_n=262_144, copy_n=1 << 30,
                 hist_n=256 << 20, seed=0)
OPS4 = (lk.LK_OP_ADD_I32, lk.LK_OP_HIST_U8, lk.LK_OP_SUM_F32, lk.LK_OP_GEMM64_F32)


def item_bytes(op: int, n: int) -> tuple[int, int, int]:
    """(in0, in1, out) bytes an item moves: the algorithmic traffic of its body."""
    if op == lk.LK_OP_ADD_I32:
        return 4 * n, 4 * n, 4 * n
    if op == lk.LK_OP_COPY_I32:
        return 4 * n, 0, 4 * n
    if op == lk.LK_OP_HIST_U8:
        return n, 0, 1024
    if op == lk.LK_OP_SUM_F32:
        return 4 * n, 0, 4
    if op == lk.LK_OP_GEMM64_F32:
        return 16384 * n, 16384 * n, 16384 * n
    return 0, 0, 0


@dataclass
class Pools:
    """Device input pools and per-op output arenas (torch tensors)."""
    i32: object
    u8: object
    f32: object
    out_add: object
    out_hist: object
    out_sum: object
    out_gemm: object
    slots: int

    @staticmethod
    def create(seed: int, i32_bytes: int = 2 << 30, u8_bytes: int = 1 << 30, f32_bytes: int = 1 << 30,
               slots: int = 4096, n_add: int = 65_536):
        import torch

        return Pools(i32=synth.device_pool("i32", i32_bytes, seed * 3 + 1),
                     u8=synth.device_pool("u8", u8_bytes, seed * 3 + 2),
                     f32=synth.device_pool("f32", f32_bytes, seed * 3 + 3),
                     out_add=torch.zeros((slots, n_add), dtype=torch.int32, device="cuda"),
                     out_hist=torch.zeros((slots, 256), dtype=torch.int32, device="cuda"),
                     out_sum=torch.zeros((slots, 4), dtype=torch.float32, device="cuda"),
                     out_gemm=torch.zeros((slots, 4096), dtype=torch.float32, device="cuda"),
                     slots=slots)


def _aligned_offsets(seed: int, key: int, count: int, span_elems: int, need: int, align: int) -> np.ndarray:
    hi = (span_elems - need) // align
    return synth.choice(seed, key, count, max(1, hi + 1)) * align


def full_chip_trace(pools: Pools, seed: int, step: int, items: int, cfg: dict = FULL_CHIP,
                    limit_bytes: int | None = None):
    """One step of the full-chip trace.  Returns (items array, meta dict).

    meta holds each item's op, input offsets (elements of its pool) and output
    slot, so that any item can be re-derived for an oracle check.  With
    `limit_bytes`, offsets stay inside the first `limit_bytes` of each pool."""
    key = 1000 * (step + 1)
    rate = cfg["rate_per_s"]
    ops = np.repeat(np.array(OPS4, dtype=np.uint32), items // 4 + 1)[:items]
    ops = ops[synth.permutation(seed, key + 1, items)]
    gaps = synth.exponential(seed, key + 2, items, 1e9 / rate)
    arrival = np.cumsum(gaps).astype(np.uint64)
    cluster = (np.arange(items) % len(cfg["sizes"])).astype(np.int32)
    n = np.zeros(items, dtype=np.uint64)
    n[ops == lk.LK_OP_ADD_I32] = cfg["n_add"]
    n[ops == lk.LK_OP_HIST_U8] = cfg["n_hist"]
    n[ops == lk.LK_OP_SUM_F32] = cfg["n_sum"]
    n[ops == lk.LK_OP_GEMM64_F32] = cfg["gemm_tiles"]
    i32_el = pools.i32.numel() if limit_bytes is None else min(pools.i32.numel(), limit_bytes // 4)
    u8_el = pools.u8.numel() if limit_bytes is None else min(pools.u8.numel(), limit_bytes)
    f32_el = pools.f32.numel() if limit_bytes is None else min(pools.f32.numel(), limit_bytes // 4)
    off0 = np.zeros(items, dtype=np.int64)
    off1 = np.zeros(items, dtype=np.int64)
    m = ops == lk.LK_OP_ADD_I32
    off0[m] = _aligned_offsets(seed, key + 3, int(m.sum()), i32_el, cfg["n_add"], 4)
    off1[m] = _aligned_offsets(seed, key + 4, int(m.sum()), i32_el, cfg["n_add"], 4)
    m = ops == lk.LK_OP_HIST_U8
    off0[m] = _aligned_offsets(seed, key + 5, int(m.sum()), u8_el, cfg["n_hist"], 16)
    m = ops == lk.LK_OP_SUM_F32
    off0[m] = _aligned_offsets(seed, key + 6, int(m.sum()), f32_el, cfg["n_sum"], 4)
    m = ops == lk.LK_OP_GEMM64_F32
    off0[m] = _aligned_offsets(seed, key + 7, int(m.sum()), f32_el, 4096 * cfg["gemm_tiles"], 4)
    off1[m] = _aligned_offsets(seed, key + 8, int(m.sum()), f32_el, 4096 * cfg["gemm_tiles"], 4)
    slot = np.zeros(items, dtype=np.int64)
    for op in OPS4:
        m = ops == op
        slot[m] = np.arange(int(m.sum())) % pools.slots

    it = np.zeros(items, dtype=lk.TRACE_ITEM_DTYPE)
    it["t_arrival_ns"] = arrival
    it["cluster"] = cluster
    it["op"] = ops
    it["n"] = n
    base = {"i32": pools.i32.data_ptr(), "u8": pools.u8.data_ptr(), "f32": pools.f32.data_ptr()}
    m = ops == lk.LK_OP_ADD_I32
    it["in0"][m] = base["i32"] + 4 * off0[m].astype(np.uint64)
    it["in1"][m] = base["i32"] + 4 * off1[m].astype(np.uint64)
    it["out"][m] = pools.out_add.data_ptr() + slot[m].astype(np.uint64) * (4 * pools.out_add.shape[1])
    m = ops == lk.LK_OP_HIST_U8
    it["in0"][m] = base["u8"] + off0[m].astype(np.uint64)
    it["out"][m] = pools.out_hist.data_ptr() + slot[m].astype(np.uint64) * 1024
    m = ops == lk.LK_OP_SUM_F32
    it["in0"][m] = base["f32"] + 4 * off0[m].astype(np.uint64)
    it["out"][m] = pools.out_sum.data_ptr() + slot[m].astype(np.uint64) * 16
    m = ops == lk.LK_OP_GEMM64_F32
    it["in0"][m] = base["f32"] + 4 * off0[m].astype(np.uint64)
    it["in1"][m] = base["f32"] + 4 * off1[m].astype(np.uint64)
    it["out"][m] = pools.out_gemm.data_ptr() + slot[m].astype(np.uint64) * 16384
    b = np.array([item_bytes(int(o), int(k)) for o, k in zip(ops, n)], dtype=np.uint64).reshape(-1, 3)
    it["in0_bytes"], it["in1_bytes"], it["out_bytes"] = b[:, 0], b[:, 1], b[:, 2]
    meta = dict(op=ops, off0=off0, off1=off1, slot=slot, n=n)
    return it, meta


def attach_host_buffers(it: np.ndarray, meta: dict, host: dict, host_out: dict) -> None:
    """E2E mode: point each item's h_in*/h_out at pinned host copies of its
    input slices (host pools hold the first bytes of the device pools) and at
    per-op pinned output buffers."""
    ops = meta["op"]
    for op in OPS4:
        m = ops == op
        if op == lk.LK_OP_ADD_I32:
            it["h_in0"][m] = host["i32"].data_ptr() + 4 * meta["off0"][m].astype(np.uint64)
            it["h_in1"][m] = host["i32"].data_ptr() + 4 * meta["off1"][m].astype(np.uint64)
            it["h_out"][m] = host_out["add"].data_ptr() + meta["slot"][m].astype(np.uint64) * (4 * host_out["add"].shape[1])
        elif op == lk.LK_OP_HIST_U8:
            it["h_in0"][m] = host["u8"].data_ptr() + meta["off0"][m].astype(np.uint64)
            it["h_out"][m] = host_out["hist"].data_ptr() + meta["slot"][m].astype(np.uint64) * 1024
        elif op == lk.LK_OP_SUM_F32:
            it["h_in0"][m] = host["f32"].data_ptr() + 4 * meta["off0"][m].astype(np.uint64)
            it["h_out"][m] = host_out["sum"].data_ptr() + meta["slot"][m].astype(np.uint64) * 16
        else:
            it["h_in0"][m] = host["f32"].data_ptr() + 4 * meta["off0"][m].astype(np.uint64)
            it["h_in1"][m] = host["f32"].data_ptr() + 4 * meta["off1"][m].astype(np.uint64)
            it["h_out"][m] = host_out["gemm"].data_ptr() + meta["slot"][m].astype(np.uint64) * 16384


def item_inputs_to_host(pools: Pools, meta: dict, i: int):
    """Copy item i's inputs back to the host (numpy) for an oracle check."""
    op = int(meta["op"][i])
    n = int(meta["n"][i])
    o0, o1 = int(meta["off0"][i]), int(meta["off1"][i])
    if op == lk.LK_OP_ADD_I32:
        return pools.i32[o0:o0 + n].cpu().numpy(), pools.i32[o1:o1 + n].cpu().numpy()
    if op == lk.LK_OP_HIST_U8:
        return (pools.u8[o0:o0 + n].cpu().numpy(),)
    if op == lk.LK_OP_SUM_F32:
        return (pools.f32[o0:o0 + n].cpu().numpy(),)
    if op == lk.LK_OP_GEMM64_F32:
        t = 4096 * n
        return (pools.f32[o0:o0 + t].cpu().numpy().reshape(n, 64, 64),
                pools.f32[o1:o1 + t].cpu().numpy().reshape(n, 64, 64))
    return ()


def item_output_to_host(pools: Pools, meta: dict, i: int):
    op = int(meta["op"][i])
    s = int(meta["slot"][i])
    n = int(meta["n"][i])
    if op == lk.LK_OP_ADD_I32:
        return pools.out_add[s, :n].cpu().numpy()
    if op == lk.LK_OP_HIST_U8:
        return pools.out_hist[s].cpu().numpy()
    if op == lk.LK_OP_SUM_F32:
        return float(pools.out_sum[s, 0].cpu())
    return pools.out_gemm[s].cpu().numpy().reshape(1, 64, 64)


def small_inputs(cfg: dict = SMALL):
    N, n = cfg["items"], cfg["n"]
    a = synth.int32_uniform(cfg["seed"], 1, N * n, cfg["lo"], cfg["hi"]).reshape(N, n)
    b = synth.int32_uniform(cfg["seed"], 2, N * n, cfg["lo"], cfg["hi"]).reshape(N, n)
    return a, b


def isolation_traces(periods: int, be_items: int, crit_in, crit_out, copy_src, copy_dst, hist_in, hist_out,
                     cfg: dict = ISOLATION, loaded: bool = True):
    """Trace of the isolation configuration: cluster 0 releases a sum every
    period (absolute release times); cluster 1 (if loaded) runs copies and
    histograms alternately, all released at time 0 (each starts when the one
    before it finished, in closed-loop mode)."""
    crit = np.zeros(periods, dtype=lk.TRACE_ITEM_DTYPE)
    crit["t_arrival_ns"] = np.arange(periods, dtype=np.uint64) * np.uint64(cfg["period_ns"])
    crit["cluster"] = 0
    crit["op"] = lk.LK_OP_SUM_F32
    crit["n"] = cfg["crit_n"]
    crit["in0"] = crit_in.data_ptr()
    crit["out"] = crit_out.data_ptr()
    if not loaded:
        return crit
    be = np.zeros(be_items, dtype=lk.TRACE_ITEM_DTYPE)
    be["cluster"] = 1
    copy = (np.arange(be_items) % 2) == 0
    be["op"] = np.where(copy, lk.LK_OP_COPY_I32, lk.LK_OP_HIST_U8)
    be["n"] = np.where(copy, copy_src.numel(), hist_in.numel())
    be["in0"] = np.where(copy, copy_src.data_ptr(), hist_in.data_ptr())
    be["out"] = np.where(copy, copy_dst.data_ptr(), hist_out.data_ptr())
    return np.concatenate([crit, be])


def batching_batch(pools: Pools, seed: int, b: int, cfg: dict = BATCHING, max_count: int | None = None):
    """Batch b of the batching stream: (BATCH_ITEM_DTYPE array, meta).  Inputs
    are slices of the pools at random 16-B-aligned offsets; add outputs land at
    random offsets of the add arena and sum outputs in slots (outputs of
    different items may overlap: this stream is for timing; parity uses
    `batching_parity_batch`)."""
    key = 50_000 + 100 * b
    count = int(synth.log_uniform_int(seed, key, 1, 1, cfg["max_count"] if max_count is None else max_count)[0])
    ops = np.where(synth.choice(seed, key + 1, count, 2) == 0, lk.LK_OP_SUM_F32, lk.LK_OP_ADD_I32).astype(np.uint32)
    n = synth.log_uniform_int(seed, key + 2, count, cfg["n_lo"], cfg["n_hi"]).astype(np.uint64)
    off0 = np.zeros(count, dtype=np.int64)
    off1 = np.zeros(count, dtype=np.int64)
    offo = np.zeros(count, dtype=np.int64)
    u0 = synth.unit_open(seed, key + 3, count)
    u1 = synth.unit_open(seed, key + 4, count)
    u2 = synth.unit_open(seed, key + 5, count)
    it = np.zeros(count, dtype=lk.BATCH_ITEM_DTYPE)
    it["op"], it["n"] = ops, n
    add_out = pools.out_add.view(-1)
    for i in range(count):
        k = int(n[i])
        if ops[i] == lk.LK_OP_ADD_I32:
            off0[i] = int(u0[i] * (pools.i32.numel() - k)) // 4 * 4
            off1[i] = int(u1[i] * (pools.i32.numel() - k)) // 4 * 4
            offo[i] = int(u2[i] * (add_out.numel() - k)) // 4 * 4
        else:
            off0[i] = int(u0[i] * (pools.f32.numel() - k)) // 4 * 4
            offo[i] = i % pools.slots
    m = ops == lk.LK_OP_ADD_I32
    it["in0"][m] = pools.i32.data_ptr() + 4 * off0[m].astype(np.uint64)
    it["in1"][m] = pools.i32.data_ptr() + 4 * off1[m].astype(np.uint64)
    it["out"][m] = add_out.data_ptr() + 4 * offo[m].astype(np.uint64)
    m = ~m
    it["in0"][m] = pools.f32.data_ptr() + 4 * off0[m].astype(np.uint64)
    it["out"][m] = pools.out_sum.data_ptr() + 16 * offo[m].astype(np.uint64)
    bytes_ = np.where(ops == lk.LK_OP_ADD_I32, 12 * n, 4 * n + 4).astype(np.float64)
    return it, dict(op=ops, n=n, off0=off0, off1=off1, offo=offo, bytes=float(bytes_.sum()))


def batching_parity_batch(pools: Pools, seed: int, count: int = 48, n_hi: int = 1 << 20):
    """A batch of the same mix whose items write disjoint outputs (add outputs
    back to back in the add arena, sums in distinct slots), for oracle checks."""
    ops = np.where(synth.choice(seed, 77_001, count, 2) == 0, lk.LK_OP_SUM_F32, lk.LK_OP_ADD_I32).astype(np.uint32)
    n = synth.log_uniform_int(seed, 77_002, count, 1024, n_hi).astype(np.uint64)
    u0 = synth.unit_open(seed, 77_003, count)
    u1 = synth.unit_open(seed, 77_004, count)
    it = np.zeros(count, dtype=lk.BATCH_ITEM_DTYPE)
    it["op"], it["n"] = ops, n
    meta = dict(op=ops, n=n, off0=np.zeros(count, np.int64), off1=np.zeros(count, np.int64),
                offo=np.zeros(count, np.int64))
    add_out = pools.out_add.view(-1)
    cursor = 0
    for i in range(count):
        k = int(n[i])
        if ops[i] == lk.LK_OP_ADD_I32:
            meta["off0"][i] = int(u0[i] * (pools.i32.numel() - k)) // 4 * 4
            meta["off1"][i] = int(u1[i] * (pools.i32.numel() - k)) // 4 * 4
            meta["offo"][i] = cursor
            cursor += (k + 3) // 4 * 4
            it[i]["in0"] = pools.i32.data_ptr() + 4 * int(meta["off0"][i])
            it[i]["in1"] = pools.i32.data_ptr() + 4 * int(meta["off1"][i])
            it[i]["out"] = add_out.data_ptr() + 4 * int(meta["offo"][i])
        else:
            meta["off0"][i] = int(u0[i] * (pools.f32.numel() - k)) // 4 * 4
            meta["offo"][i] = pools.slots - 1 - i
            it[i]["in0"] = pools.f32.data_ptr() + 4 * int(meta["off0"][i])
            it[i]["out"] = pools.out_sum.data_ptr() + 16 * int(meta["offo"][i])
    return it, meta


def serving_requests(pools: Pools, seed: int, rate: float, seconds: float, cfg: dict = SERVING,
                     s_hi: int | None = None, outputs=None):
    """Open-loop Poisson requests at `rate` per second for `seconds`; inputs are
    slices of the pools; outputs from the server's arena unless `outputs`
    (a list of device tensors, one per request) is given.  Returns the
    REQUEST_DTYPE array and the input bytes of each request."""
    key = 90_000 + int(rate)
    mean_gap = 1e9 / rate
    count = max(1, int(rate * seconds))
    t = np.cumsum(synth.exponential(seed, key, count, mean_gap)).astype(np.uint64)
    ops = np.array([lk.LK_OP_ADD_I32, lk.LK_OP_HIST_U8, lk.LK_OP_SUM_F32, lk.LK_OP_GEMM64_F32],
                   dtype=np.uint32)[synth.choice(seed, key + 1, count, 4)]
    S = synth.log_uniform_int(seed, key + 2, count, cfg["s_lo"], cfg["s_hi"] if s_hi is None else s_hi)
    n = np.where(ops == lk.LK_OP_HIST_U8, S, np.where(ops == lk.LK_OP_GEMM64_F32, np.maximum(1, S // 49152), S // 4))
    n = n.astype(np.uint64)
    u0 = synth.unit_open(seed, key + 3, count)
    u1 = synth.unit_open(seed, key + 4, count)
    r = np.zeros(count, dtype=lk.REQUEST_DTYPE)
    r["t_arrival_ns"], r["op"], r["n"] = t, ops, n
    r["producer"] = np.arange(count) % cfg["producers"]
    for i in range(count):
        k = int(n[i])
        if ops[i] == lk.LK_OP_ADD_I32:
            r[i]["in0"] = pools.i32.data_ptr() + 4 * (int(u0[i] * (pools.i32.numel() - k)) // 4 * 4)
            r[i]["in1"] = pools.i32.data_ptr() + 4 * (int(u1[i] * (pools.i32.numel() - k)) // 4 * 4)
        elif ops[i] == lk.LK_OP_HIST_U8:
            r[i]["in0"] = pools.u8.data_ptr() + int(u0[i] * (pools.u8.numel() - k)) // 16 * 16
        elif ops[i] == lk.LK_OP_SUM_F32:
            r[i]["in0"] = pools.f32.data_ptr() + 4 * (int(u0[i] * (pools.f32.numel() - k)) // 4 * 4)
        else:
            t4 = 4096 * k
            r[i]["in0"] = pools.f32.data_ptr() + 4 * (int(u0[i] * (pools.f32.numel() - t4)) // 4 * 4)
            r[i]["in1"] = pools.f32.data_ptr() + 4 * (int(u1[i] * (pools.f32.numel() - t4)) // 4 * 4)
        if outputs is not None:
            r[i]["out"] = outputs[i].data_ptr()
    in_bytes = np.where(ops == lk.LK_OP_ADD_I32, 8 * n, np.where(ops == lk.LK_OP_HIST_U8, n,
                        np.where(ops == lk.LK_OP_SUM_F32, 4 * n, 32768 * n))).astype(np.float64)
    return r, in_bytes
