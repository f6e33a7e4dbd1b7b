#!/usr/bin/env python3
"""Benchmark: submit->complete latency of persistent-thread dispatch on one GB300.

Workload (one step = 10,000 submissions): 148 SMs as 4 LightKernel clusters of
37 CTAs x 256 threads; the four work bodies in equal shares, shuffled (int32
add of 65,536 elements, histogram of 1 MiB of bytes, float32 sum of 65,536
N(0,1) values, one 64x64x64 float32 GEMM tile); Poisson arrivals at 20,000/s;
round-robin clusters; one native submitter thread per cluster.  Inputs are
slices of 4 GiB of device pools at random offsets (larger than L2).

Each step boots a context (one persistent-kernel launch), runs the step's
trace through it and disposes it.  The line reports the p99 latency over all
timed items, the same trace as ordinary cudaLaunchKernel+cudaStreamSynchronize
launches (the submitting threads of both arms pinned to the same host cores),
the host-mapped round-trip floor, the small configuration (4 SMs as 2 x 2,
closed loop), the one-deep mailbox, batching, serving, isolation and the
paper's life cycle, the work bodies' HBM bandwidth in finite mode
(roofline), an end-to-end run with host buffers, and the oracle timed on the
host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lk|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "p99/max submit→complete latency (µs) vs cudaLaunch+sync; body HBM GB/s"
WORKLOAD = ("full chip, plain: 148 SMs as 4 LK clusters of 37 (256 threads/CTA); per step 10,000 submissions "
            "mixing int32 add (65,536 el), uint8->256-bin int32 histogram (1 MiB), fp32 sum (65,536 N(0,1)), "
            "fp32 GEMM tile 64x64x64 in equal shares; Poisson arrivals at 20k/s; round-robin clusters")
ITEMS_PER_STEP = 10_000
FALLBACK_HBM = 6800.0


def pct(v, q):
    v = np.sort(np.asarray(v, dtype=np.float64))
    if v.size == 0:
        return None
    k = int(np.ceil(q * v.size))
    return float(v[max(1, min(k, v.size)) - 1])   # nearest rank


def submitter_cpus(local_rank: int, n: int = 4) -> int:
    """First of `n` consecutive host cores for the submitting threads of both
    arms (persistent kernel and ordinary launches), or -1 (not pinned) when
    this process may not use them.  Unpinned, a submitter that shares a core
    with other host work is sometimes descheduled for tens of microseconds
    while its item is in flight (measured: the device finished such items in
    7 us; the host saw 70 us)."""
    base = 2 + n * local_rank
    try:
        allowed = os.sched_getaffinity(0)
    except (AttributeError, OSError):
        return -1
    return base if set(range(base, base + n)) <= allowed else -1


def keep_off_submitter_cores(local_rank: int, n: int = 4):
    """Move this process's own threads, and every thread or process it starts
    from now on, off the cores that submitter_cpus reserves; the submitting
    threads pin themselves there.  Returns (first submitter core or -1, the
    affinity to restore for the CPU baseline, or None)."""
    base = submitter_cpus(local_rank, n)
    if base < 0:
        return -1, None
    allowed = os.sched_getaffinity(0)
    rest = allowed - set(range(base, base + n))
    if not rest:
        return base, None
    try:
        os.sched_setaffinity(0, rest)
    except OSError:
        return base, None
    return base, allowed


def lat_summary(us):
    return {"p50": pct(us, 0.50), "p99": pct(us, 0.99), "p999": pct(us, 0.999), "max": pct(us, 1.0),
            "mean": float(np.mean(us)) if len(us) else None, "count": int(len(us))}


def host_info():
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count()
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                model = line.split(":", 1)[1].strip()
    except Exception:
        pass
    return {"cores": cores, "arch": os.uname().machine, "cpu": model}


# ---- distributed plumbing (replicas; barrier and max over ranks on the host) ----
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group("gloo", rank=self.rank, world_size=self.world)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch

        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t[0])

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch

        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t[0])


# ---- clocks sampled during the timed region -----------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- oracle timing (CPU baseline and the reference arm) ---------------------------
def oracle_sample(seed: int, count: int):
    """`count` items of the workload's body mix, inputs generated on the host."""
    from paper_2310_01212_gb300 import lk, synth

    ops = [lk.LK_OP_ADD_I32, lk.LK_OP_HIST_U8, lk.LK_OP_SUM_F32, lk.LK_OP_GEMM64_F32]
    items = []
    for i in range(count):
        op = ops[i % 4]
        k = 10_000 + 10 * i
        if op == lk.LK_OP_ADD_I32:
            items.append((op, synth.int32_uniform(seed, k, 65536, -(1 << 20), 1 << 20),
                          synth.int32_uniform(seed, k + 1, 65536, -(1 << 20), 1 << 20)))
        elif op == lk.LK_OP_HIST_U8:
            items.append((op, synth.bytes_uniform(seed, k, 1 << 20)))
        elif op == lk.LK_OP_SUM_F32:
            items.append((op, synth.normal_f32(seed, k, 65536)))
        else:
            items.append((op, synth.normal_f32(seed, k, 4096).reshape(1, 64, 64),
                          synth.normal_f32(seed, k + 1, 4096).reshape(1, 64, 64)))
    return items


def time_oracle(items, budget_s: float):
    """Per-item oracle times (us), single thread, until the items or the budget run out."""
    import oracle
    from paper_2310_01212_gb300 import lk

    fns = {lk.LK_OP_ADD_I32: oracle.add_i32, lk.LK_OP_HIST_U8: oracle.hist_u8, lk.LK_OP_SUM_F32: oracle.sum_f32,
           lk.LK_OP_GEMM64_F32: oracle.gemm64_f32}
    out = []
    t_end = time.perf_counter() + budget_s
    for it in items:
        t0 = time.perf_counter_ns()
        fns[it[0]](*it[1:])
        out.append((time.perf_counter_ns() - t0) / 1000.0)
        if time.perf_counter() > t_end:
            break
    return np.array(out)


def time_oracle_pool(items, workers: int) -> float:
    """Items per second of the oracle over `items` on `workers` host threads
    (its C routines run without the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from paper_2310_01212_gb300 import lk

    fns = {lk.LK_OP_ADD_I32: oracle.add_i32, lk.LK_OP_HIST_U8: oracle.hist_u8, lk.LK_OP_SUM_F32: oracle.sum_f32,
           lk.LK_OP_GEMM64_F32: oracle.gemm64_f32}
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=workers) as ex:
        n = sum(1 for _ in ex.map(lambda it: fns[it[0]](*it[1:]), items))
    return n / (time.perf_counter() - t0)


def run_reference(args, dist: Dist):
    """The oracle, as it stands, on the host cores: same metric and workload."""
    import oracle

    oracle.build()
    if dist.rank != 0:
        return
    per_step = 200
    lat = []
    t_wall = time.perf_counter()
    for s in range(args.warmup + args.steps):
        items = oracle_sample(1000 + s, per_step)
        us = time_oracle(items, budget_s=30.0)
        if s >= args.warmup:
            lat.append(us)
    wall = time.perf_counter() - t_wall
    lat = np.concatenate(lat)
    hi = host_info()
    v = pct(lat, 0.99)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "us", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / (args.warmup + args.steps),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "binary64 accumulation (oracle)", "data": "synthetic (seeded)",
            "config": bench_config(args), "host": hi,
            "latency_us": lat_summary(lat),
            "cpu_baseline": {"value": v, "unit": "us", "cores": 1, "kind": "oracle",
                             "sample": f"{lat.size} items of the workload's body mix ({per_step} per step, "
                                       f"bodies in equal shares), per-item time, one host thread"},
            "e2e": {"value": v, "unit": "us", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def rnd1(x):
    return None if x is None else round(float(x), 1)


def bench_config(args, cfg=None) -> dict:
    """The workload as both arms report it (identical dicts)."""
    return {"workload": WORKLOAD, "partition": "4 clusters x 37 SMs", "threads_per_cta": 256,
            "items_per_step": args.items, "rate_per_s": 20000.0,
            "parallelism": f"replicas x{args.gpus} (no collective)",
            "l2": "inputs larger than L2: 4 GiB of device pools, random 16-B-aligned offsets"}


def build_headline(d: dict, hbm: float) -> dict:
    """The headline numbers of the printed line, from the detail dict (every
    value there is already a summary; nothing is recomputed)."""
    def trio(x):
        return [rnd1(x["p50"]), rnd1(x["p99"]), rnd1(x["max"])]

    nop = d["dispatch_nop_us"]
    bw = d["body_detail"]
    iso = d["isolation"]
    small = d["config_small"]
    bat = d["batching"]
    gcmp = bat["graph_compared"]
    srv = d["serving"]
    sat = max(srv["rates"].values(), key=lambda e: e["throughput_gbs"])
    hd = srv["host_dispatcher"]["rates"]
    sat_h = max(hd.values(), key=lambda e: e["throughput_gbs"]) if hd else None
    hc = srv["host_dispatcher_coalesced"]["rates"]
    sat_c = max(hc.values(), key=lambda e: e["throughput_gbs"]) if hc else None
    low = srv["rates"][min(srv["rates"], key=int)]
    return {
        "lk_us_p50_p99_max": trio(d["latency_us"]),
        "launch_sync_us_p50_p99_max": trio(d["baseline_launch_sync_us"]),
        "occupancy_grid_us_p50_p99_max": trio(d["baseline_occupancy_grid_us"]),
        "arrival_to_complete_us_p50_p99_max": trio(d["arrival_to_complete_us"]),
        "by_op_us_p50_p99_max": {k: {"lk": v["lk"], "launch_sync": v["launch_sync"]}
                                 for k, v in d.get("latency_by_op_us_p50_p99_max", {}).items()},
        "floor_p50_us": rnd1(d["pingpong_floor_us"]["p50"]),
        "nop_p50_us": {"relay": rnd1(nop["lk"]["p50"]), "direct": rnd1(nop["lk_direct"]["p50"]),
                       "mailbox": rnd1(nop["lk_mailbox"]["p50"]), "launch_sync": rnd1(nop["launch_sync"]["p50"]),
                       "ring_1sm": rnd1(d["paper_mailbox_vs_ring"]["ring_1sm_nop_us"]["p50"])},
        "floor_over_nop_p50": round(d["pingpong_floor_us"]["p50"] / nop["lk"]["p50"], 3),
        "nop_device_p50_us": {k[:-3]: rnd1(v["p50"]) for k, v in nop["lk_device_phases"].items()
                              if k.endswith("_us") and "p50" in v},
        "tail": {"lk_max_item": d["tail_attribution"]["lk_top10"][0],
                 "lk_device_pick_to_done_max_us": rnd1(d["tail_attribution"]["lk_device_pick_to_done_us"]["max"]),
                 "items_over_25us_lk_vs_launch_sync": [d["tail_attribution"]["lk_items_over_25us"],
                                                       d["tail_attribution"]["launch_sync_items_over_25us"]]},
        "small_us_p99_max": {"lk": [rnd1(small["lk_us"]["p99"]), rnd1(small["lk_us"]["max"])],
                             "launch_sync": [rnd1(small["launch_sync_us"]["p99"]),
                                             rnd1(small["launch_sync_us"]["max"])],
                             "bit_exact": small["bit_exact"]},
        "body_gbs": {k: round(v["gbs"]) for k, v in bw.items()},
        "body_frac_of_measured_hbm": {k: round(v["gbs"] / hbm, 3) for k, v in bw.items()},
        "isolation": {"periods": iso["periods"], "alone_p999_us": rnd1(iso["alone_us"]["p999"]),
                      "loaded_p999_us": rnd1(iso["loaded_us"]["p999"]),
                      "inflation_p999": round(iso["inflation_p999"], 2),
                      "inflation_max": round(iso["inflation_max"], 2),
                      "cap_2tbs_inflation_p999": round(iso["best_effort_rate_cap_gbs"]["2000"]["inflation_p999"], 2),
                      "yield": {"inflation_p999": round(iso["best_effort_yield"]["inflation_p999"], 2),
                                "best_effort_gbs": round(iso["best_effort_yield"]["best_effort_gbs"]),
                                "unyielded_best_effort_gbs": round(iso["best_effort_gbs"])}},
        "batching_gbs": {"lk_prefix": round(bat["lk_gbs"]), "prefix_items": bat["items"],
                         "lk_vs_graph": [round(gcmp["lk_gbs"]), round(gcmp["graph_gbs"])]},
        "serving_saturation_gbs": {"device_queue": round(sat["throughput_gbs"]),
                                   "host_dispatcher": round(sat_h["throughput_gbs"]) if sat_h else None,
                                   "host_coalesced": round(sat_c["throughput_gbs"]) if sat_c else None,
                                   "device_queue_hbm_traffic_frac": round(sat["traffic_gbs"] / hbm, 3)},
        "serving_lowest_rate_us_p50_p99": [rnd1(low["latency_us"]["p50"]), rnd1(low["latency_us"]["p99"])],
        "parity": {"sampled_items_bad": d["parity"]["mismatches"],
                   "exec_log_violations": d["parity"]["exec_log"]["violations"],
                   "body_checks_bad": sum(v["parity"]["mismatches"] for v in bw.values()),
                   "batching_bad": bat["parity_mismatches"], "small_exact": small["bit_exact"]},
    }


def item_device_us(items, log) -> np.ndarray:
    """Device-side pick -> done (us) of each trace item, from one context's
    execution log.  Each cluster's items were posted by one thread in
    arrival order, so the k-th item of cluster c is its descriptor seq k+1."""
    out = np.full(items.size, np.nan)
    key = log["cluster"].astype(np.int64) << 40 | log["seq"].astype(np.int64)
    last = log["t_done_ns"] > 0
    # first pickup of each descriptor (the master's, when it relays)
    uk, inv = np.unique(key, return_inverse=True)
    first = np.full(uk.size, np.iinfo(np.int64).max, np.int64)
    np.minimum.at(first, inv, log["t_pick_ns"].astype(np.int64))
    dmap = dict(zip(key[last].tolist(), (log["t_done_ns"][last].astype(np.int64) - first[inv[last]]).tolist()))
    for c in np.unique(items["cluster"]):
        idx = np.nonzero(items["cluster"] == c)[0]
        idx = idx[np.argsort(items["t_arrival_ns"][idx], kind="stable")]
        for k, i in enumerate(idx):
            v = dmap.get(int(c) << 40 | (k + 1))
            if v is not None:
                out[i] = v / 1000.0
    return out


def e2e_parts(res) -> dict:
    """Split end-to-end trace latencies into copy in / dispatch / copy out."""
    cin = (res["t_post_ns"].astype(np.int64) - res["t_submit_ns"].astype(np.int64)) / 1000.0
    dis = (res["t_observed_ns"].astype(np.int64) - res["t_post_ns"].astype(np.int64)) / 1000.0
    cout = (res["t_complete_ns"].astype(np.int64) - res["t_observed_ns"].astype(np.int64)) / 1000.0
    tot = (res["t_complete_ns"].astype(np.int64) - res["t_submit_ns"].astype(np.int64)) / 1000.0
    top = np.argsort(tot)[::-1][: max(1, tot.size // 100)]   # the slowest 1 %: where their time went
    # when the slow copies happen: submit time (ms into the trace) and worker
    # thread of the 12 slowest copies, to tell a periodic host event from a
    # steady rate
    slow = np.argsort(np.maximum(cin, cout))[::-1][:12]
    return {"copy_in": lat_summary(cin), "dispatch": lat_summary(dis), "copy_out": lat_summary(cout),
            "slowest_1pct_mean": {"copy_in": float(np.mean(cin[top])), "dispatch": float(np.mean(dis[top])),
                                  "copy_out": float(np.mean(cout[top]))},
            "slowest_copies": [[round(float(res["t_submit_ns"][i]) / 1e6, 3), int(res["thread"][i]),
                                round(float(cin[i]), 1), round(float(cout[i]), 1)] for i in slow]}


def exec_log_phases(log) -> dict:
    """Per descriptor, from one context's execution log (device %globaltimer,
    32 ns ticks): pick -> last CTA start (relay), last start -> last end
    (body), last end -> completion stamp of the last CTA to arrive; medians
    and p99 in us over the descriptors."""
    key = log["cluster"].astype(np.int64) << 40 | log["seq"].astype(np.int64)
    uk, inv = np.unique(key, return_inverse=True)
    pick = np.full(uk.size, np.iinfo(np.int64).max, np.int64)
    start = np.zeros(uk.size, np.int64)
    end = np.zeros(uk.size, np.int64)
    done = np.zeros(uk.size, np.int64)
    # the descriptor's first pickup (the master's, when it relays)
    np.minimum.at(pick, inv, log["t_pick_ns"].astype(np.int64))
    np.maximum.at(start, inv, log["t_start_ns"].astype(np.int64))
    np.maximum.at(end, inv, log["t_end_ns"].astype(np.int64))
    np.maximum.at(done, inv, log["t_done_ns"].astype(np.int64))
    ok = done > 0
    out = {"descriptors": int(ok.sum())}
    for name, v in (("pick_to_last_start", start - pick), ("last_start_to_last_end", end - start),
                    ("last_end_to_done", done - end), ("pick_to_done", done - pick)):
        v = v[ok] / 1000.0
        out[name + "_us"] = {"p50": pct(v, 0.5), "p99": pct(v, 0.99)}
    # per CTA: median of its own pickup - the descriptor's first pickup
    # (how late each CTA sees the relay, or the host's post with LK_INIT_DIRECT)
    rk = log["cluster"].astype(np.int64) << 20 | log["rank"].astype(np.int64)
    per = {}
    d = (log["t_pick_ns"].astype(np.int64) - pick[inv]) / 1000.0
    for key in np.unique(rk):
        m = rk == key
        per[int(key)] = (float(np.median(d[m])), int(log["smid"][m][0]), int(key & 0xfffff))
    meds = np.array([v[0] for v in per.values()])
    worst = sorted(per.values(), reverse=True)[:5]
    out["per_cta_first_pick_to_own_pick_us"] = {"min": float(meds.min()), "p50": float(np.median(meds)),
                                       "max": float(meds.max()),
                                       "worst5_us_smid_rank": [[round(a, 3), b, c] for a, b, c in worst]}
    return out


# ---- oracle checks of the bench's outputs (checking code stays out of the package) ----
def check_batching_parity(pools, meta: dict) -> int:
    """Number of items of a batching parity batch whose output differs from
    the oracle (int32 adds bit-exact, sums within 1e-4 sum|x|)."""
    import oracle
    from paper_2310_01212_gb300 import lk

    bad = 0
    add_out = pools.out_add.view(-1)
    for i in range(meta["op"].size):
        k = int(meta["n"][i])
        if meta["op"][i] == lk.LK_OP_ADD_I32:
            a = pools.i32[int(meta["off0"][i]):int(meta["off0"][i]) + k].cpu().numpy()
            b = pools.i32[int(meta["off1"][i]):int(meta["off1"][i]) + k].cpu().numpy()
            o = add_out[int(meta["offo"][i]):int(meta["offo"][i]) + k].cpu().numpy()
            bad += 0 if np.array_equal(o, oracle.add_i32(a, b)) else 1
        else:
            x = pools.f32[int(meta["off0"][i]):int(meta["off0"][i]) + k].cpu().numpy()
            o = float(pools.out_sum[int(meta["offo"][i]), 0].cpu())
            bad += 0 if abs(o - oracle.sum_f32(x)) <= 1e-4 * oracle.abs_sum_f32(x) else 1
    return bad


# ---- the LightKernel arm ------------------------------------------------------------
def kernel_source_sha() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2310_01212_gb300", "csrc")
    for f in ("lk_kernel.cu", "lk_bodies.cuh", "lk_device.cuh", "lk_layout.h"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(name: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the kernel source as it is now (else None)."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha") != kernel_source_sha():
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": FALLBACK_HBM}, "fallback"


def check_body_output(name: str, op: int, cnt: int, a, b, o, seed: int) -> dict:
    """Compare the output of a finite-mode bandwidth launch with the oracle at
    the size it was timed: add / copy on seeded 1M-element windows at random
    offsets, the sum and the histogram whole, a seeded 1 % of the GEMM tiles.
    Returns {"checked": what, "mismatches": k}."""
    import oracle
    from paper_2310_01212_gb300 import lk, synth

    win = 1 << 20
    if op in (lk.LK_OP_ADD_I32, lk.LK_OP_COPY_I32):
        starts = synth.choice(seed, 31, 4, (cnt - win) // 4 + 1) * 4
        bad = 0
        for st in starts:
            st = int(st)
            x = a[st:st + win].cpu().numpy()
            want = oracle.add_i32(x, b[st:st + win].cpu().numpy()) if op == lk.LK_OP_ADD_I32 else oracle.copy_i32(x)
            bad += int(np.count_nonzero(o[st:st + win].cpu().numpy() != want))
        return {"checked": f"{len(starts)} windows of {win} elements at seeded offsets", "mismatches": bad}
    if op == lk.LK_OP_SUM_F32:
        x = a.cpu().numpy()
        ok = abs(float(o[0].cpu()) - oracle.sum_f32(x)) <= 1e-4 * oracle.abs_sum_f32(x)
        return {"checked": f"the whole sum of {cnt} values", "mismatches": 0 if ok else 1}
    if op == lk.LK_OP_HIST_U8:
        ok = np.array_equal(o.cpu().numpy().astype(np.int64), oracle.hist_u8(a.cpu().numpy()))
        return {"checked": f"the whole histogram of {cnt} bytes", "mismatches": 0 if ok else 1}
    pick = np.sort(synth.choice(seed, 32, max(1, cnt // 100), cnt))
    A = a.view(cnt, 64, 64)[torch_index(pick, a)].cpu().numpy()
    B = b.view(cnt, 64, 64)[torch_index(pick, b)].cpu().numpy()
    C = o.view(cnt, 64, 64)[torch_index(pick, o)].cpu().numpy()
    err = np.abs(C.astype(np.float64) - oracle.gemm64_f32(A, B)) > 1e-4 * oracle.gemm64_abs_bound(A, B)
    bad = int(np.count_nonzero(err.reshape(len(pick), -1).any(axis=1)))
    return {"checked": f"{len(pick)} of {cnt} tiles (seeded 1 %), every element", "mismatches": bad}


def torch_index(idx: np.ndarray, like):
    import torch

    return torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int64)).to(like.device)


def body_bandwidth(pools, lk, n_sms: int, reps: int = 5, per_launch: int = 3, threads: int = 256,
                   seed: int = 0):
    """Finite mode on every SM as one cluster: `per_launch` descriptors of one
    body per launch; CUDA-event time of each launch (boot included).  After
    each body's launches its output is checked against the oracle at the
    timed size (check_body_output); a mismatch fails the leg."""
    import torch

    i32, u8, f32 = pools.i32, pools.u8, pools.f32
    n = 1 << 28
    out = pools.out_add.view(-1)[:n]
    half = f32.numel() // 2
    tiles = half // 4096
    cases = {
        "add_i32": (lk.LK_OP_ADD_I32, n, i32[:n], i32[n:2 * n], out, 12 * n),
        "copy_i32": (lk.LK_OP_COPY_I32, n, i32[:n], None, out, 8 * n),
        "sum_f32": (lk.LK_OP_SUM_F32, n, f32[:n], None, pools.out_sum[0], 4 * n + 4),
        "hist_u8": (lk.LK_OP_HIST_U8, u8.numel(), u8, None, pools.out_hist[0], u8.numel() + 1024),
        "gemm64_f32": (lk.LK_OP_GEMM64_F32, tiles, f32[:half], f32[half:2 * half],
                       pools.out_add.view(torch.float32).view(-1)[:half], 3 * half * 4),
    }
    # the block size is a context parameter: the histogram, bound by shared-
    # memory reductions, is also timed at 512 threads per CTA
    runs = [(name, case, threads, 0) for name, case in cases.items()]
    runs.append(("hist_u8_512_threads", cases["hist_u8"], 512, 0))
    # the float32 FFMA path of the GEMM tile (what split row blocks and two
    # CTAs per SM run), at the same size
    runs.append(("gemm64_f32_ffma", cases["gemm64_f32"], threads, lk.LK_INIT_GEMM_FFMA))
    res = {}
    for name, (op, cnt, a, b, o, nbytes), t_cta, fl in runs:
        ms = []
        for _ in range(reps):
            t, _log = lk.lk_run_finite([n_sms], [(op, cnt)] * per_launch, [0] * per_launch,
                                       in0=[a] * per_launch, in1=[b] * per_launch if b is not None else None,
                                       out=[o] * per_launch, threads_per_cta=t_cta, exec_log_cap=per_launch + 1,
                                       flags=fl)
            ms.append(t)
        avg = float(np.mean(ms))
        torch.cuda.synchronize()
        chk = check_body_output(name, op, cnt, a, b, o, seed)
        if chk["mismatches"]:
            raise RuntimeError(f"body bandwidth leg {name}: {chk['mismatches']} mismatches against the oracle")
        res[name] = {"gbs": nbytes * per_launch / (avg * 1e-3) / 1e9, "launch_ms": avg, "bytes_per_launch":
                     nbytes * per_launch, "descriptors_per_launch": per_launch, "threads_per_cta": t_cta,
                     "parity": chk, "flags": fl}
        if op == lk.LK_OP_GEMM64_F32:
            res[name]["tflops"] = 524288.0 * cnt * per_launch / (avg * 1e-3) / 1e12
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lk", choices=["lk", "reference"])
    ap.add_argument("--items", type=int, default=ITEMS_PER_STEP)
    ap.add_argument("--iso-periods", type=int, default=60_000,
                    help="critical periods (1 ms each) of the disjoint-layout isolation run: alone, loaded, "
                         "and loaded with the best effort yielding")
    ap.add_argument("--iso-sweep-periods", type=int, default=2000,
                    help="critical periods of each co-resident and rate-capped isolation run")
    ap.add_argument("--batch-items", type=int, default=1_000_000,
                    help="descriptors of the batching stream to run (whole batches; 1,000,000 = the whole "
                         "stream, about 13.8 TB)")
    ap.add_argument("--graph-batches", type=int, default=8,
                    help="batches of that prefix also timed as CUDA graphs of ordinary launches")
    ap.add_argument("--detail", default="bench_detail.json",
                    help="file that receives every leg's full result (the printed line keeps the headline)")
    ap.add_argument("--serve-seconds", type=float, default=0.25, help="seconds of arrivals per serving rate")
    ap.add_argument("--phase-runs", type=int, default=100, help="runs of the paper's life-cycle measurement")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    full_mask = None
    if args.impl != "reference":
        # before torch and the CUDA driver start their threads
        pin, full_mask = keep_off_submitter_cores(int(os.environ.get("LOCAL_RANK", "0")))
    dist = Dist()
    if args.impl == "reference":
        run_reference(args, dist)
        return

    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2310_01212_gb300 import lk, synth, workloads as wl
    import oracle

    torch.cuda.set_device(dist.local)
    dev = torch.cuda.current_device()
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    cfg = dict(wl.FULL_CHIP)
    seed = cfg["seed"] + 7919 * dist.rank
    items_per_step = args.items

    # dispatch floor (no context alive)
    rtt = lk.lk_pingpong(20_000, device=dev)[1000:] / 1000.0

    pools = wl.Pools.create(seed)
    traces = [wl.full_chip_trace(pools, seed, s, items_per_step, cfg) for s in range(args.warmup + args.steps)]
    torch.cuda.synchronize()

    # ---- timed region: K steps of (boot, trace, dispose) ---------------------------
    sizes = cfg["sizes"]
    lat, lat_arr, kernel_ms, dev_us, sub_ms, step_of = [], [], [], [], [], []
    clocks = ClockSampler(dev)
    log_verdict = None
    for s in range(args.warmup + args.steps):
        if s == args.warmup:
            torch.cuda.synchronize()
            dist.barrier()
            clocks.start()
            t_timed = time.perf_counter()
        timed = s >= args.warmup
        last = s == args.warmup + args.steps - 1
        ctx = lk.lk_init(sizes, device=dev, threads_per_cta=cfg["threads"], exec_log_cap=4096,
                         idle_lease_ns=5_000_000_000)
        rc, res = lk.lk_run_trace(ctx, traces[s][0], n_threads=len(sizes), pin_cpu_base=pin)
        if rc != lk.LK_OK:
            raise RuntimeError(f"trace failed: {lk.lk_strerror(rc)}")
        # the device's own pick -> done of every item (execution log; read
        # after the trace, while the context idles)
        log, dropped = lk.lk_exec_log(ctx)
        if timed:
            dev_us.append(item_device_us(traces[s][0], log))
        if last:
            last_res = res
            ops = traces[s][1]["op"]
            n_posted = [int(np.sum(np.arange(items_per_step) % 4 == c)) for c in range(4)]
            posted_op = np.concatenate([ops[np.arange(items_per_step) % 4 == c] for c in range(4)])
            pinned = sum((lk.lk_cluster_info(ctx, c) for c in range(4)), [])
            log_verdict = oracle.check_exec_log(log["seq"], log["cluster"], log["rank"], log["smid"], log["op"],
                                                log["order"], sizes, n_posted, pinned_smid=pinned,
                                                posted_op=posted_op)
            log_verdict["dropped"] = int(dropped)
        ctx.dispose()
        if timed:
            lat.append((res["t_complete_ns"] - res["t_submit_ns"]) / 1000.0)
            sub_ms.append(res["t_submit_ns"] / 1e6)
            step_of.append(np.full(res.size, s - args.warmup))
            lat_arr.append((res["t_complete_ns"] - traces[s][0]["t_arrival_ns"]) / 1000.0)
            kernel_ms.append(ctx.kernel_ms)
    torch.cuda.synchronize()
    dist.barrier()
    wall = time.perf_counter() - t_timed
    lat = np.concatenate(lat)
    lat_arr = np.concatenate(lat_arr)
    dev_us = np.concatenate(dev_us)
    sub_ms = np.concatenate(sub_ms)
    step_of = np.concatenate(step_of)
    op_all = np.concatenate([traces[s][0]["op"] for s in range(args.warmup, args.warmup + args.steps)])

    # ---- parity: a seeded sample of the last step's items against the oracle -------
    it, meta = traces[-1]
    pick = synth.choice(seed, 99, 64, items_per_step)
    bad = 0
    for i in pick:
        op = int(meta["op"][i])
        ins = wl.item_inputs_to_host(pools, meta, int(i))
        got = wl.item_output_to_host(pools, meta, int(i))
        if op == lk.LK_OP_ADD_I32:
            ok = np.array_equal(got, oracle.add_i32(*ins))
        elif op == lk.LK_OP_HIST_U8:
            ok = np.array_equal(got.astype(np.int64), oracle.hist_u8(*ins))
        elif op == lk.LK_OP_SUM_F32:
            ok = abs(got - oracle.sum_f32(*ins)) <= 1e-4 * oracle.abs_sum_f32(*ins)
        else:
            ok = bool(np.all(np.abs(got.astype(np.float64) - oracle.gemm64_f32(*ins))
                             <= 1e-4 * oracle.gemm64_abs_bound(*ins)))
        bad += 0 if ok else 1

    # ---- the same timed traces as ordinary launches ---------------------------------
    base = []
    for s in range(args.warmup, args.warmup + args.steps):
        rc, res = lk.lk_baseline_run_trace(traces[s][0], [sz for sz in sizes], threads=cfg["threads"],
                                           n_threads=len(sizes), device=dev, pin_cpu_base=pin)
        if rc != lk.LK_OK:
            raise RuntimeError(f"baseline failed: {lk.lk_strerror(rc)}")
        base.append((res["t_complete_ns"] - res["t_submit_ns"]) / 1000.0)
    base = np.concatenate(base)
    # per body: which op sets the p99 (the device's own pick -> done beside it)
    by_op = {}
    for o in np.unique(op_all):
        m = op_all == o
        dv = dev_us[m][np.isfinite(dev_us[m])]
        by_op[lk.OP_NAMES.get(int(o), str(int(o)))] = {
            "lk": [rnd1(np.percentile(lat[m], q)) for q in (50, 99)] + [rnd1(lat[m].max())],
            "launch_sync": [rnd1(np.percentile(base[m], q)) for q in (50, 99)] + [rnd1(base[m].max())],
            "device_pick_to_done": [rnd1(np.percentile(dv, q)) for q in (50, 99)] if dv.size else None}
    top_lk = np.argsort(lat)[::-1][:10]
    top_base = np.argsort(base)[::-1][:10]
    nan2none = lambda x: None if not np.isfinite(x) else round(float(x), 2)
    tail = {"lk_top10": [{"us": round(float(lat[i]), 2), "device_pick_to_done_us": nan2none(dev_us[i]),
                          "op": lk.OP_NAMES.get(int(op_all[i]), str(int(op_all[i]))),
                          "step": int(step_of[i]), "submit_ms": round(float(sub_ms[i]), 3)} for i in top_lk],
            "launch_sync_top10": [{"us": round(float(base[i]), 2),
                                   "op": lk.OP_NAMES.get(int(op_all[i]), str(int(op_all[i])))} for i in top_base],
            "lk_items_over_25us": int(np.sum(lat > 25.0)), "launch_sync_items_over_25us": int(np.sum(base > 25.0)),
            "lk_device_pick_to_done_us": lat_summary(dev_us[np.isfinite(dev_us)]),
            "lk_items_without_device_stamp": int(np.sum(~np.isfinite(dev_us))),
            "note": "device pick->done from the execution log (%globaltimer); the rest of an item's latency is "
                    "host-side: posting, the descriptor's trip over the host link, completion observed"}
    # the occupancy-chosen grid: what an ordinary launch of the body picks on
    # its own (one CTA per SM at this shared-memory size, so every SM), for the
    # last timed step's trace
    occ_grid = n_sms
    rc, res = lk.lk_baseline_run_trace(traces[-1][0], [occ_grid] * len(sizes), threads=cfg["threads"],
                                       n_threads=len(sizes), device=dev, pin_cpu_base=pin)
    if rc != lk.LK_OK:
        raise RuntimeError(f"occupancy-grid baseline failed: {lk.lk_strerror(rc)}")
    base_occ = (res["t_complete_ns"] - res["t_submit_ns"]) / 1000.0
    # the clock sampler (nvidia-smi, every 200 ms) ran through both arms, so
    # that any disturbance it causes falls on both alike
    clk = clocks.stop()

    # ---- dispatch alone: closed-loop NOPs, persistent kernel vs launch+sync ---------
    nop = np.zeros(2 * items_per_step, dtype=lk.TRACE_ITEM_DTYPE)
    nop["cluster"] = np.arange(nop.size) % 4
    nop["op"] = lk.LK_OP_NOP
    with lk.lk_init(sizes, device=dev, idle_lease_ns=5_000_000_000,
                    exec_log_cap=nop.size // len(sizes) + 64) as ctx:
        rc, r1 = lk.lk_run_trace(ctx, nop, n_threads=1, closed_loop=True, pin_cpu_base=pin)
        nop_phases = exec_log_phases(lk.lk_exec_log(ctx)[0])
    with lk.lk_init(sizes, device=dev, idle_lease_ns=5_000_000_000, flags=lk.LK_INIT_DIRECT,
                    exec_log_cap=nop.size // len(sizes) + 64) as ctx:
        rc, r3 = lk.lk_run_trace(ctx, nop, n_threads=1, closed_loop=True, pin_cpu_base=pin)
        nop_phases_direct = exec_log_phases(lk.lk_exec_log(ctx)[0])
    with lk.lk_init(sizes, device=dev, idle_lease_ns=5_000_000_000, flags=lk.LK_INIT_MAILBOX) as ctx:
        rc, r4 = lk.lk_run_trace(ctx, nop, n_threads=1, closed_loop=True, pin_cpu_base=pin)
    rc2, r2 = lk.lk_baseline_run_trace(nop, sizes, threads=cfg["threads"], n_threads=1, device=dev, pin_cpu_base=pin)
    skip = nop.size // 20   # first items warm the path
    nop_lk = (r1["t_complete_ns"] - r1["t_submit_ns"])[skip:] / 1000.0
    nop_direct = (r3["t_complete_ns"] - r3["t_submit_ns"])[skip:] / 1000.0
    nop_mbox = (r4["t_complete_ns"] - r4["t_submit_ns"])[skip:] / 1000.0
    nop_base = (r2["t_complete_ns"] - r2["t_submit_ns"])[skip:] / 1000.0

    # ---- the small configuration: 4 SMs as 2 clusters of 2, closed loop -----------
    # 10,000 int32 adds of 4,096 elements, round-robin, one outstanding at a
    # time; the same items as launch+sync of 2 CTAs each; outputs checked
    scfg = wl.SMALL
    sa, sb = wl.small_inputs(scfg)
    n_small, n_el = sa.shape
    dsa, dsb = torch.from_numpy(sa).to(dev), torch.from_numpy(sb).to(dev)
    sout = torch.zeros((n_small, n_el), dtype=torch.int32, device=dev)
    sit = np.zeros(n_small, dtype=lk.TRACE_ITEM_DTYPE)
    sit["cluster"] = np.arange(n_small) % len(scfg["sizes"])
    sit["op"] = lk.LK_OP_ADD_I32
    sit["n"] = n_el
    row = np.arange(n_small, dtype=np.uint64) * np.uint64(4 * n_el)
    sit["in0"], sit["in1"], sit["out"] = dsa.data_ptr() + row, dsb.data_ptr() + row, sout.data_ptr() + row
    torch.cuda.synchronize()
    with lk.lk_init(scfg["sizes"], device=dev, threads_per_cta=scfg["threads"], idle_lease_ns=5_000_000_000) as ctx:
        rc, rs = lk.lk_run_trace(ctx, sit, n_threads=1, closed_loop=True, pin_cpu_base=pin)
    if rc != lk.LK_OK:
        raise RuntimeError(f"small-config trace failed: {lk.lk_strerror(rc)}")
    small_exact = bool(np.array_equal(sout.cpu().numpy(), oracle.add_i32(sa, sb)))
    rc, rsb = lk.lk_baseline_run_trace(sit, scfg["sizes"], threads=scfg["threads"], n_threads=1, device=dev,
                                       pin_cpu_base=pin)
    if rc != lk.LK_OK:
        raise RuntimeError(f"small-config baseline failed: {lk.lk_strerror(rc)}")
    small = {"workload": "4 SMs as 2 LK clusters of 2 (256 threads/CTA); 10,000 closed-loop int32 adds of 4,096 "
                         "elements uniform in [-2^20, 2^20], seed 0, round-robin",
             "lk_us": lat_summary((rs["t_complete_ns"] - rs["t_submit_ns"]) / 1000.0),
             "launch_sync_us": lat_summary((rsb["t_complete_ns"] - rsb["t_submit_ns"]) / 1000.0),
             "bit_exact": small_exact}
    del dsa, dsb, sout

    # ---- the paper's one-deep mailbox against the ring (Sec. II.D, Table 1) ---------
    # one SM (the paper's cluster), closed-loop NOPs; then the last timed step's
    # mixed trace (open loop, Poisson arrivals) through one-deep mailboxes
    mbox = {}
    nop1 = nop[: nop.size // 2].copy()
    nop1["cluster"] = 0
    for key, fl in (("ring_1sm", 0), ("mailbox_1sm", lk.LK_INIT_MAILBOX)):
        with lk.lk_init([1], device=dev, idle_lease_ns=5_000_000_000, flags=fl) as ctx:
            rc, r = lk.lk_run_trace(ctx, nop1, n_threads=1, closed_loop=True, pin_cpu_base=pin)
        if rc != lk.LK_OK:
            raise RuntimeError(f"1-SM NOP trace failed: {lk.lk_strerror(rc)}")
        mbox[key + "_nop_us"] = lat_summary((r["t_complete_ns"] - r["t_submit_ns"])[skip // 2:] / 1000.0)
    last_trace = traces[-1][0]
    with lk.lk_init(sizes, device=dev, threads_per_cta=cfg["threads"], idle_lease_ns=5_000_000_000,
                    flags=lk.LK_INIT_MAILBOX) as ctx:
        rc, r = lk.lk_run_trace(ctx, last_trace, n_threads=len(sizes), pin_cpu_base=pin)
    if rc != lk.LK_OK:
        raise RuntimeError(f"mailbox trace failed: {lk.lk_strerror(rc)}")
    mbox["mixed_trace_mailbox"] = {
        "submit_to_complete_us": lat_summary((r["t_complete_ns"] - r["t_submit_ns"]) / 1000.0),
        "arrival_to_complete_us": lat_summary((r["t_complete_ns"] - last_trace["t_arrival_ns"]) / 1000.0)}
    mbox["mixed_trace_ring_last_step"] = {
        "submit_to_complete_us": lat_summary((last_res["t_complete_ns"] - last_res["t_submit_ns"]) / 1000.0),
        "arrival_to_complete_us": lat_summary((last_res["t_complete_ns"] - last_trace["t_arrival_ns"]) / 1000.0)}

    # ---- end to end: host buffers, copies inside the timed path ---------------------
    lim = 256 << 20
    host = {"i32": pools.i32[: lim // 4].cpu().pin_memory(), "u8": pools.u8[:lim].cpu().pin_memory(),
            "f32": pools.f32[: lim // 4].cpu().pin_memory()}
    host_out = {"add": torch.zeros((pools.slots, cfg["n_add"]), dtype=torch.int32).pin_memory(),
                "hist": torch.zeros((pools.slots, 256), dtype=torch.int32).pin_memory(),
                "sum": torch.zeros((pools.slots, 4), dtype=torch.float32).pin_memory(),
                "gemm": torch.zeros((pools.slots, 4096), dtype=torch.float32).pin_memory()}
    e2e_it, e2e_meta = wl.full_chip_trace(pools, seed, 777, items_per_step, cfg, limit_bytes=lim)
    wl.attach_host_buffers(e2e_it, e2e_meta, host, host_out)
    torch.cuda.synchronize()
    with lk.lk_init(sizes, device=dev, idle_lease_ns=5_000_000_000) as ctx:
        rc, re = lk.lk_run_trace(ctx, e2e_it, n_threads=len(sizes), mode=lk.LK_TRACE_E2E, pin_cpu_base=pin)
    if rc != lk.LK_OK:
        raise RuntimeError(f"e2e trace failed: {lk.lk_strerror(rc)}")
    e2e = (re["t_complete_ns"] - re["t_submit_ns"]) / 1000.0
    rc, rb = lk.lk_baseline_run_trace(e2e_it, sizes, threads=cfg["threads"], n_threads=len(sizes), device=dev,
                                      mode=lk.LK_TRACE_E2E, pin_cpu_base=pin)
    e2e_base = (rb["t_complete_ns"] - rb["t_submit_ns"]) / 1000.0
    h2d = int(e2e_it["in0_bytes"].sum() + e2e_it["in1_bytes"].sum())
    d2h = int(e2e_it["out_bytes"].sum())

    # ---- batching: one post per batch vs one CUDA graph of ordinary launches -------
    from paper_2310_01212_gb300 import autotune

    tuned = autotune.load()
    # a seeded prefix of the 1,000,000-descriptor stream: whole batches until
    # at least --batch-items descriptors
    bbat = []
    while sum(len(it) for it, _ in bbat) < args.batch_items:
        bbat.append(wl.batching_batch(pools, seed, len(bbat)))
    gsub = bbat[: max(1, min(args.graph_batches, len(bbat)))]
    par_items, par_meta = wl.batching_parity_batch(pools, seed)
    torch.cuda.synchronize()
    lk_sub_s = []
    tune_kw = dict(max_parts=tuned["max_parts"], part_bytes=tuned["part_bytes"])
    with lk.lk_init([n_sms], device=dev, threads_per_cta=tuned["threads"], max_batch_units=1 << 16,
                    idle_lease_ns=30_000_000_000) as ctx:
        h = lk.lk_submit_batch(ctx, 0, par_items, **tune_kw)
        if lk.lk_wait(ctx, h, 60_000_000_000) != lk.LK_OK:
            raise RuntimeError("parity batch did not finish")
        # check now: the timed batches below write into the same output arenas
        torch.cuda.current_stream().synchronize()
        batch_bad = check_batching_parity(pools, par_meta)
        # the graph-compared subset, one batch at a time (post, wait)
        for items, _ in gsub:
            t0 = time.perf_counter_ns()
            h = lk.lk_submit_batch(ctx, 0, items, **tune_kw)
            if h is None or lk.lk_wait(ctx, h, 120_000_000_000) != lk.LK_OK:
                raise RuntimeError("batch did not finish")
            lk_sub_s.append((time.perf_counter_ns() - t0) / 1e9)
        # the whole prefix: batch b+1 is posted while batch b runs (two unit
        # tables per cluster), then b is waited for
        t0 = time.perf_counter_ns()
        prev = None
        for items, _ in bbat:
            h = lk.lk_submit_batch(ctx, 0, items, **tune_kw)
            if h is None:
                raise RuntimeError("batch tables busy")
            if prev is not None and lk.lk_wait(ctx, prev, 120_000_000_000) != lk.LK_OK:
                raise RuntimeError("batch did not finish")
            prev = h
        if lk.lk_wait(ctx, prev, 120_000_000_000) != lk.LK_OK:
            raise RuntimeError("batch did not finish")
        lk_all_s = (time.perf_counter_ns() - t0) / 1e9
    graph_s = []
    for items, _ in gsub:
        ms = lk.lk_baseline_graph(items, n_sms, threads=tuned["threads"], reps=2, device=dev)
        graph_s.append(float(ms[-1]) / 1e3)
    sub_bytes = float(sum(m["bytes"] for _, m in gsub))
    sub_count = int(sum(len(it) for it, _ in gsub))
    all_bytes = float(sum(m["bytes"] for _, m in bbat))
    all_count = int(sum(len(it) for it, _ in bbat))
    batching = {"batches": len(bbat), "items": all_count, "bytes": all_bytes,
                "lk_gbs": all_bytes / lk_all_s / 1e9, "lk_items_per_s": all_count / lk_all_s,
                "lk_seconds": lk_all_s,
                "graph_compared": {"batches": len(gsub), "items": sub_count, "bytes": sub_bytes,
                                   "lk_gbs": sub_bytes / np.sum(lk_sub_s) / 1e9,
                                   "graph_gbs": sub_bytes / np.sum(graph_s) / 1e9,
                                   "lk_items_per_s": sub_count / np.sum(lk_sub_s),
                                   "graph_items_per_s": sub_count / np.sum(graph_s),
                                   "lk_batch_ms": [round(1e3 * x, 3) for x in lk_sub_s],
                                   "graph_batch_ms": [round(1e3 * x, 3) for x in graph_s],
                                   "how": "the first batches of the prefix, one post and wait each, against "
                                          "one CUDA graph of ordinary launches per batch"},
                "items_per_batch": [len(it) for it, _ in bbat],
                "tuned": tuned, "cluster": f"{n_sms} SMs as one cluster",
                "parity_mismatches": batch_bad, "parity_items": int(len(par_items)),
                "sample": f"{len(bbat)} batches ({all_count} descriptors) of the seeded 1M-descriptor stream "
                          f"(the whole stream once the count reaches 1,000,000), batch b+1 posted while batch b "
                          f"runs"}

    # ---- serving: continuous admission under open-loop arrivals, per rate ----------
    hbm_serv = float(measured_peaks()[0].get("hbm_gbs", FALLBACK_HBM))
    # the device-resident queue at every rate (the clusters' CTAs claim work
    # units themselves); the host dispatcher (chunks posted per cluster) and
    # its coalesced variant at the top rates for comparison; unit sizes swept
    # at the top rate
    scfg = wl.SERVING
    arena = torch.empty(scfg["arena_bytes"], dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    serving = {"budget_bytes": scfg["budget_bytes"], "arena_bytes": scfg["arena_bytes"],
               "part_bytes": scfg["part_bytes"], "min_part_bytes": scfg["min_part_bytes"],
               "window_units_per_cta": scfg["queue_window"],
               "producers": scfg["producers"], "seconds_per_rate": args.serve_seconds,
               "partition": "4 clusters x 37 SMs", "rates": {},
               "host_dispatcher": {"chunk_bytes": scfg["chunk_bytes"], "window": scfg["window"], "rates": {}},
               "host_dispatcher_coalesced": {"coalesce_bytes": scfg["coalesce_bytes"],
                                             "coalesce_part_bytes": scfg["coalesce_part_bytes"], "rates": {}},
               "part_bytes_sweep_top_rate": {}}
    top = scfg["rates"][-3:]
    qkw = dict(mode=lk.LK_SERVE_QUEUE, part_bytes=scfg["part_bytes"], min_part_bytes=scfg["min_part_bytes"],
               window=scfg["queue_window"])
    runs = [("rates", r, qkw) for r in scfg["rates"]]
    runs += [("host_dispatcher", r, dict(mode=lk.LK_SERVE_CHUNKS, chunk_bytes=scfg["chunk_bytes"],
                                         window=scfg["window"])) for r in top]
    runs += [("host_dispatcher_coalesced", r, dict(mode=lk.LK_SERVE_CHUNKS, chunk_bytes=scfg["chunk_bytes"],
                                                   window=scfg["window"], coalesce_bytes=scfg["coalesce_bytes"],
                                                   coalesce_part_bytes=scfg["coalesce_part_bytes"]))
             for r in top[-1:]]
    runs += [("part_bytes_sweep_top_rate", scfg["rates"][-1], dict(qkw, part_bytes=pb))
             for pb in (2 << 20, 4 << 20, 16 << 20)]
    with lk.lk_init(scfg["sizes"], device=dev, threads_per_cta=scfg["threads"], idle_lease_ns=30_000_000_000) as ctx:
        for where, rate, kw in runs:
            reqs, inb = wl.serving_requests(pools, seed, rate, args.serve_seconds)
            rc, res = lk.lk_serve(ctx, reqs, n_producers=scfg["producers"], budget_bytes=scfg["budget_bytes"],
                                  arena=arena, arena_bytes=scfg["arena_bytes"], timeout_ns=300_000_000_000, **kw)
            if rc != lk.LK_OK:
                raise RuntimeError(f"serving ({where}) at {rate}/s failed: {lk.lk_strerror(rc)}")
            lat_s = (res["t_complete_ns"] - reqs["t_arrival_ns"]) / 1000.0
            out_b = np.where(reqs["op"] == lk.LK_OP_ADD_I32, inb / 2, np.where(reqs["op"] == lk.LK_OP_GEMM64_F32,
                                                                             inb / 2, 0.0))
            wait_s = (res["t_admit_ns"] - reqs["t_arrival_ns"]) / 1000.0
            span = float(res["t_complete_ns"].max()) / 1e9
            entry = {"requests": int(reqs.size), "latency_us": lat_summary(lat_s),
                     "admission_wait_us": lat_summary(wait_s),
                     "throughput_req_per_s": reqs.size / span,
                     "throughput_gbs": float(inb.sum()) / span / 1e9,
                     # HBM traffic: the inputs plus the outputs (an add writes half its input
                     # bytes, a GEMM tile 16 KB per 32 KB read; sums and histograms ~0)
                     "traffic_gbs": float(inb.sum() + out_b.sum()) / span / 1e9,
                     "offered_gbs": float(inb.sum()) / (float(reqs["t_arrival_ns"].max()) / 1e9) / 1e9,
                     "units_or_chunks": int(res["chunks"].sum())}
            # the slowest requests, each against its own bytes at the measured HBM peak
            top = np.argsort(lat_s)[::-1][:5]
            entry["slowest"] = [{"op": lk.OP_NAMES[int(reqs["op"][i])], "mb": rnd1((inb[i] + out_b[i]) / 1e6),
                                 "units": int(res["chunks"][i]), "us": rnd1(lat_s[i]), "admit_us": rnd1(wait_s[i]),
                                 "hbm_us": rnd1((inb[i] + out_b[i]) / (hbm_serv * 1e3))} for i in top]
            if where == "rates":
                serving["rates"][str(rate)] = entry
            elif where == "part_bytes_sweep_top_rate":
                serving[where][str(kw["part_bytes"])] = entry
            else:
                serving[where]["rates"][str(rate)] = entry
    del arena

    # ---- isolation: critical 16-SM cluster vs best-effort 132-SM cluster -----------
    iso = wl.ISOLATION
    crit_out = torch.zeros(4, device="cuda")
    copy_src = torch.empty(iso["copy_n"], dtype=torch.int32, device="cuda")
    copy_dst = torch.empty_like(copy_src)
    hist_in = pools.u8[: iso["hist_n"]]
    hist_out = torch.zeros(256, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    def iso_run(init_kw, periods, be_rate=0, alone=True, roles=False):
        """`periods` critical periods alone, then under best-effort load, on one
        layout; be_rate caps the best-effort cluster's loads (bytes/us, 0 = none);
        roles makes cluster 0 critical and cluster 1 yield to it (lk_set_role)."""
        out = {"periods": periods}
        for loaded in ((False, True) if alone else (True,)):
            be_items = 0
            if loaded:
                # enough best-effort work to outlast the critical run: time one pair first
                with lk.lk_init(init_kw["sizes"], device=dev, idle_lease_ns=5_000_000_000,
                                **{k: v for k, v in init_kw.items() if k != "sizes"}) as ctx:
                    lk.lk_set_rate(ctx, 1, be_rate)
                    probe_tr = wl.isolation_traces(1, 4, pools.f32, crit_out, copy_src, copy_dst, hist_in, hist_out)
                    rc, rp = lk.lk_run_trace(ctx, probe_tr[1:], n_threads=1, closed_loop=True)
                pair_ns = float(rp["t_complete_ns"][-1]) / 2.0
                be_items = int(2 * periods * iso["period_ns"] / max(pair_ns, 1.0) * 1.1) + 4
            tr = wl.isolation_traces(periods, be_items, pools.f32, crit_out, copy_src, copy_dst, hist_in, hist_out,
                                     loaded=loaded)
            with lk.lk_init(init_kw["sizes"], device=dev, threads_per_cta=iso["threads"], idle_lease_ns=5_000_000_000,
                            **{k: v for k, v in init_kw.items() if k != "sizes"}) as ctx:
                lk.lk_set_rate(ctx, 1, be_rate)
                if roles:
                    lk.lk_set_role(ctx, 0, lk.LK_ROLE_CRITICAL)
                    lk.lk_set_role(ctx, 1, lk.LK_ROLE_YIELD)
                rc, rr = lk.lk_run_trace(ctx, tr, n_threads=2, closed_loop=True, timeout_ns=600_000_000_000,
                                         pin_cpu_base=pin)
            if rc != lk.LK_OK:
                raise RuntimeError(f"isolation trace failed: {lk.lk_strerror(rc)}")
            crit = rr[:periods]
            lat_c = (crit["t_complete_ns"] - crit["t_submit_ns"]) / 1000.0
            rel_c = (crit["t_complete_ns"] - tr["t_arrival_ns"][:periods]) / 1000.0
            key = "loaded" if loaded else "alone"
            out[key + "_us"] = lat_summary(lat_c)
            out[key + "_release_to_complete_us"] = lat_summary(rel_c)
            if loaded:
                be = rr[periods:]
                be_ops = tr["op"][periods:]
                moved = np.where(be_ops == lk.LK_OP_COPY_I32, 8.0 * iso["copy_n"], float(iso["hist_n"] + 1024)).sum()
                span = float(be["t_complete_ns"].max() - be["t_submit_ns"].min())
                out["best_effort_gbs"] = moved / span
                out["best_effort_items"] = int(be.size)
                last_crit = float(crit["t_complete_ns"].max())
                out["load_covered_critical_run"] = bool(float(be["t_complete_ns"].max()) >= last_crit)
        return out

    iso_res = iso_run({"sizes": iso["sizes"]}, args.iso_periods)
    # several persistent CTAs per SM (Sec. II.C's next step): the critical
    # cluster's 16 CTAs share SMs 0-15 with a best-effort cluster that spans
    # every SM, instead of owning 16 SMs the best-effort work cannot use
    with lk.lk_init([n_sms], device=dev, idle_lease_ns=5_000_000_000) as ctx:
        sm_ids = lk.lk_cluster_info(ctx, 0)          # the SM ids the GPU reports, ascending
    nc = iso["sizes"][0]
    co = iso_run({"sizes": [nc, n_sms], "ctas_per_sm": 2, "smids": sm_ids[:nc] + sm_ids}, args.iso_sweep_periods)
    co["inflation_p999"] = co["loaded_us"]["p999"] / co["alone_us"]["p999"]
    co["layout"] = (f"ctas_per_sm = 2; critical: one CTA on each of the {nc} lowest SM ids; best effort: "
                    f"one CTA on every one of the {n_sms} SMs (the other CTA of the critical SMs)")
    # best-effort load-rate caps (token-bucket pacing of its TMA loads): the
    # critical tail against the throughput given up, on the disjoint layout
    paced = {}
    for cap_gbs in (1000, 2000, 3000, 4000):
        pr = iso_run({"sizes": iso["sizes"]}, args.iso_sweep_periods, be_rate=cap_gbs * 1000, alone=False)
        paced[str(cap_gbs)] = {"loaded_us": pr["loaded_us"], "best_effort_gbs": pr["best_effort_gbs"],
                               "inflation_p999": pr["loaded_us"]["p999"] / iso_res["alone_us"]["p999"],
                               "load_covered_critical_run": pr["load_covered_critical_run"]}
    # load yielding: the best-effort cluster holds its loads while a critical
    # descriptor runs (lk_set_role), instead of a standing cap
    yr = iso_run({"sizes": iso["sizes"]}, args.iso_periods, alone=False, roles=True)
    iso_res["best_effort_yield"] = {"periods": yr["periods"], "loaded_us": yr["loaded_us"],
                                    "best_effort_gbs": yr["best_effort_gbs"],
                                    "inflation_p999": yr["loaded_us"]["p999"] / iso_res["alone_us"]["p999"],
                                    "load_covered_critical_run": yr["load_covered_critical_run"]}
    iso_res["inflation_p999"] = iso_res["loaded_us"]["p999"] / iso_res["alone_us"]["p999"]
    iso_res["inflation_max"] = iso_res["loaded_us"]["max"] / iso_res["alone_us"]["max"]
    iso_res["coresident"] = co
    iso_res["best_effort_rate_cap_gbs"] = paced
    iso_sum_ok = abs(float(crit_out[0].cpu()) - oracle.sum_f32(pools.f32[: iso["crit_n"]].cpu().numpy())) <= \
        1e-4 * oracle.abs_sum_f32(pools.f32[: iso["crit_n"]].cpu().numpy())
    iso_copy_ok = bool(torch.equal(copy_dst[-(1 << 20):], copy_src[-(1 << 20):]))
    iso_res["parity"] = {"critical_sum_ok": bool(iso_sum_ok), "copy_tail_ok": iso_copy_ok}
    del copy_src, copy_dst

    # ---- the paper's life cycle (Sec. III, Tables 2-3): Init/Trigger/Wait/Dispose ----
    PAPER = {"single_sm": {"LK": (509e6, 239, 190e3, 30e6), "CUDA": (496e6, 3.9e3, 175e3, 274e3)},
             "full_gpu": {"LK": (503e6, 210, 190e3, 30e6), "CUDA": (497e6, 3.8e3, 176e3, 247e3)},
             "worst_single_sm": {"LK": (521e6, 1.1e3, 203e3, 33e6), "CUDA": (501e6, 7.7e3, 176e3, 893e3)}}
    phases = {"iters": 20000, "runs": args.phase_runs, "unit": "us (host CLOCK_MONOTONIC)",
              "paper_context": "GTX 980 + i7 at 3.6 GHz, host cycles / 3.6e3 = us; Tables 2-3", "configs": {}}
    names = ("init", "trigger", "wait", "dispose")
    for label, nsm in (("single_sm", 1), ("full_gpu", n_sms)):
        t_lk = lk.lk_phase_run(sms=nsm, iters=20000, runs=args.phase_runs, device=dev)
        t_cu = lk.lk_baseline_phase_run(sms=nsm, iters=20000, runs=args.phase_runs, device=dev)
        entry = {}
        for sysname, t in (("LK", t_lk), ("CUDA", t_cu)):
            entry[sysname] = {nm: {"avg": float(np.mean(t[nm + "_ns"])) / 1e3, "worst": float(np.max(t[nm + "_ns"])) / 1e3,
                                   "first": float(t[nm + "_ns"][0]) / 1e3}
                              for nm in names}
        entry["paper_avg_us"] = {k: [round(v / 3.6e3, 3) for v in vals] for k, vals in PAPER[label].items()}
        if label == "single_sm":
            entry["paper_worst_us"] = {k: [round(v / 3.6e3, 3) for v in vals] for k, vals in PAPER["worst_single_sm"].items()}
        phases["configs"][label] = entry

    # ---- body bandwidth (finite mode) and the roofline ------------------------------
    bw = body_bandwidth(pools, lk, n_sms)
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM))
    add = bw["add_i32"]
    traffic = profiled_traffic("lk_finite_add_i32_2p28.txt")
    roofline = {"kernel": f"lk_finite (the persistent kernel, 256 threads, in finite mode), add_i32 n=2^28 "
                          f"x{add['descriptors_per_launch']} per launch, {n_sms} SMs as one cluster",
                "bound": "hbm", "achieved": add["gbs"], "peak": hbm, "unit": "GB/s", "frac": add["gbs"] / hbm,
                "peak_source": f"{peak_src} (hbm_gbs, burst copy)", "traffic": traffic,
                "algorithmic_bytes_per_launch": add["bytes_per_launch"]}

    # ---- CPU baseline: the oracle on a bounded sample ------------------------------
    cpu = None
    if dist.rank == 0:
        import oracle as _o

        _o.build()
        if full_mask:
            try:
                os.sched_setaffinity(0, full_mask)   # the oracle may use every core
            except OSError:
                pass
        sample = oracle_sample(424242, 400)
        us = time_oracle(sample, budget_s=15.0)
        names = ["add_i32", "hist_u8", "sum_f32", "gemm64_f32"]   # the sample cycles through the bodies
        workers = host_info()["cores"]
        cpu = {"value": pct(us, 0.99), "unit": "us", "cores": 1, "kind": "oracle",
               "sample": f"{us.size} items of the workload's body mix (equal shares), per-item time, one host thread",
               "p50": pct(us, 0.5),
               "per_body_p50_us": {nm: pct(us[j::4], 0.5) for j, nm in enumerate(names) if us[j::4].size},
               "all_cores": {"items_per_s": time_oracle_pool(sample, workers), "threads": workers,
                             "sample": f"the same {len(sample)} items on a thread pool"}}

    p99 = dist.max(pct(lat, 0.99))
    mx = dist.max(pct(lat, 1.0))
    items_all = dist.sum(float(lat.size))
    wall_all = dist.max(wall)
    kms = dist.max(float(np.mean(kernel_ms)))
    if dist.rank != 0:
        return
    detail = {
        "config": bench_config(args, cfg),
        "step": "lk_init + trace + lk_dispose (one persistent-kernel launch)",
        "submitter_cpus": list(range(pin, pin + 4)) if pin >= 0 else "not pinned",
        "host": host_info(),
        "latency_us": lat_summary(lat),
        "arrival_to_complete_us": lat_summary(lat_arr),
        "baseline_launch_sync_us": lat_summary(base),
        "latency_by_op_us_p50_p99_max": by_op,
        "tail_attribution": tail,
        "baseline_occupancy_grid_us": dict(lat_summary(base_occ), grid=occ_grid,
                                           note="one step's trace; grid from the occupancy API (1 CTA/SM x all SMs)"),
        "config_small": small,
        "dispatch_nop_us": {"lk": lat_summary(nop_lk), "lk_direct": lat_summary(nop_direct),
                            "lk_mailbox": lat_summary(nop_mbox), "launch_sync": lat_summary(nop_base),
                            "lk_device_phases": nop_phases, "lk_direct_device_phases": nop_phases_direct},
        "paper_mailbox_vs_ring": mbox,
        "pingpong_floor_us": lat_summary(rtt),
        "throughput_items_per_s": items_all / wall_all,
        "wall_ms_per_step": 1000.0 * wall_all / args.steps,
        "body_detail": bw,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"latency_us": lat_summary(e2e), "launch_sync_e2e_us": lat_summary(e2e_base),
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "parts_us": {"lk": e2e_parts(re), "launch_sync": e2e_parts(rb)},
                "how": "per item: pinned host->device input copies, lk submit, wait, device->host output copy; "
                       "parts: copy in (submit -> post), dispatch (post -> completion observed), copy out "
                       "(observed -> complete), host clock"},
        "paper_phases": phases,
        "batching": batching,
        "serving": serving,
        "isolation": iso_res,
        "clocks": clk,
        "parity": {"sampled_items": int(len(pick)), "mismatches": bad, "exec_log": log_verdict},
    }
    with open(args.detail, "w") as fh:
        json.dump(detail, fh, indent=1)

    headline = build_headline(detail, hbm)
    line = {
        "metric": METRIC, "value": p99, "unit": "us", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": kms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32 / uint8->int32 / fp32 (GEMM whole tiles: fp32 split in two bf16 parts, tcgen05, fp32 accumulate)",
        "data": "synthetic (seeded device pools)",
        "config": bench_config(args, cfg),
        "max_us": mx,
        "headline": headline,
        "roofline": {k: (round(v, 4) if isinstance(v, float) else v) for k, v in roofline.items()
                     if k in ("bound", "achieved", "peak", "unit", "frac", "traffic")},
        "cpu_baseline": {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")} if cpu else None,
        "e2e": {"value": pct(e2e, 0.99), "unit": "us", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "launch_sync_p99": rnd1(pct(e2e_base, 0.99)),
                "p99_copy_in_dispatch_copy_out_us": [rnd1(detail["e2e"]["parts_us"]["lk"][k]["p99"])
                                                     for k in ("copy_in", "dispatch", "copy_out")]},
        "gpu_launches": args.steps,
        "clocks": {k: clk.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "detail_file": os.path.basename(args.detail),
    }
    print(json.dumps(line, separators=(",", ":")))


if __name__ == "__main__":
    main()
