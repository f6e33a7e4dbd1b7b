"""Autotuner for batches: block size and the split rule.

A batch item of input size B bytes runs as parts = clamp(ceil(B / part_bytes),
1, max_parts) work units (lk_batch_tune); the block size is the context's
threads per CTA.  The tuner times a fixed seeded set of batching-stream
batches for every (threads, max_parts, part_bytes) on the grid, through
lk_submit_batch on a context of every SM, and keeps the fastest.  The result
is written to autotune_gb300.json beside this file and read by `load()`.

  python -m paper_2310_01212_gb300.autotune [--batches 4] [--max-count 512]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import build, lk, workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "autotune_gb300.json")
GRID = dict(threads=(128, 256, 512), max_parts=(1, 2, 4, 8), part_bytes=(1 << 20, 4 << 20, 16 << 20))
DEFAULT = dict(threads=256, max_parts=8, part_bytes=4 << 20)


def load() -> dict:
    if os.path.exists(TABLE):
        with open(TABLE) as f:
            best = json.load(f).get("best")
        if best:
            return best
    return dict(DEFAULT)


def time_batches(ctx, batches, max_parts: int, part_bytes: int, reps: int = 2) -> float:
    """Seconds for all batches, best of `reps` passes (one post + wait each)."""
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        for items in batches:
            while True:
                h = lk.lk_submit_batch(ctx, 0, items, max_parts=max_parts, part_bytes=part_bytes)
                if h is not None:
                    break
            if lk.lk_wait(ctx, h, 60_000_000_000) != lk.LK_OK:
                raise RuntimeError("batch did not finish")
        best = min(best, time.perf_counter() - t0)
    return best


def tune(pools, n_sms: int, seed: int = 999, n_batches: int = 4, max_count: int = 512, grid: dict = GRID,
         device: int = 0) -> dict:
    import torch

    batches = [wl.batching_batch(pools, seed, b, max_count=max_count)[0] for b in range(n_batches)]
    torch.cuda.synchronize()
    results = []
    for threads in grid["threads"]:
        with lk.lk_init([n_sms], device=device, threads_per_cta=threads, max_batch_units=1 << 16,
                        idle_lease_ns=10_000_000_000) as ctx:
            time_batches(ctx, batches[:1], 8, 4 << 20, reps=1)   # warm-up
            for mp in grid["max_parts"]:
                for pb in grid["part_bytes"]:
                    s = time_batches(ctx, batches, mp, pb)
                    results.append(dict(threads=threads, max_parts=mp, part_bytes=pb, seconds=s))
    best = min(results, key=lambda r: r["seconds"])
    return dict(best={k: best[k] for k in ("threads", "max_parts", "part_bytes")}, results=results,
                batches=n_batches, max_count=max_count, seed=seed)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--batches", type=int, default=4)
    ap.add_argument("--max-count", type=int, default=512)
    ap.add_argument("--out", default=TABLE)
    args = ap.parse_args()
    import torch

    build.build()
    n_sms = torch.cuda.get_device_properties(0).multi_processor_count
    pools = wl.Pools.create(0)
    out = tune(pools, n_sms, n_batches=args.batches, max_count=args.max_count)
    out["device"] = torch.cuda.get_device_name(0)
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out["best"]))
    for r in sorted(out["results"], key=lambda r: r["seconds"])[:8]:
        print(r)


if __name__ == "__main__":
    main()
