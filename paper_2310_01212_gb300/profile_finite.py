"""Run one finite-mode launch of the persistent kernel for a profiler.

Finite mode pre-fills the mailbox ring in device memory (ending with EXIT),
so the kernel needs no host interaction while it runs and a profiler can
replay it.  The inputs are allocated here and sized by --log2n, so that a
capture stays small (a few GB on the device at most).

  python -m paper_2310_01212_gb300.profile_finite --op add_i32 --log2n 26 [--sms N] [--threads 256] [--launches 1]
        [--ffma]                 GEMM tiles on the FFMA path
        [--partition 37,37,37,37 --cluster 0 --per-launch 256 --pool-log2 30]
                                 descriptors on one cluster of a partition, inputs at random
                                 offsets of a pool larger than L2 (per-cluster counters)
"""
from __future__ import annotations

import argparse

from . import build, lk

OPS = {"add_i32": lk.LK_OP_ADD_I32, "copy_i32": lk.LK_OP_COPY_I32, "sum_f32": lk.LK_OP_SUM_F32,
       "hist_u8": lk.LK_OP_HIST_U8, "gemm64_f32": lk.LK_OP_GEMM64_F32, "nop": lk.LK_OP_NOP}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="add_i32", choices=sorted(OPS))
    ap.add_argument("--log2n", type=int, default=26, help="elements (bytes for hist_u8, tiles for gemm: n/4096)")
    ap.add_argument("--sms", type=int, default=0, help="CTAs in the one cluster (0 = every SM)")
    ap.add_argument("--threads", type=int, default=256)
    ap.add_argument("--per-launch", type=int, default=1, help="descriptors per launch")
    ap.add_argument("--launches", type=int, default=1)
    ap.add_argument("--ffma", action="store_true", help="LK_INIT_GEMM_FFMA: GEMM tiles on the FFMA path")
    ap.add_argument("--partition", default="", help="cluster sizes, e.g. 37,37,37,37 (default: one cluster of --sms)")
    ap.add_argument("--cluster", type=int, default=0, help="the cluster of --partition that runs the descriptors")
    ap.add_argument("--pool-log2", type=int, default=0,
                    help="inputs: each descriptor reads a random 16-B-aligned slice of a pool of 2^L bytes "
                         "(0: every descriptor reads the same input)")
    args = ap.parse_args()

    import torch

    build.build()
    sms = args.sms or torch.cuda.get_device_properties(0).multi_processor_count
    op = OPS[args.op]
    n = 1 << args.log2n
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    in1 = None
    if op in (lk.LK_OP_ADD_I32, lk.LK_OP_COPY_I32):
        in0 = torch.randint(-(1 << 20), 1 << 20, (n,), dtype=torch.int32, device="cuda", generator=g)
        in1 = torch.randint(-(1 << 20), 1 << 20, (n,), dtype=torch.int32, device="cuda", generator=g) \
            if op == lk.LK_OP_ADD_I32 else None
        out, cnt = torch.empty_like(in0), n
    elif op == lk.LK_OP_SUM_F32:
        in0 = torch.randn((n,), device="cuda", generator=g)
        out, cnt = torch.empty(4, device="cuda"), n
    elif op == lk.LK_OP_HIST_U8:
        in0 = torch.randint(0, 256, (n,), dtype=torch.uint8, device="cuda", generator=g)
        out, cnt = torch.empty(256, dtype=torch.int32, device="cuda"), n
    elif op == lk.LK_OP_GEMM64_F32:
        in0 = torch.randn((n,), device="cuda", generator=g)
        in1 = torch.randn((n,), device="cuda", generator=g)
        out, cnt = torch.empty_like(in0), n // 4096
    else:
        in0, out, cnt = None, None, 0
    k = args.per_launch
    sizes = [int(x) for x in args.partition.split(",")] if args.partition else [sms]
    ins0, ins1 = [in0] * k, [in1] * k
    if args.pool_log2 and in0 is not None:
        # config-shaped inputs: slices of a pool larger than L2 at seeded offsets
        esize = in0.element_size()
        pool_el = (1 << args.pool_log2) // esize
        p0 = torch.empty(pool_el, dtype=in0.dtype, device="cuda")
        p1 = torch.empty(pool_el, dtype=in0.dtype, device="cuda") if in1 is not None else None
        p0.copy_(in0.repeat((pool_el + in0.numel() - 1) // in0.numel())[:pool_el])
        if p1 is not None:
            p1.copy_(in1.repeat((pool_el + in1.numel() - 1) // in1.numel())[:pool_el])
        span = (pool_el - in0.numel()) // (16 // esize)
        offs = torch.randint(0, max(1, span), (k,), generator=torch.Generator().manual_seed(7)).tolist()
        ins0 = [p0[o * (16 // esize):o * (16 // esize) + in0.numel()] for o in offs]
        ins1 = [p1[o * (16 // esize):o * (16 // esize) + in1.numel()] for o in offs] if p1 is not None else ins1
    torch.cuda.synchronize()
    for _ in range(args.launches):
        ms, _log = lk.lk_run_finite(sizes, [(op, cnt)] * k, [args.cluster] * k,
                                    in0=ins0 if in0 is not None else None,
                                    in1=ins1 if in1 is not None else None,
                                    out=[out] * k if out is not None else None, threads_per_cta=args.threads,
                                    exec_log_cap=k + 1, flags=lk.LK_INIT_GEMM_FFMA if args.ffma else 0)
        print(f"{args.op} n=2^{args.log2n} x{k} on cluster {args.cluster} of {sizes}, {args.threads} threads: "
              f"{ms:.4f} ms")


if __name__ == "__main__":
    main()
