"""Run one finite-mode launch of the persistent kernel for a profiler.

Finite mode pre-fills the mailbox ring in device memory (ending with EXIT),
so the kernel needs no host interaction while it runs and a profiler can
replay it.  The inputs are allocated here and sized by --log2n, so that a
capture stays small (a few GB on the device at most).

  python -m paper_2310_01212_gb300.profile_finite --op add_i32 --log2n 26 [--sms N] [--threads 256] [--launches 1]
                                                  [--ffma]   (GEMM tiles on the FFMA path)
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
    torch.cuda.synchronize()
    k = args.per_launch
    for _ in range(args.launches):
        ms, _log = lk.lk_run_finite([sms], [(op, cnt)] * k, [0] * k, in0=[in0] * k if in0 is not None else None,
                                    in1=[in1] * k if in1 is not None else None,
                                    out=[out] * k if out is not None else None, threads_per_cta=args.threads,
                                    exec_log_cap=k + 1, flags=lk.LK_INIT_GEMM_FFMA if args.ffma else 0)
        print(f"{args.op} n=2^{args.log2n} x{k} on {sms} SMs, {args.threads} threads: {ms:.4f} ms")


if __name__ == "__main__":
    main()
