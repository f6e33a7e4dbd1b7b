"""Helpers shared by the GPU tests (inputs move host -> device with torch;
results come back to the host and are compared with the oracle)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def to_dev(a: np.ndarray):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t) -> np.ndarray:
    import torch

    torch.cuda.current_stream().synchronize()
    return t.cpu().numpy()


def sum_ok(got: float, x: np.ndarray, oracle) -> bool:
    """|s_gpu - S| <= 1e-4 * sum|x| against the binary64 oracle sum."""
    return abs(float(got) - oracle.sum_f32(x)) <= 1e-4 * oracle.abs_sum_f32(x)


def gemm_ok(C: np.ndarray, A: np.ndarray, B: np.ndarray, oracle) -> bool:
    """Per element |C - C64| <= 1e-4 * sum_k |a_ik b_kj| (exact zero bound -> exact)."""
    C64 = oracle.gemm64_f32(A, B)
    bound = oracle.gemm64_abs_bound(A, B)
    return bool(np.all(np.abs(C.astype(np.float64) - C64) <= 1e-4 * bound))


def check_log(oracle, ctx, log, sizes, n_posted, posted_op=None):
    """Run the oracle's execution-log checker on a context's log: the
    completion time of each descriptor is the t_done of its last arriver."""
    from paper_2310_01212_gb300 import lk

    pinned = sum((lk.lk_cluster_info(ctx, c) for c in range(len(sizes))), [])
    off = np.concatenate([[0], np.cumsum(n_posted)])
    t_complete = np.zeros(int(off[-1]), dtype=np.uint64)
    last = log[log["t_done_ns"] > 0]
    idx = off[last["cluster"].astype(np.int64)] + last["seq"].astype(np.int64) - 1
    t_complete[idx] = last["t_done_ns"]
    res = oracle.check_exec_log(log["seq"], log["cluster"], log["rank"], log["smid"], log["op"], log["order"],
                                sizes, n_posted, pinned_smid=pinned, posted_op=posted_op,
                                t_end=log["t_end_ns"], t_complete=t_complete)
    # exactly one last arriver per descriptor
    assert len(last) == int(off[-1])
    return res, pinned
