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
