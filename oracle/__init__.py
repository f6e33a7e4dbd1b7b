"""CPU oracle for the LightKernel hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package.  It shares no code with the
CUDA path (``paper_2310_01212_gb300``) and never imports it.

* ``lk_oracle.c`` holds the work bodies (plain loops, binary64 accumulation)
  and the execution-log checker; ``build()`` compiles it with gcc.
* ``protocol.py`` is a sequential simulator of the host<->GPU dispatch
  protocol of Sec. II.D (dual mailbox, Table 1 status codes) and of its
  multi-slot ring generalisation, with a seeded scheduler and an exhaustive
  state-space search for tiny instances.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liblk_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile lk_oracle.c into oracle/_build/liblk_oracle.so (gcc, -O2)."""
    src = os.path.join(_HERE, "lk_oracle.c")
    hdr = os.path.join(_HERE, "lk_oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


class CheckResult(ctypes.Structure):
    _fields_ = [("violations", ctypes.c_int64), ("first_index", ctypes.c_int64),
                ("first_code", ctypes.c_int32), ("counts", ctypes.c_int32 * 10)]


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            l = ctypes.CDLL(build())
            P = ctypes.c_void_p
            S = ctypes.c_size_t
            l.lko_add_i32.argtypes = [P, P, P, S]
            l.lko_copy_i32.argtypes = [P, P, S]
            l.lko_hist_u8.argtypes = [P, S, P]
            l.lko_sum_f32.argtypes = [P, S]
            l.lko_sum_f32.restype = ctypes.c_double
            l.lko_abs_sum_f32.argtypes = [P, S]
            l.lko_abs_sum_f32.restype = ctypes.c_double
            l.lko_gemm64_f32.argtypes = [P, P, P, S]
            l.lko_gemm64_abs_bound.argtypes = [P, P, P, S]
            l.lko_spin_xor.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64]
            l.lko_spin_xor.restype = ctypes.c_uint32
            l.lko_lcg_jump.argtypes = [ctypes.c_uint32, ctypes.c_uint64]
            l.lko_lcg_jump.restype = ctypes.c_uint32
            l.lko_lcg_brute.argtypes = [ctypes.c_uint32, ctypes.c_uint64]
            l.lko_lcg_brute.restype = ctypes.c_uint32
            l.lko_check_exec_log.argtypes = [S] + [P] * 6 + [ctypes.c_int32] + [P] * 6 + [ctypes.POINTER(CheckResult)]
            l.lko_check_exec_log.restype = ctypes.c_int64
            _lib = l
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def add_i32(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.int32)
    assert a.shape == b.shape
    out = np.empty_like(a)
    lib().lko_add_i32(_p(a), _p(b), _p(out), a.size)
    return out


def copy_i32(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.int32)
    out = np.empty_like(x)
    lib().lko_copy_i32(_p(x), _p(out), x.size)
    return out


def hist_u8(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint8)
    bins = np.zeros(256, dtype=np.int64)
    lib().lko_hist_u8(_p(x), x.size, _p(bins))
    return bins


def sum_f32(x: np.ndarray) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32)
    return float(lib().lko_sum_f32(_p(x), x.size))


def abs_sum_f32(x: np.ndarray) -> float:
    x = np.ascontiguousarray(x, dtype=np.float32)
    return float(lib().lko_abs_sum_f32(_p(x), x.size))


def gemm64_f32(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A, B: (..., 64, 64) float32 tiles -> binary64 products of the same shape."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    assert A.shape == B.shape and A.shape[-2:] == (64, 64)
    C = np.empty(A.shape, dtype=np.float64)
    lib().lko_gemm64_f32(_p(A), _p(B), _p(C), A.size // 4096)
    return C


def gemm64_abs_bound(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    C = np.empty(A.shape, dtype=np.float64)
    lib().lko_gemm64_abs_bound(_p(A), _p(B), _p(C), A.size // 4096)
    return C


def spin_xor(rank: int, threads: int, iters: int) -> int:
    return int(lib().lko_spin_xor(rank, threads, iters))


def lcg_jump(x0: int, iters: int) -> int:
    return int(lib().lko_lcg_jump(x0, iters))


def lcg_brute(x0: int, iters: int) -> int:
    return int(lib().lko_lcg_brute(x0, iters))


# violation codes of the execution-log checker (lk_oracle.h)
VIOLATIONS = {0: "ok", 1: "bad_cluster", 2: "bad_rank", 3: "bad_seq", 4: "duplicate", 5: "missing",
              6: "fifo", 7: "wrong_sm", 8: "wrong_op", 9: "early_complete"}


def check_exec_log(seq, cluster, rank, smid, op, order, cluster_size, n_posted,
                   pinned_smid=None, posted_op=None, t_end=None, t_complete=None) -> dict:
    """Run the C checker; returns {"violations": n, "first": name, "counts": {name: k}}."""
    seq = np.ascontiguousarray(seq, dtype=np.uint64)
    m = seq.size
    cluster = np.ascontiguousarray(cluster, dtype=np.int32)
    rank = np.ascontiguousarray(rank, dtype=np.int32)
    smid = np.ascontiguousarray(smid, dtype=np.int32)
    op = np.ascontiguousarray(op, dtype=np.int32)
    order = np.ascontiguousarray(order, dtype=np.uint64)
    assert all(a.size == m for a in (cluster, rank, smid, op, order))
    cs = np.ascontiguousarray(cluster_size, dtype=np.int32)
    npost = np.ascontiguousarray(n_posted, dtype=np.uint64)
    ps = None if pinned_smid is None else np.ascontiguousarray(pinned_smid, dtype=np.int32)
    po = None if posted_op is None else np.ascontiguousarray(posted_op, dtype=np.int32)
    te = None if t_end is None else np.ascontiguousarray(t_end, dtype=np.uint64)
    tc = None if t_complete is None else np.ascontiguousarray(t_complete, dtype=np.uint64)
    if ps is not None:
        assert ps.size == int(cs.sum())
    if po is not None:
        assert po.size == int(npost.sum())
    res = CheckResult()
    n = lib().lko_check_exec_log(m, _p(seq), _p(cluster), _p(rank), _p(smid), _p(op), _p(order),
                                 cs.size, _p(cs), None if ps is None else _p(ps), _p(npost),
                                 None if po is None else _p(po), None if te is None else _p(te),
                                 None if tc is None else _p(tc), ctypes.byref(res))
    return {"violations": int(n), "first": VIOLATIONS[res.first_code] if n else "ok",
            "first_index": int(res.first_index),
            "counts": {VIOLATIONS[i]: int(res.counts[i]) for i in range(10) if res.counts[i]}}
