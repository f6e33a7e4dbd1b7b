"""Python binding of the LightKernel C ABI (include/lk.h).

Argument marshalling only: every step of the dispatch path and every work body
runs in liblk.so (host runtime + persistent CUDA kernel).  There is no Python
or CPU fallback: if the library is missing, loading fails with an error.

Functions keep the C names (lk_init, lk_submit, lk_poll, lk_wait, lk_sync,
lk_dispose, ...).  Device pointers may be given as ints or as objects with a
``data_ptr()`` method (torch tensors); a tensor must be a contiguous CUDA
tensor holding at least the bytes the operation touches (``op_bytes``), which
is checked here before the call.  Failures raise ``LkError`` carrying the
C return code, except where a code is an expected answer (lk_poll's
LK_PENDING, lk_wait's LK_ETIMEDOUT, lk_submit's LK_EAGAIN), which are returned.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

# ---- constants (include/lk.h) ------------------------------------------------
LK_OK, LK_PENDING = 0, 1
LK_EINVAL, LK_EAGAIN, LK_ETIMEDOUT, LK_EDEVICE, LK_ESTATE, LK_ENOMEM, LK_EBUSY = -1, -2, -3, -4, -5, -6, -7
LK_ST_INIT, LK_ST_FINISHED, LK_ST_WORKING, LK_ST_NOP, LK_ST_EXITED, LK_ST_ERROR = 0, 1, 2, 4, 8, 32
LK_CMD_NOP, LK_CMD_EXIT, LK_CMD_WORK = 4, 8, 16
LK_INIT_DIRECT = 1
LK_INIT_MAILBOX = 2
LK_INIT_GEMM_FFMA = 4
LK_RATE_MIN = 1000
LK_OP_NOP, LK_OP_ADD_I32, LK_OP_HIST_U8, LK_OP_SUM_F32, LK_OP_GEMM64_F32, LK_OP_COPY_I32 = 0, 1, 2, 3, 4, 5
LK_OP_COMBINE_SUM, LK_OP_COMBINE_HIST = 6, 7
LK_OP_SPIN = 8
LK_OP_BATCH = 9
LK_OP_SERVE = 10
LK_SERVE_CHUNKS, LK_SERVE_QUEUE = 0, 1
LK_ROLE_NONE, LK_ROLE_CRITICAL, LK_ROLE_YIELD = 0, 1, 2
(LK_DERR_NONE, LK_DERR_LEASE, LK_DERR_ABORT, LK_DERR_BOOT, LK_DERR_STALL, LK_DERR_BADDESC, LK_DERR_STAGING,
 LK_DERR_BOUNDS) = range(8)
OP_INPUTS = {LK_OP_NOP: 0, LK_OP_ADD_I32: 2, LK_OP_HIST_U8: 1, LK_OP_SUM_F32: 1, LK_OP_GEMM64_F32: 2,
             LK_OP_COPY_I32: 1, 6: 1, 7: 1, 8: 0}
OP_NAMES = {LK_OP_NOP: "nop", LK_OP_ADD_I32: "add_i32", LK_OP_HIST_U8: "hist_u8", LK_OP_SUM_F32: "sum_f32",
            LK_OP_GEMM64_F32: "gemm64_f32", LK_OP_COPY_I32: "copy_i32"}


class LkError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


# ---- structures ----------------------------------------------------------------
class lk_init_params(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("num_clusters", ctypes.c_int),
                ("sms_per_cluster", ctypes.POINTER(ctypes.c_int)), ("smids", ctypes.POINTER(ctypes.c_int)),
                ("threads_per_cta", ctypes.c_int), ("ring_depth", ctypes.c_int),
                ("backoff_base_ns", ctypes.c_uint64), ("backoff_cap_ns", ctypes.c_uint64),
                ("idle_lease_ns", ctypes.c_uint64), ("boot_timeout_ns", ctypes.c_uint64),
                ("exec_log_cap", ctypes.c_uint32), ("flags", ctypes.c_uint32),
                ("max_batch_units", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("serve_units", ctypes.c_uint32)]


class lk_desc(ctypes.Structure):
    _fields_ = [("op", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("n", ctypes.c_uint64),
                ("aux", ctypes.c_uint64)]


EXEC_REC_DTYPE = np.dtype([("seq", "<u8"), ("cluster", "<u4"), ("rank", "<u4"), ("smid", "<u4"), ("op", "<u4"),
                           ("order", "<u8"), ("t_pick_ns", "<u8"), ("t_start_ns", "<u8"), ("t_end_ns", "<u8"),
                           ("t_done_ns", "<u8")])
assert EXEC_REC_DTYPE.itemsize == 64

BATCH_ITEM_DTYPE = np.dtype([("in0", "<u8"), ("in1", "<u8"), ("out", "<u8"), ("op", "<u4"), ("parts", "<u4"),
                             ("n", "<u8")])
assert BATCH_ITEM_DTYPE.itemsize == 40


class lk_batch_tune(ctypes.Structure):
    _fields_ = [("max_parts", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("part_bytes", ctypes.c_uint64)]


REQUEST_DTYPE = np.dtype([("t_arrival_ns", "<u8"), ("op", "<u4"), ("producer", "<u4"), ("n", "<u8"), ("in0", "<u8"),
                          ("in1", "<u8"), ("out", "<u8")])
REQUEST_RES_DTYPE = np.dtype([("t_admit_ns", "<u8"), ("t_complete_ns", "<u8"), ("out", "<u8"), ("status", "<i4"),
                              ("chunks", "<u4")])
assert REQUEST_DTYPE.itemsize == 48 and REQUEST_RES_DTYPE.itemsize == 32


class lk_serve_params(ctypes.Structure):
    _fields_ = [("n_producers", ctypes.c_int), ("window", ctypes.c_int), ("chunk_bytes", ctypes.c_uint64),
                ("budget_bytes", ctypes.c_uint64), ("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_uint64),
                ("timeout_ns", ctypes.c_uint64), ("coalesce_bytes", ctypes.c_uint64), ("coalesce_max", ctypes.c_uint32),
                ("coalesce_part_bytes", ctypes.c_uint32), ("mode", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32),
                ("part_bytes", ctypes.c_uint64), ("min_part_bytes", ctypes.c_uint64)]


TRACE_ITEM_DTYPE = np.dtype([("t_arrival_ns", "<u8"), ("cluster", "<i4"), ("op", "<u4"), ("n", "<u8"),
                             ("in0", "<u8"), ("in1", "<u8"), ("out", "<u8"), ("h_in0", "<u8"), ("h_in1", "<u8"),
                             ("h_out", "<u8"), ("in0_bytes", "<u8"), ("in1_bytes", "<u8"), ("out_bytes", "<u8")])
LK_TRACE_OPEN, LK_TRACE_CLOSED, LK_TRACE_E2E = 0, 1, 2
TRACE_RES_DTYPE = np.dtype([("t_submit_ns", "<u8"), ("t_complete_ns", "<u8"), ("status", "<i4"),
                            ("thread", "<i4"), ("t_post_ns", "<u8"), ("t_observed_ns", "<u8")])
assert TRACE_ITEM_DTYPE.itemsize == 96 and TRACE_RES_DTYPE.itemsize == 40

# ---- library loading -------------------------------------------------------------
_libs: dict = {}
_lock = threading.Lock()


def library_path(fake: bool = False, bounds: bool = False) -> str:
    return _build.FAKE if fake else (_build.BOUNDS if bounds else _build.LIB)


def load(fake: bool = False, bounds: bool = False) -> ctypes.CDLL:
    """Load liblk.so (or the fake-device test build, or the bounds-checking
    build liblk_bounds.so).  Raises if it is missing."""
    key = (bool(fake), bool(bounds) and not fake)
    with _lock:
        if key in _libs:
            return _libs[key]
        path = library_path(*key)
        if not os.path.exists(path):
            raise OSError(f"{path} is missing: run paper_2310_01212_gb300.build.build() "
                          "(no CPU fallback exists)")
        lib = ctypes.CDLL(path)
        P, I, U64, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t
        sig = {
            "lk_init": (I, [ctypes.POINTER(P), ctypes.POINTER(lk_init_params)]),
            "lk_submit": (I, [P, I, ctypes.POINTER(lk_desc), ctypes.POINTER(P), I, P, ctypes.POINTER(U64)]),
            "lk_poll": (I, [P, U64]),
            "lk_wait": (I, [P, U64, U64]),
            "lk_sync": (I, [P, U64]),
            "lk_heartbeat": (I, [P]),
            "lk_set_rate": (I, [P, I, U64]),
            "lk_set_role": (I, [P, I, I]),
            "lk_serve_parts": (ctypes.c_uint32, [ctypes.c_uint32, U64, ctypes.c_uint32, U64, U64, U64, U64]),
            "lk_dispose": (I, [P, U64]),
            "lk_dispose_timed": (I, [P, U64, ctypes.POINTER(ctypes.c_float)]),
            "lk_cluster_info": (I, [P, I, ctypes.POINTER(I), I]),
            "lk_status": (I, [P, I]),
            "lk_device_error": (I, [P]),
            "lk_num_sms": (I, [P]),
            "lk_num_ctas": (I, [P]),
            "lk_exec_log": (I, [P, P, SZ, ctypes.POINTER(SZ), ctypes.POINTER(U64)]),
            "lk_strerror": (ctypes.c_char_p, [I]),
            "lk_run_finite": (I, [ctypes.POINTER(lk_init_params), ctypes.POINTER(lk_desc), ctypes.POINTER(I),
                                  ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), SZ,
                                  ctypes.POINTER(ctypes.c_float), P, SZ, ctypes.POINTER(SZ)]),
            "lk_run_trace": (I, [P, P, SZ, I, I, I, U64, P]),
            "lk_baseline_run_trace": (I, [I, P, SZ, I, ctypes.POINTER(I), I, I, I, I, P]),
            "lk_pingpong": (I, [I, I, ctypes.POINTER(U64)]),
            "lk_launch_noalloc": (I, [I, ctypes.POINTER(lk_desc), ctypes.POINTER(P), I, P, I, I, P]),
            "lk_bounds_violations": (I, [I, ctypes.POINTER(U64), ctypes.POINTER(ctypes.c_uint32)]),
            "lk_submit_batch": (I, [P, I, P, ctypes.c_uint32, ctypes.POINTER(lk_batch_tune), ctypes.POINTER(U64)]),
            "lk_serve": (I, [P, P, SZ, ctypes.POINTER(lk_serve_params), P]),
            "lk_serve_queue_state_bytes": (U64, [ctypes.c_uint32]),
            "lk_phase_run": (I, [I, I, I, U64, I, P, P]),
            "lk_baseline_phase_run": (I, [I, I, I, U64, I, P, P]),
            "lk_baseline_graph": (I, [I, P, ctypes.c_uint32, I, I, I, ctypes.POINTER(ctypes.c_float)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _libs[key] = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().lk_strerror(code).decode()
    except OSError:
        return load(True).lk_strerror(code).decode()


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def op_bytes(op: int, n: int, ctas: int = 0) -> tuple:
    """Bytes of (in0, in1, out) that one descriptor of `op` over `n` reads or
    writes, from the operation definitions in include/lk.h; `ctas` = the CTAs
    that run it (LK_OP_SPIN writes one uint32 per CTA)."""
    n = int(n)
    if op == LK_OP_ADD_I32:
        return 4 * n, 4 * n, 4 * n
    if op == LK_OP_HIST_U8:
        return n, 0, 1024
    if op == LK_OP_SUM_F32:
        return 4 * n, 0, 4
    if op == LK_OP_GEMM64_F32:
        return 16384 * n, 16384 * n, 16384 * n
    if op == LK_OP_COPY_I32:
        return 4 * n, 0, 4 * n
    if op == LK_OP_COMBINE_SUM:
        return (16 * (n - 1) + 4 if n else 0), 0, 4
    if op == LK_OP_COMBINE_HIST:
        return 1024 * n, 0, 1024
    if op == LK_OP_SPIN:
        return 0, 0, 4 * int(ctas)
    return 0, 0, 0


def _checked(x, need: int, what: str) -> int:
    """Device address of x.  A tensor (an object with is_cuda / numel /
    element_size) must live on a CUDA device, be contiguous and hold at least
    `need` bytes, else LkError(LK_EINVAL) before anything reaches the library.
    Plain ints are the caller's responsibility (the library checks alignment)."""
    if x is None or isinstance(x, int):
        return _ptr(x)
    if hasattr(x, "is_cuda") and hasattr(x, "numel"):
        if not x.is_cuda:
            raise LkError(LK_EINVAL, f"{what}: not a CUDA tensor")
        if not x.is_contiguous():
            raise LkError(LK_EINVAL, f"{what}: not contiguous")
        have = int(x.numel()) * int(x.element_size())
        if have < need:
            raise LkError(LK_EINVAL, f"{what}: holds {have} bytes, the operation touches {need}")
    return int(x.data_ptr())


def _operands(op: int, n: int, ins, out, ctas: int = 0) -> tuple:
    """(in0, in1, out) addresses, each tensor checked against op_bytes."""
    need = op_bytes(op, n, ctas)
    ins = tuple(ins or ())
    a = [_checked(ins[i], need[i] if i < 2 else 0, f"in{i}") for i in range(len(ins))]
    return a, _checked(out, need[2], "out")


def make_params(sizes, device: int = 0, smids=None, threads_per_cta: int = 256, ring_depth: int = 1024,
                backoff_base_ns: int = 0, backoff_cap_ns: int = 256, idle_lease_ns: int = 10_000_000_000,
                boot_timeout_ns: int = 10_000_000_000, exec_log_cap: int = 0, flags: int = 0,
                max_batch_units: int = 0, ctas_per_sm: int = 0, serve_units: int = 0):
    """lk_init_params plus the arrays it points to (kept alive by the tuple)."""
    sz = (ctypes.c_int * len(sizes))(*sizes)
    sm = None if smids is None else (ctypes.c_int * len(smids))(*smids)
    p = lk_init_params(device, len(sizes), sz, sm, threads_per_cta, ring_depth, backoff_base_ns, backoff_cap_ns,
                       idle_lease_ns, boot_timeout_ns, exec_log_cap, flags, max_batch_units, ctas_per_sm, serve_units)
    return p, (sz, sm)


# ---- the C ABI, one function each ---------------------------------------------------
class Context:
    """A running LightKernel context (owns an lk_ctx*)."""

    def __init__(self, sizes, fake: bool = False, bounds: bool = False, **kw):
        self.kernel_ms = -1.0
        self.lib = load(fake, bounds)
        self.sizes = list(sizes)
        self._params, self._keep = make_params(self.sizes, **kw)
        self.ptr = ctypes.c_void_p()
        rc = self.lib.lk_init(ctypes.byref(self.ptr), ctypes.byref(self._params))
        if rc != LK_OK:
            self.ptr = None
            raise LkError(rc, "lk_init")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.dispose()

    def __del__(self):
        try:
            self.dispose()
        except Exception:
            pass

    def dispose(self, timeout_ns: int = 20_000_000_000) -> int:
        if not self.ptr:
            return LK_OK
        ms = ctypes.c_float(-1.0)
        rc = self.lib.lk_dispose_timed(self.ptr, timeout_ns, ctypes.byref(ms))
        if rc != LK_EBUSY:
            self.ptr = None
            self.kernel_ms = ms.value
        return rc


def lk_init(sizes, fake: bool = False, **kw) -> Context:
    return Context(sizes, fake=fake, **kw)


def lk_submit(ctx: Context, cluster: int, op: int, n: int, ins=(), out=None, aux: int = 0) -> int | None:
    """Returns the handle, or None if the cluster's ring is full (LK_EAGAIN)."""
    d = lk_desc(op, 0, n, aux)
    ctas = ctx.sizes[cluster] if 0 <= cluster < len(ctx.sizes) else 0
    a, o = _operands(op, n, ins, out, ctas)
    arr = (ctypes.c_void_p * max(1, len(a)))(*a) if a else None
    h = ctypes.c_uint64()
    rc = ctx.lib.lk_submit(ctx.ptr, cluster, ctypes.byref(d), arr, len(a), o, ctypes.byref(h))
    if rc == LK_EAGAIN:
        return None
    if rc != LK_OK:
        raise LkError(rc, "lk_submit")
    return h.value


def lk_poll(ctx: Context, h: int) -> int:
    rc = ctx.lib.lk_poll(ctx.ptr, h)
    if rc < 0:
        raise LkError(rc, "lk_poll")
    return rc


def lk_wait(ctx: Context, h: int, timeout_ns: int = 10_000_000_000) -> int:
    rc = ctx.lib.lk_wait(ctx.ptr, h, timeout_ns)
    if rc not in (LK_OK, LK_ETIMEDOUT):
        raise LkError(rc, "lk_wait")
    return rc


def lk_sync(ctx: Context, timeout_ns: int = 10_000_000_000) -> int:
    rc = ctx.lib.lk_sync(ctx.ptr, timeout_ns)
    if rc not in (LK_OK, LK_ETIMEDOUT):
        raise LkError(rc, "lk_sync")
    return rc


def lk_heartbeat(ctx: Context) -> int:
    return ctx.lib.lk_heartbeat(ctx.ptr)


def lk_set_rate(ctx: Context, cluster: int, bytes_per_us: int) -> None:
    """Default load-rate cap of `cluster` (bytes per microsecond; 0 = none)."""
    rc = ctx.lib.lk_set_rate(ctx.ptr, cluster, bytes_per_us)
    if rc != LK_OK:
        raise LkError(rc, "lk_set_rate")


def lk_set_role(ctx: Context, cluster: int, role: int) -> None:
    """Role of `cluster` for load yielding: LK_ROLE_CRITICAL, LK_ROLE_YIELD or LK_ROLE_NONE."""
    rc = ctx.lib.lk_set_role(ctx.ptr, cluster, role)
    if rc != LK_OK:
        raise LkError(rc, "lk_set_role")


def lk_dispose(ctx: Context, timeout_ns: int = 20_000_000_000) -> int:
    return ctx.dispose(timeout_ns)


def lk_cluster_info(ctx: Context, cluster: int) -> list:
    cap = 1024
    buf = (ctypes.c_int * cap)()
    n = ctx.lib.lk_cluster_info(ctx.ptr, cluster, buf, cap)
    if n < 0:
        raise LkError(n, "lk_cluster_info")
    return list(buf[:n])


def lk_status(ctx: Context, cluster: int) -> int:
    rc = ctx.lib.lk_status(ctx.ptr, cluster)
    if rc < 0:
        raise LkError(rc, "lk_status")
    return rc


def lk_device_error(ctx: Context) -> int:
    return ctx.lib.lk_device_error(ctx.ptr)


def lk_num_sms(ctx: Context) -> int:
    return ctx.lib.lk_num_sms(ctx.ptr)


def lk_num_ctas(ctx: Context) -> int:
    return ctx.lib.lk_num_ctas(ctx.ptr)


def lk_exec_log(ctx: Context, cap: int | None = None):
    """Execution log as a numpy structured array (EXEC_REC_DTYPE) and the dropped count."""
    if cap is None:
        cap = max(1, sum(ctx.sizes) * max(1, ctx._params.exec_log_cap))
    buf = np.zeros(cap, dtype=EXEC_REC_DTYPE)
    n = ctypes.c_size_t()
    dropped = ctypes.c_uint64()
    rc = ctx.lib.lk_exec_log(ctx.ptr, buf.ctypes.data, cap, ctypes.byref(n), ctypes.byref(dropped))
    if rc != LK_OK:
        raise LkError(rc, "lk_exec_log")
    return buf[: n.value], dropped.value


def lk_strerror(code: int) -> str:
    return strerror(code)


def lk_run_finite(sizes, descs, cluster_of, in0=None, in1=None, out=None, log_cap: int = 0, fake: bool = False,
                  **kw):
    """Finite mode: one launch runs the listed descriptors and returns.
    descs: list of (op, n).  Returns (elapsed_ms, exec log array)."""
    lib = load(fake)
    p, keep = make_params(sizes, exec_log_cap=kw.pop("exec_log_cap", max(1, len(descs))), **kw)
    cnt = len(descs)
    D = (lk_desc * max(1, cnt))(*[lk_desc(op, 0, n, 0) for op, n in descs])
    C = (ctypes.c_int * max(1, cnt))(*cluster_of)

    def ctas_of(i):
        c = int(cluster_of[i])
        return sizes[c] if 0 <= c < len(sizes) else 0

    def arr(xs, k):
        if xs is None:
            return None
        return (ctypes.c_void_p * max(1, cnt))(
            *[_checked(x, op_bytes(descs[i][0], descs[i][1], ctas_of(i))[k] if i < cnt else 0, f"descriptor {i}")
              for i, x in enumerate(xs)])

    ms = ctypes.c_float(-1.0)
    logbuf = np.zeros(max(1, log_cap), dtype=EXEC_REC_DTYPE)
    ln = ctypes.c_size_t()
    rc = lib.lk_run_finite(ctypes.byref(p), D, C, arr(in0, 0), arr(in1, 1), arr(out, 2), cnt, ctypes.byref(ms),
                           logbuf.ctypes.data if log_cap else None, log_cap, ctypes.byref(ln))
    if rc != LK_OK:
        raise LkError(rc, "lk_run_finite")
    return ms.value, logbuf[: ln.value]


def lk_run_trace(ctx: Context, items: np.ndarray, n_threads: int, closed_loop: bool = False, pin_cpu_base: int = -1,
                 timeout_ns: int = 120_000_000_000, mode: int | None = None):
    items = np.ascontiguousarray(items, dtype=TRACE_ITEM_DTYPE)
    res = np.zeros(items.size, dtype=TRACE_RES_DTYPE)
    if mode is None:
        mode = LK_TRACE_CLOSED if closed_loop else LK_TRACE_OPEN
    rc = ctx.lib.lk_run_trace(ctx.ptr, items.ctypes.data, items.size, n_threads, mode, pin_cpu_base,
                              timeout_ns, res.ctypes.data)
    return rc, res


def lk_baseline_run_trace(items: np.ndarray, ctas_of_slot, threads: int, n_threads: int, device: int = 0,
                          pin_cpu_base: int = -1, mode: int = LK_TRACE_CLOSED):
    lib = load()
    items = np.ascontiguousarray(items, dtype=TRACE_ITEM_DTYPE)
    res = np.zeros(items.size, dtype=TRACE_RES_DTYPE)
    cs = (ctypes.c_int * len(ctas_of_slot))(*ctas_of_slot)
    rc = lib.lk_baseline_run_trace(device, items.ctypes.data, items.size, len(ctas_of_slot), cs, threads,
                                   n_threads, mode, pin_cpu_base, res.ctypes.data)
    return rc, res


def lk_bounds_violations(device: int = 0) -> tuple[int, int]:
    """(violations, first site) counted by the bounds-checking build since
    it was loaded.  Call it with no context running on the device."""
    lib = load(bounds=True)
    cnt, site = ctypes.c_uint64(), ctypes.c_uint32()
    rc = lib.lk_bounds_violations(device, ctypes.byref(cnt), ctypes.byref(site))
    if rc != LK_OK:
        raise LkError(rc, "lk_bounds_violations")
    return int(cnt.value), int(site.value)


def lk_pingpong(iters: int, device: int = 0) -> np.ndarray:
    lib = load()
    buf = (ctypes.c_uint64 * iters)()
    rc = lib.lk_pingpong(device, iters, buf)
    if rc != LK_OK:
        raise LkError(rc, "lk_pingpong")
    return np.frombuffer(buf, dtype=np.uint64).copy()


def lk_launch_noalloc(op: int, n: int, ins=(), out=None, ctas: int = 37, threads: int = 256, stream=None,
                      device: int = 0) -> int:
    """One ordinary launch that allocates nothing (see include/lk.h).  Returns
    without waiting; `stream` is a cudaStream_t as an int (torch:
    ``torch.cuda.current_stream().cuda_stream``) or None."""
    lib = load()
    d = lk_desc(op, 0, n, 0)
    a, o = _operands(op, n, ins, out, ctas)
    arr = (ctypes.c_void_p * max(1, len(a)))(*a) if a else None
    return lib.lk_launch_noalloc(device, ctypes.byref(d), arr, len(a), o, ctas, threads, stream or 0)


def batch_items(rows) -> np.ndarray:
    """rows: iterable of (op, n, ins, out[, parts]) with pointers as ints or tensors."""
    rows = list(rows)
    a = np.zeros(len(rows), dtype=BATCH_ITEM_DTYPE)
    for i, r in enumerate(rows):
        op, n, ins, out = r[:4]
        a[i]["op"], a[i]["n"] = op, n
        p, o = _operands(op, n, ins, out)
        a[i]["in0"] = p[0] if len(p) > 0 else 0
        a[i]["in1"] = p[1] if len(p) > 1 else 0
        a[i]["out"] = o
        a[i]["parts"] = r[4] if len(r) > 4 else 0
    return a


def lk_submit_batch(ctx: Context, cluster: int, items: np.ndarray, max_parts: int = 0, part_bytes: int = 0) -> int | None:
    """Post a batch (BATCH_ITEM_DTYPE array).  Returns the handle, or None if
    the ring or the batch tables are busy (LK_EAGAIN)."""
    items = np.ascontiguousarray(items, dtype=BATCH_ITEM_DTYPE)
    t = lk_batch_tune(max_parts, 0, part_bytes)
    h = ctypes.c_uint64()
    rc = ctx.lib.lk_submit_batch(ctx.ptr, cluster, items.ctypes.data if items.size else None, items.size,
                                 ctypes.byref(t), ctypes.byref(h))
    if rc == LK_EAGAIN:
        return None
    if rc != LK_OK:
        raise LkError(rc, "lk_submit_batch")
    return h.value


def lk_baseline_graph(items: np.ndarray, max_ctas: int, threads: int = 256, reps: int = 1, device: int = 0):
    """The batch as one CUDA graph of ordinary launches; returns per-repetition ms."""
    lib = load()
    items = np.ascontiguousarray(items, dtype=BATCH_ITEM_DTYPE)
    ms = (ctypes.c_float * reps)()
    rc = lib.lk_baseline_graph(device, items.ctypes.data if items.size else None, items.size, max_ctas, threads,
                               reps, ms)
    if rc != LK_OK:
        raise LkError(rc, "lk_baseline_graph")
    return np.frombuffer(ms, dtype=np.float32).copy()


def lk_serve(ctx: Context, reqs: np.ndarray, n_producers: int, budget_bytes: int, arena=None, arena_bytes: int = 0,
             window: int = 0, chunk_bytes: int = 0, timeout_ns: int = 0, coalesce_bytes: int = 0,
             coalesce_max: int = 0, coalesce_part_bytes: int = 0, mode: int = LK_SERVE_CHUNKS,
             max_inflight: int = 0, part_bytes: int = 0, min_part_bytes: int = 0):
    """Serve REQUEST_DTYPE requests; returns (rc, REQUEST_RES_DTYPE results).
    mode LK_SERVE_QUEUE runs them through the device-resident queue (the
    arena's first lk_serve_queue_state_bytes(max_inflight) bytes hold its
    state); LK_SERVE_CHUNKS through the host dispatcher."""
    reqs = np.ascontiguousarray(reqs, dtype=REQUEST_DTYPE)
    res = np.zeros(reqs.size, dtype=REQUEST_RES_DTYPE)
    prm = lk_serve_params(n_producers, window, chunk_bytes, budget_bytes, _ptr(arena) or None, arena_bytes, timeout_ns,
                          coalesce_bytes, coalesce_max, coalesce_part_bytes, mode, max_inflight, part_bytes,
                          min_part_bytes)
    rc = ctx.lib.lk_serve(ctx.ptr, reqs.ctypes.data if reqs.size else None, reqs.size, ctypes.byref(prm),
                          res.ctypes.data if reqs.size else None)
    return rc, res


def lk_serve_queue_state_bytes(max_inflight: int = 0) -> int:
    """Arena bytes the device queue's state takes (LK_SERVE_QUEUE)."""
    try:
        lib = load()
    except OSError:
        lib = load(True)
    return int(lib.lk_serve_queue_state_bytes(max_inflight))


PHASE_DTYPE = np.dtype([("init_ns", "<u8"), ("trigger_ns", "<u8"), ("wait_ns", "<u8"), ("dispose_ns", "<u8")])


def lk_phase_run(sms: int, iters: int, runs: int, threads: int = 256, out=None, device: int = 0, fake: bool = False):
    """The paper's life cycle on LK (Init/Trigger/Wait/Dispose per run)."""
    lib = load(fake)
    res = np.zeros(runs, dtype=PHASE_DTYPE)
    rc = lib.lk_phase_run(device, sms, threads, iters, runs, _ptr(out) or None, res.ctypes.data)
    if rc != LK_OK:
        raise LkError(rc, "lk_phase_run")
    return res


def lk_baseline_phase_run(sms: int, iters: int, runs: int, threads: int = 256, out=None, device: int = 0):
    """The traditional life cycle (Alloc/Spawn/Wait/Dispose per run)."""
    lib = load()
    res = np.zeros(runs, dtype=PHASE_DTYPE)
    rc = lib.lk_baseline_phase_run(device, sms, threads, iters, runs, _ptr(out) or None, res.ctypes.data)
    if rc != LK_OK:
        raise LkError(rc, "lk_baseline_phase_run")
    return res


def lk_serve_parts(op: int, n: int, ctas: int, backlog_units: int = 0, backlog_bytes: int = 0,
                   part_bytes: int = 0, min_part_bytes: int = 0) -> int:
    """Units the device queue gives a request (the split rule of include/lk.h); 0 if refused."""
    try:
        lib = load()
    except OSError:
        lib = load(True)
    return int(lib.lk_serve_parts(op, n, ctas, backlog_units, backlog_bytes, part_bytes, min_part_bytes))
