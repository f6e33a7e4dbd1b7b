"""Build the native libraries in-tree (paper_2310_01212_gb300/_build/).

* liblk.so       the product: persistent kernel + host runtime, sm_103a only.
* liblk_fake.so  test build of the same host runtime over a host-thread
                 stand-in for the GPU (no CUDA needed to run it).
* liblk_bounds.so  test build of liblk.so with -DLK_DEBUG_BOUNDS: every body
                 checks its indexes and addresses and skips an access that
                 would leave its operand or region (lk_bounds_violations).

nvcc compiles the CUDA translation unit while g++ compiles the host runtime,
in parallel; nothing here uses cmake.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(OUT, "liblk.so")
BOUNDS = os.path.join(OUT, "liblk_bounds.so")
FAKE = os.path.join(OUT, "liblk_fake.so")
GENCODE = "arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _sources():
    names = [f for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".cpp", ".h"))]
    return [os.path.join(CSRC, f) for f in names] + [os.path.join(INCLUDE, "lk.h"), __file__]


def _stale(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run_all(cmds):
    procs = [(c, subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)) for c in cmds]
    errs = []
    for c, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errs.append(" ".join(c) + "\n" + out)
    if errs:
        raise RuntimeError("native build failed:\n" + "\n".join(errs))


def build(force: bool = False, fake: bool = True, cuda: bool = True, bounds: bool = True) -> None:
    os.makedirs(OUT, exist_ok=True)
    pid = os.getpid()
    cmds, moves = [], []
    need_cuda = cuda and (force or _stale(LIB))
    need_fake = fake and (force or _stale(FAKE))
    need_bounds = cuda and bounds and (force or _stale(BOUNDS))
    common = ["-O3", "-std=c++17", f"-I{INCLUDE}", f"-I{CSRC}"]
    ro = os.path.join(OUT, f"lk_runtime.{pid}.o")
    if need_cuda or need_bounds:
        cmds.append(["g++", *common, "-fPIC", "-Wall", "-c", os.path.join(CSRC, "lk_runtime.cpp"),
                     "-I/usr/local/cuda/include", "-o", ro])
    if need_cuda:
        ko = os.path.join(OUT, f"lk_kernel.{pid}.o")
        cmds.append([_nvcc(), "-gencode", GENCODE, "-lineinfo", *common, "-Xcompiler", "-fPIC",
                     "-c", os.path.join(CSRC, "lk_kernel.cu"), "-o", ko])
    if need_bounds:
        kbo = os.path.join(OUT, f"lk_kernel_bounds.{pid}.o")
        cmds.append([_nvcc(), "-gencode", GENCODE, "-lineinfo", "-DLK_DEBUG_BOUNDS", *common, "-Xcompiler",
                     "-fPIC", "-c", os.path.join(CSRC, "lk_kernel.cu"), "-o", kbo])
    if need_fake:
        tmpf = FAKE + f".{pid}.tmp"
        cmds.append(["g++", *common, "-fPIC", "-Wall", "-shared", "-pthread",
                     os.path.join(CSRC, "lk_runtime.cpp"), os.path.join(CSRC, "lk_backend_fake.cpp"),
                     "-o", tmpf])
        moves.append((tmpf, FAKE))
    if cmds:
        _run_all(cmds)
    links = []
    if need_cuda:
        links.append((ko, LIB))
    if need_bounds:
        links.append((kbo, BOUNDS))
    if links:
        _run_all([[_nvcc(), "-gencode", GENCODE, "-shared", "-Xcompiler", "-fPIC", k, ro, "-lpthread", "-o",
                   out + f".{pid}.tmp"] for k, out in links])
        for k, out in links:
            moves.append((out + f".{pid}.tmp", out))
            os.remove(k)
        os.remove(ro)
    for a, b in moves:
        os.replace(a, b)


if __name__ == "__main__":
    build(force=True)
    print(LIB)
