"""Build the native libraries in-tree (paper_2310_01212_gb300/_build/).

* liblk.so       the product: persistent kernel + host runtime, sm_103a only.
* liblk_fake.so  test build of the same host runtime over a host-thread
                 stand-in for the GPU (no CUDA needed to run it).

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


def build(force: bool = False, fake: bool = True, cuda: bool = True) -> None:
    os.makedirs(OUT, exist_ok=True)
    pid = os.getpid()
    cmds, moves = [], []
    need_cuda = cuda and (force or _stale(LIB))
    need_fake = fake and (force or _stale(FAKE))
    common = ["-O3", "-std=c++17", f"-I{INCLUDE}", f"-I{CSRC}"]
    if need_cuda:
        ko = os.path.join(OUT, f"lk_kernel.{pid}.o")
        ro = os.path.join(OUT, f"lk_runtime.{pid}.o")
        cmds.append([_nvcc(), "-gencode", GENCODE, "-lineinfo", *common, "-Xcompiler", "-fPIC",
                     "-c", os.path.join(CSRC, "lk_kernel.cu"), "-o", ko])
        cmds.append(["g++", *common, "-fPIC", "-Wall", "-c", os.path.join(CSRC, "lk_runtime.cpp"),
                     "-I/usr/local/cuda/include", "-o", ro])
    if need_fake:
        tmpf = FAKE + f".{pid}.tmp"
        cmds.append(["g++", *common, "-fPIC", "-Wall", "-shared", "-pthread",
                     os.path.join(CSRC, "lk_runtime.cpp"), os.path.join(CSRC, "lk_backend_fake.cpp"),
                     "-o", tmpf])
        moves.append((tmpf, FAKE))
    if cmds:
        _run_all(cmds)
    if need_cuda:
        tmp = LIB + f".{pid}.tmp"
        _run_all([[_nvcc(), "-gencode", GENCODE, "-shared", "-Xcompiler", "-fPIC", ko, ro,
                   "-lpthread", "-o", tmp]])
        moves.append((tmp, LIB))
        for o in (ko, ro):
            os.remove(o)
    for a, b in moves:
        os.replace(a, b)


if __name__ == "__main__":
    build(force=True)
    print(LIB)
