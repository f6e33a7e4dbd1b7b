"""The C ABI library loads on a machine without a GPU, exports every function
include/lk.h declares, and its struct layouts match the Python binding.  No
compute call is made here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lk.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lk_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lk_init", "lk_submit", "lk_poll", "lk_wait", "lk_dispose", "lk_cluster_info", "lk_exec_log",
                 "lk_strerror", "lk_run_finite", "lk_run_trace", "lk_baseline_run_trace", "lk_pingpong"):
        assert must in names


@pytest.mark.parametrize("fake,bounds", [(False, False), (True, False), (False, True)])
def test_library_exports_every_declared_symbol(native_built, fake, bounds):
    from paper_2310_01212_gb300 import lk

    lib = ctypes.CDLL(lk.library_path(fake, bounds))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_product_build_checks_no_bounds(native_built):
    # lk_bounds_violations answers only in liblk_bounds.so; the product
    # library refuses it without touching the device
    from paper_2310_01212_gb300 import lk

    lib = lk.load()
    cnt, site = ctypes.c_uint64(), ctypes.c_uint32()
    assert lib.lk_bounds_violations(0, ctypes.byref(cnt), ctypes.byref(site)) == lk.LK_EINVAL


def test_strerror_without_gpu(native_built):
    from paper_2310_01212_gb300 import lk

    lib = lk.load()
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert lib.lk_strerror(code).decode().startswith("LK_")


def test_struct_layouts_match_binding(native_built, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "lk.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\\n", sizeof(lk_init_params), sizeof(lk_desc), sizeof(lk_exec_rec),
         sizeof(lk_trace_item), sizeof(lk_trace_result));
  printf("%zu %zu %zu %zu\\n", offsetof(lk_exec_rec, order), offsetof(lk_exec_rec, t_done_ns),
         offsetof(lk_trace_item, in0), offsetof(lk_init_params, exec_log_cap));
  printf("%zu %zu %zu %zu\\n", sizeof(lk_serve_params), offsetof(lk_serve_params, mode),
         offsetof(lk_serve_params, part_bytes), offsetof(lk_init_params, serve_units));
  return 0;
}
""")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-std=c11", f"-I{ROOT}/include", str(src), "-o", str(exe)])
    l1, l2, l3 = subprocess.check_output([str(exe)], text=True).split("\n")[:3]
    from paper_2310_01212_gb300 import lk

    assert [int(x) for x in l1.split()] == [ctypes.sizeof(lk.lk_init_params), ctypes.sizeof(lk.lk_desc),
                                           lk.EXEC_REC_DTYPE.itemsize, lk.TRACE_ITEM_DTYPE.itemsize,
                                           lk.TRACE_RES_DTYPE.itemsize]
    assert [int(x) for x in l2.split()] == [lk.EXEC_REC_DTYPE.fields["order"][1],
                                           lk.EXEC_REC_DTYPE.fields["t_done_ns"][1],
                                           lk.TRACE_ITEM_DTYPE.fields["in0"][1],
                                           lk.lk_init_params.exec_log_cap.offset]
    assert [int(x) for x in l3.split()] == [ctypes.sizeof(lk.lk_serve_params), lk.lk_serve_params.mode.offset,
                                           lk.lk_serve_params.part_bytes.offset, lk.lk_init_params.serve_units.offset]


def test_cuda_library_targets_sm_103a_only(native_built):
    # the build uses one -gencode, sm_103a; the binding fails loudly without it
    from paper_2310_01212_gb300 import build

    assert build.GENCODE == "arch=compute_103a,code=sm_103a"
    assert os.path.exists(build.LIB)
