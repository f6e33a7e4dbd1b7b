"""The compute-bound loop of Sec. III on the GPU (persistent kernel and
ordinary launch) against the oracle's jump-ahead closed form."""
import numpy as np
import pytest

from gpu_util import host, need_gpu
from paper_2310_01212_gb300 import lk

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_ready(native_built):
    return need_gpu()


@pytest.mark.parametrize("S,iters,threads", [(1, 20000, 256), (3, 1, 128), (8, 0, 256), (37, 5000, 512), (5, 7, 256), (2, 9, 1024), (6, 20003, 256)])
def test_spin_matches_closed_form(torch_ready, oracle_lib, S, iters, threads):
    torch = torch_ready
    out = torch.zeros(S, dtype=torch.int32, device="cuda")
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([S], threads_per_cta=threads, idle_lease_ns=5_000_000_000) as c:
        assert lk.lk_wait(c, lk.lk_submit(c, 0, lk.LK_OP_SPIN, iters, (), out)) == lk.LK_OK
        assert lk.lk_wait(c, lk.lk_submit(c, 0, lk.LK_OP_SPIN, iters, (), None)) == lk.LK_OK   # out optional
    got = host(out).view(np.uint32)
    want = [oracle_lib.spin_xor(r, threads, iters) for r in range(S)]
    assert got.tolist() == want


def test_phase_runs_compute_the_same(torch_ready, oracle_lib):
    torch = torch_ready
    a = torch.zeros(4, dtype=torch.int32, device="cuda")
    b = torch.zeros(4, dtype=torch.int32, device="cuda")
    torch.cuda.current_stream().synchronize()
    t_lk = lk.lk_phase_run(sms=4, iters=20005, runs=3, out=a)
    t_cu = lk.lk_baseline_phase_run(sms=4, iters=20005, runs=3, out=b)
    want = [oracle_lib.spin_xor(r, 256, 20005) for r in range(4)]
    assert host(a).view(np.uint32).tolist() == want
    assert host(b).view(np.uint32).tolist() == want
    assert np.all(t_lk["wait_ns"] > 0) and np.all(t_cu["wait_ns"] > 0)
