"""The bounds-checking build (liblk_bounds.so, compiled with -DLK_DEBUG_BOUNDS):
every body checks each index and address against its operand, its share and
its shared-memory or TMEM region before the access.  Run through the
persistent kernel over every share shape and layout (one and two CTAs per SM,
128 to 512 threads, the three histogram paths, both GEMM paths, a batch), no
check fails and every result still matches the oracle."""
import pytest

from gpu_util import need_gpu
from paper_2310_01212_gb300 import lk
from test_gpu_batch import MIX, _check, _make

pytestmark = pytest.mark.gpu

# (cluster sizes, CTAs per SM, threads per CTA)
LAYOUTS = [([1], 1, 256), ([37], 1, 256), ([3, 2], 2, 256), ([5], 1, 512), ([3], 1, 128)]
BODIES = ([(lk.LK_OP_ADD_I32, n, 0) for n in (1, 5, 4099, (1 << 20) + 13)]
          + [(lk.LK_OP_COPY_I32, n, 0) for n in (3, 65543)]
          + [(lk.LK_OP_SUM_F32, n, 0) for n in (0, 1027, (1 << 20) + 13)]
          + [(lk.LK_OP_HIST_U8, n, 0) for n in (100, 65543, (1 << 20) + 13, (1 << 22) + 5)]
          + [(lk.LK_OP_GEMM64_F32, t, 0) for t in (1, 3, 40)])


@pytest.fixture(scope="module")
def torch_ready(native_built):
    return need_gpu()


@pytest.mark.parametrize("sizes,per_sm,threads", LAYOUTS)
def test_every_body_within_bounds(torch_ready, oracle_lib, sizes, per_sm, threads):
    torch = torch_ready
    rows, refs = _make(torch, 51, BODIES)
    torch.cuda.current_stream().synchronize()
    with lk.lk_init(sizes, bounds=True, idle_lease_ns=5_000_000_000, ctas_per_sm=per_sm,
                    threads_per_cta=threads) as c:
        hs = [lk.lk_submit(c, i % len(sizes), op, n, ins, out) for i, (op, n, ins, out, _) in enumerate(rows)]
        for h in hs:
            rc = lk.lk_wait(c, h)
            assert rc == lk.LK_OK, (lk.lk_strerror(rc), lk.lk_device_error(c))
    _check(oracle_lib, rows, refs)
    assert lk.lk_bounds_violations() == (0, 0)


def test_batch_within_bounds(torch_ready, oracle_lib):
    torch = torch_ready
    rows, refs = _make(torch, 52, MIX)
    items = lk.batch_items(rows)
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([37], bounds=True, idle_lease_ns=5_000_000_000) as c:
        h = lk.lk_submit_batch(c, 0, items, part_bytes=1 << 20)
        assert lk.lk_wait(c, h) == lk.LK_OK
    _check(oracle_lib, rows, refs)
    assert lk.lk_bounds_violations() == (0, 0)
