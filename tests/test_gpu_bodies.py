"""GPU parity of every work body against the oracle, through the C ABI:
bit-exact for integer work, within 1e-4 * sum|x| of binary64 for float32.
Sizes span several CTAs' shares, ragged tails and the empty case."""
import numpy as np
import pytest

from gpu_util import gemm_ok, host, need_gpu, sum_ok, to_dev
from paper_2310_01212_gb300 import lk, synth

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 3, 4, 5, 17, 1023, 4096, 65536 + 7, (1 << 20) + 13]
# (CTAs in the cluster, persistent CTAs per SM): two per SM halves every
# shared-memory region (streaming stages, histogram copies, GEMM stages)
SP = [(1, 1), (2, 1), (37, 1), (2, 2), (37, 2)]


@pytest.fixture(scope="module")
def torch_ready(native_built):
    return need_gpu()


@pytest.mark.parametrize("S,per_sm", SP)
def test_add_copy_bit_exact(torch_ready, oracle_lib, S, per_sm):
    torch = torch_ready
    cases = []
    for i, n in enumerate(SIZES):
        a = synth.int32_uniform(11, 2 * i, n, -(2**31), 2**31 - 1)
        b = synth.int32_uniform(11, 2 * i + 1, n, -(2**31), 2**31 - 1)
        cases.append((n, a, b, to_dev(a), to_dev(b), torch.zeros(max(n, 1), dtype=torch.int32, device="cuda"),
                      torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")))
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([S], idle_lease_ns=5_000_000_000, ctas_per_sm=per_sm) as c:
        hs = []
        for n, a, b, da, db, oa, oc in cases:
            hs.append(lk.lk_submit(c, 0, lk.LK_OP_ADD_I32, n, (da, db), oa))
            hs.append(lk.lk_submit(c, 0, lk.LK_OP_COPY_I32, n, (da,), oc))
        for h in hs:
            assert lk.lk_wait(c, h) == lk.LK_OK
    for n, a, b, da, db, oa, oc in cases:
        assert np.array_equal(host(oa)[:n], oracle_lib.add_i32(a, b)), n
        assert np.array_equal(host(oc)[:n], oracle_lib.copy_i32(a)), n


@pytest.mark.parametrize("S,per_sm", SP)
def test_hist_bit_exact(torch_ready, oracle_lib, S, per_sm):
    torch = torch_ready
    cases = []
    for i, n in enumerate(SIZES):
        x = synth.bytes_uniform(12, i, n)
        cases.append((x, to_dev(x) if n else torch.zeros(16, dtype=torch.uint8, device="cuda"),
                      torch.full((256,), -1, dtype=torch.int32, device="cuda")))
    # value v appears v+1 times (shuffled): every bin distinct
    x = np.concatenate([np.full(v + 1, v, np.uint8) for v in range(256)])
    x = x[synth.permutation(12, 99, x.size)]
    cases.append((x, to_dev(x), torch.full((256,), -1, dtype=torch.int32, device="cuda")))
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([S], idle_lease_ns=5_000_000_000, ctas_per_sm=per_sm) as c:
        hs = [lk.lk_submit(c, 0, lk.LK_OP_HIST_U8, x.size, (dx,), out) for x, dx, out in cases]
        for h in hs:
            assert lk.lk_wait(c, h) == lk.LK_OK
    for x, dx, out in cases:
        assert np.array_equal(host(out).astype(np.int64), oracle_lib.hist_u8(x)), x.size


@pytest.mark.parametrize("threads", [128, 256, 512, 1024])
def test_hist_block_sizes_and_skew(torch_ready, oracle_lib, threads):
    """Large shares stream through one ring per warp (its size depends on the
    block size): many laps of every warp's ring, ragged warp parts, and skewed
    inputs where the warps sharing a counter copy hit the same words."""
    torch = torch_ready
    n_big = (1 << 24) + 4099
    xs = [synth.bytes_uniform(14, 0, n_big),
          np.full(300_017, 201, np.uint8),                           # one bin only
          (synth.bytes_uniform(14, 1, 1_000_003) & 3).astype(np.uint8),   # four bins
          synth.bytes_uniform(14, 2, 16 * 1024 * 37 + 16)]          # just above the small-share cut
    cases = [(x, to_dev(x), torch.full((256,), -1, dtype=torch.int32, device="cuda")) for x in xs]
    torch.cuda.current_stream().synchronize()
    for sizes in ([1], [37]):
        for _, _, out in cases:
            out.fill_(-1)
        torch.cuda.current_stream().synchronize()
        with lk.lk_init(sizes, idle_lease_ns=5_000_000_000, threads_per_cta=threads) as c:
            hs = [lk.lk_submit(c, 0, lk.LK_OP_HIST_U8, x.size, (dx,), out) for x, dx, out in cases]
            for h in hs:
                assert lk.lk_wait(c, h) == lk.LK_OK
        for x, _, out in cases:
            assert np.array_equal(host(out).astype(np.int64), oracle_lib.hist_u8(x)), (sizes, x.size)


@pytest.mark.parametrize("S,per_sm", SP)
def test_sum_within_tolerance_and_exact_closed_form(torch_ready, oracle_lib, S, per_sm):
    torch = torch_ready
    cases = []
    for i, n in enumerate(SIZES):
        x = synth.normal_f32(13, i, n)
        cases.append((x, to_dev(x) if n else torch.zeros(4, device="cuda"), torch.full((4,), 7.0, device="cuda"), False))
    # integer-valued floats whose partial sums stay below 2^24: every order is exact
    for n in (100003, 65536):
        x = ((np.arange(n) % 7) - 3).astype(np.float32)
        cases.append((x, to_dev(x), torch.full((4,), 7.0, device="cuda"), True))
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([S], idle_lease_ns=5_000_000_000, ctas_per_sm=per_sm) as c:
        hs = [lk.lk_submit(c, 0, lk.LK_OP_SUM_F32, x.size, (dx,), out) for x, dx, out, _ in cases]
        for h in hs:
            assert lk.lk_wait(c, h) == lk.LK_OK
    for x, dx, out, exact in cases:
        got = float(host(out)[0])
        if exact:
            assert got == oracle_lib.sum_f32(x)
        else:
            assert sum_ok(got, x, oracle_lib), (x.size, got, oracle_lib.sum_f32(x))


@pytest.mark.parametrize("S,per_sm", SP)
def test_gemm_tiles(torch_ready, oracle_lib, S, per_sm):
    torch = torch_ready
    cases = []
    for i, t in enumerate([1, 2, 3, 5, 37, 100]):
        A = synth.normal_f32(14, 2 * i, t * 4096).reshape(t, 64, 64)
        B = synth.normal_f32(14, 2 * i + 1, t * 4096).reshape(t, 64, 64)
        cases.append((A, B, to_dev(A), to_dev(B), torch.zeros((t, 64, 64), device="cuda")))
    I = np.broadcast_to(np.eye(64, dtype=np.float32), (3, 64, 64)).copy()
    B = synth.normal_f32(14, 77, 3 * 4096).reshape(3, 64, 64)
    cases.append((I, B, to_dev(I), to_dev(B), torch.zeros((3, 64, 64), device="cuda")))
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([S], idle_lease_ns=5_000_000_000, ctas_per_sm=per_sm) as c:
        hs = [lk.lk_submit(c, 0, lk.LK_OP_GEMM64_F32, A.shape[0], (dA, dB), dC) for A, B, dA, dB, dC in cases]
        for h in hs:
            assert lk.lk_wait(c, h) == lk.LK_OK
    for A, B, dA, dB, dC in cases:
        assert gemm_ok(host(dC), A, B, oracle_lib), A.shape
    # identity tile: exact on the FFMA path (row blocks of split tiles, or two
    # CTAs per SM); whole tiles with one CTA per SM run on the tensor cores,
    # where B comes back as B_hi + B_lo, two bf16 parts rounded to nearest
    # (|err| <= 2^-17 |b| for the pair, plus the float32 rounding of the sum)
    got = host(cases[-1][4])
    if per_sm == 1 and S <= 3:
        assert np.all(np.abs(got - B) <= 2.0 ** -16 * np.abs(B)), np.max(np.abs(got - B) / np.abs(B))
    else:
        assert np.array_equal(got, B)


@pytest.mark.parametrize("S", [1, 5])
def test_gemm_ffma_flag(torch_ready, oracle_lib, S):
    """LK_INIT_GEMM_FFMA keeps whole tiles on the FFMA path: the identity tile
    is exact there, and both paths stay within the per-element bound."""
    torch = torch_ready
    t = 40
    A = synth.normal_f32(15, 1, t * 4096).reshape(t, 64, 64)
    B = synth.normal_f32(15, 2, t * 4096).reshape(t, 64, 64)
    I = np.broadcast_to(np.eye(64, dtype=np.float32), (t, 64, 64)).copy()
    dA, dB, dI = to_dev(A), to_dev(B), to_dev(I)
    outs = {f: (torch.zeros((t, 64, 64), device="cuda"), torch.zeros((t, 64, 64), device="cuda"))
            for f in (0, lk.LK_INIT_GEMM_FFMA)}
    torch.cuda.current_stream().synchronize()
    for f, (o_ab, o_ib) in outs.items():
        with lk.lk_init([S], idle_lease_ns=5_000_000_000, flags=f) as c:
            hs = [lk.lk_submit(c, 0, lk.LK_OP_GEMM64_F32, t, (dA, dB), o_ab),
                  lk.lk_submit(c, 0, lk.LK_OP_GEMM64_F32, t, (dI, dB), o_ib)]
            for h in hs:
                assert lk.lk_wait(c, h) == lk.LK_OK
    for f, (o_ab, o_ib) in outs.items():
        assert gemm_ok(host(o_ab), A, B, oracle_lib)
        if f:
            assert np.array_equal(host(o_ib), B)
        else:
            got = host(o_ib)
            assert np.all(np.abs(got - B) <= 2.0 ** -16 * np.abs(B))


@pytest.mark.parametrize("flags", [0, lk.LK_INIT_DIRECT, lk.LK_INIT_MAILBOX], ids=["relay", "direct", "mailbox"])
def test_histograms_into_one_output_leave_the_last(torch_ready, oracle_lib, flags):
    """Histogram descriptors posted back to back into one output (sizes from a
    few KB to 16 MiB, so the CTAs of one run behind the next) leave exactly
    the last one's bins: rank 0 clears the output only after the previous
    descriptor finished everywhere."""
    torch = torch_ready
    sizes = [1 << 24, 4099, 1 << 20, 123_457, 1 << 24, 77, 3 << 20]
    xs = [synth.bytes_uniform(17, i, n) for i, n in enumerate(sizes)]
    dx = [to_dev(x) for x in xs]
    out = torch.zeros(256, dtype=torch.int32, device="cuda")
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([37], flags=flags, idle_lease_ns=5_000_000_000) as c:
        for rep in range(3):
            hs = []
            for x, d in zip(xs, dx):
                h = None
                while h is None:   # the one-deep mailbox takes one descriptor at a time
                    h = lk.lk_submit(c, 0, lk.LK_OP_HIST_U8, x.size, (d,), out)
                hs.append(h)
            for h in hs:
                assert lk.lk_wait(c, h) == lk.LK_OK
            assert np.array_equal(host(out).astype(np.int64), oracle_lib.hist_u8(xs[-1])), rep


def test_gemm_row_blocks_bit_identical(torch_ready, oracle_lib):
    """On the FFMA path a tile's result does not depend on its split into row
    blocks: one tile on 1, 2, 3 and 8 CTAs (blocks of 64, 32, 16 and 8 rows,
    each with its own micro-tile shape) gives the same bits, within the
    per-element bound of the oracle."""
    torch = torch_ready
    A = synth.normal_f32(16, 1, 4096).reshape(1, 64, 64)
    B = synth.normal_f32(16, 2, 4096).reshape(1, 64, 64)
    dA, dB = to_dev(A), to_dev(B)
    sizes = [1, 2, 3, 8]
    outs = [torch.zeros((1, 64, 64), device="cuda") for _ in sizes]
    torch.cuda.current_stream().synchronize()
    with lk.lk_init(sizes, idle_lease_ns=5_000_000_000, flags=lk.LK_INIT_GEMM_FFMA) as c:
        hs = [lk.lk_submit(c, i, lk.LK_OP_GEMM64_F32, 1, (dA, dB), o) for i, o in enumerate(outs)]
        for h in hs:
            assert lk.lk_wait(c, h) == lk.LK_OK
    got = [host(o) for o in outs]
    assert gemm_ok(got[0], A, B, oracle_lib)
    for g in got[1:]:
        assert np.array_equal(g, got[0])


def test_misaligned_pointers_rejected_on_host(torch_ready):
    torch = torch_ready
    x = torch.zeros(1024, dtype=torch.int32, device="cuda")
    with lk.lk_init([1], idle_lease_ns=5_000_000_000) as c:
        with pytest.raises(lk.LkError) as e:
            lk.lk_submit(c, 0, lk.LK_OP_COPY_I32, 16, (x.data_ptr() + 4,), x)
        assert e.value.code == lk.LK_EINVAL
        h = lk.lk_submit(c, 0, lk.LK_OP_NOP, 0)
        assert lk.lk_wait(c, h) == lk.LK_OK


def test_short_or_host_tensors_rejected_before_the_call(torch_ready):
    """The binding compares each tensor's numel * element_size with the bytes
    the operation touches; nothing reaches the GPU when one is short."""
    torch = torch_ready
    x = torch.arange(1000, dtype=torch.int32, device="cuda")
    xh = x.cpu()
    out = torch.full((1000,), -1, dtype=torch.int32, device="cuda")
    untouched = torch.full((1000,), -1, dtype=torch.int32, device="cuda")
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([2], idle_lease_ns=5_000_000_000) as c:
        for args in [(1001, (x,), untouched), (1000, (x,), untouched[:996]), (1000, (xh,), untouched),
                     (500, (x[::2],), untouched)]:
            with pytest.raises(lk.LkError) as e:
                lk.lk_submit(c, 0, lk.LK_OP_COPY_I32, *args)
            assert e.value.code == lk.LK_EINVAL
        assert lk.lk_wait(c, lk.lk_submit(c, 0, lk.LK_OP_COPY_I32, 1000, (x,), out)) == lk.LK_OK
    assert np.array_equal(host(out), host(x))
    assert np.all(host(untouched) == -1)        # none of the rejected calls ran


def test_sum_is_identical_alone_and_in_the_mix(torch_ready, oracle_lib):
    """The split depends only on (n, cluster size): a result does not depend on
    what else ran before or beside it."""
    torch = torch_ready
    x = synth.normal_f32(15, 1, 262144)
    dx = to_dev(x)
    outs = [torch.zeros(4, device="cuda") for _ in range(3)]
    noise = to_dev(synth.int32_uniform(15, 2, 1 << 22, -100, 100))
    nout = torch.zeros(1 << 22, dtype=torch.int32, device="cuda")
    torch.cuda.current_stream().synchronize()
    with lk.lk_init([16, 16], idle_lease_ns=5_000_000_000) as c:
        lk.lk_wait(c, lk.lk_submit(c, 0, lk.LK_OP_SUM_F32, x.size, (dx,), outs[0]))
        hs = [lk.lk_submit(c, 1, lk.LK_OP_ADD_I32, 1 << 22, (noise, noise), nout) for _ in range(4)]
        h1 = lk.lk_submit(c, 0, lk.LK_OP_SUM_F32, x.size, (dx,), outs[1])
        hs += [lk.lk_submit(c, 1, lk.LK_OP_COPY_I32, 1 << 22, (noise,), nout) for _ in range(4)]
        h2 = lk.lk_submit(c, 0, lk.LK_OP_SUM_F32, x.size, (dx,), outs[2])
        for h in hs + [h1, h2]:
            assert lk.lk_wait(c, h) == lk.LK_OK
    v = [host(o)[0] for o in outs]
    assert v[0] == v[1] == v[2]
    assert sum_ok(v[0], x, oracle_lib)


def test_finite_mode_bodies(torch_ready, oracle_lib):
    torch = torch_ready
    n = 300007
    a = synth.int32_uniform(16, 1, n, -(2**20), 2**20)
    b = synth.int32_uniform(16, 2, n, -(2**20), 2**20)
    x = synth.normal_f32(16, 3, n)
    da, db, dx = to_dev(a), to_dev(b), to_dev(x)
    oa = torch.zeros(n, dtype=torch.int32, device="cuda")
    os_ = torch.zeros(4, device="cuda")
    torch.cuda.current_stream().synchronize()
    ms, log = lk.lk_run_finite([3, 2], [(lk.LK_OP_ADD_I32, n), (lk.LK_OP_SUM_F32, n)], [0, 1],
                               in0=[da, dx], in1=[db, None], out=[oa, os_], log_cap=64)
    assert ms > 0
    assert np.array_equal(host(oa), oracle_lib.add_i32(a, b))
    assert sum_ok(host(os_)[0], x, oracle_lib)
    assert sorted(log["cluster"].tolist()) == [0, 0, 0, 1, 1]
