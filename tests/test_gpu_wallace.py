"""GPU parity: the CUDA path against the FP64 oracle, through the C ABI.

Integer work (seeding, draws, index choice, how many draws each call
consumes) must agree bit for bit; FP32 values within the error model of
tests/_parity.py; 16-bit outputs are the round-to-nearest conversion of the
FP32 values.
"""
import math

import numpy as np
import pytest

import oracle
from _parity import (F16_MIN_NORMAL, U, U_BF16, U_F16, assert_fp32_close, passes_fresh)

pytestmark = pytest.mark.gpu

MASK64 = (1 << 64) - 1
WEYL = 0x61C8864680B583EB


@pytest.fixture(scope="module")
def torch():
    import torch as t
    return t


def _gen(wn, torch, h, count, dtype=0):
    tdt = {0: torch.float32, 1: torch.bfloat16, 2: torch.float16}[dtype]
    out = torch.empty(count * h.n, dtype=tdt, device="cuda")
    wn.wn_generate_ex(out, count, h, dtype)
    torch.cuda.synchronize()
    return out


def _expected_words(seed, n_draws):
    """(xorshift, Weyl) words after n_draws draws, from the oracle's draws."""
    s1, _ = oracle.splitmix64(seed)
    _, w0 = oracle.splitmix64(s1)
    w = (w0 + n_draws * WEYL) & MASK64
    last = int(oracle.draws(seed, n_draws)[-1])
    return (last - w) & MASK64, w


@pytest.mark.parametrize("seed", [0, 1, 2, 12345, MASK64])
def test_rng_draws_bit_exact(wn, seed):
    assert np.array_equal(wn.wn_rng_draws(seed, 3000), oracle.draws(seed, 3000))


@pytest.mark.parametrize("N", [4, 8, 32, 1024, 4096, 16384])
def test_init_pool_is_fp32_rounding_of_oracle(wn, N):
    seed = 1000 + N
    h = wn.wn_create_streams([N], [2], [seed], warmup_blocks=0)
    got = wn.wn_get_pool(h, 0, N)
    ref = oracle.Stream(N, 2, seed, warmup=0)
    assert np.array_equal(got, ref.pool.astype(np.float32))
    st = wn.wn_get_state(h, 0)
    assert (st["x"], st["w"]) == ref.gen_state
    assert st["k"] == N - 1 and st["blocks"] == 0 and st["r"] == 0.0


CASES = [(4, 1), (4, 3), (8, 2), (16, 1), (64, 2), (256, 4), (1024, 1), (1024, 2),
         (2048, 3), (4096, 2), (8192, 1), (16384, 3), (64, 64)]


@pytest.mark.parametrize("N,R", CASES)
def test_generate_matches_oracle(wn, torch, N, R):
    seed = 7 * N + R
    count = 5 * (N - 1) + 7  # several blocks and a ragged tail
    h = wn.wn_create(N, R, seed)
    got = _gen(wn, torch, h, count).cpu().numpy()
    ref_s = oracle.Stream(N, R, seed)
    ref = ref_s.generate(count)
    assert_fp32_close(got, ref, passes_fresh(count, N, R), f"N={N} R={R}")
    st = wn.wn_get_state(h, 0)
    assert (st["x"], st["w"]) == ref_s.gen_state
    assert st["k"] == ref_s.k and st["blocks"] == ref_s.blocks
    assert abs(st["r"] - ref_s.r) < C_R(ref_s, N, R)
    # the pool, in the library's scaling, is the oracle's renormalised pool
    pool = wn.wn_get_pool(h, 0, N).astype(np.float64)
    pool *= math.sqrt(N / float(np.sum(pool * pool)))
    assert_fp32_close(pool, ref_s.pool, R * ref_s.blocks, "pool")


def C_R(ref_s, N, R):
    return 10 * U * math.sqrt(R * ref_s.blocks) * (1 + abs(ref_s.r))


def test_continuation_is_bit_exact_and_matches_oracle(wn, torch):
    N, R, seed = 1024, 2, 99
    chunks = [1, 1021, 0, 1, 1023, 5000, 3, 2046, 777]
    total = sum(chunks)
    whole = _gen(wn, torch, wn.wn_create(N, R, seed), total).cpu().numpy()
    h = wn.wn_create(N, R, seed)
    parts = [(_gen(wn, torch, h, c).cpu().numpy() if c else np.empty(0, np.float32)) for c in chunks]
    assert np.array_equal(np.concatenate(parts), whole)
    ref = oracle.Stream(N, R, seed).generate(total)
    assert_fp32_close(whole, ref, passes_fresh(total, N, R))


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("Ns,Rs,half", [([1024, 4096, 64], [2, 2, 3], 50_001),
                                         ([64] * 4096, [2] * 4096, 20_000),
                                         ([1024] * 64, [2] * 64, 1 << 21),
                                         ([4096, 1024], [2, 1], (1 << 26) + 8)])
def test_generate_host_equals_device_path(wn, torch, Ns, Rs, half, pinned):
    # every route to host memory gives the device path's values: pinned
    # memory is written by the kernel directly; pageable memory is staged --
    # 4096 x 20000 x 4 B (> 256 MiB) in two groups of consecutive streams,
    # 64 x 2^21 x 4 B in groups of 32 streams, and 2 x (2^26 + 8) x 4 B (each
    # stream's part above 256 MiB) in rounds of per-stream chunks with pitched
    # copies
    n = len(Ns)
    seeds = list(range(5, 5 + n))
    dev = _gen(wn, torch, wn.wn_create_streams(Ns, Rs, seeds), 2 * half).cpu().view(n, 2 * half)
    h = wn.wn_create_streams(Ns, Rs, seeds)
    host = torch.empty(n * half, dtype=torch.float32, pin_memory=pinned)
    for c in range(2):  # consecutive calls continue each stream's sequence
        wn.wn_generate_host(host, half, h)
        torch.cuda.synchronize()
        assert torch.equal(host.view(n, half), dev[:, c * half:(c + 1) * half])


def test_count_zero_changes_nothing(wn, torch):
    h = wn.wn_create(64, 2, 5)
    before = wn.wn_get_state(h, 0)
    wn.wn_generate_ex(torch.empty(1, device="cuda"), 0, h)
    assert wn.wn_get_state(h, 0) == before


def test_single_stream_full_size(wn, torch):
    # N = 1024 pool, R = 2, seed 1, 2^24 FP32 values in one call
    N, R, seed, count = 1024, 2, 1, 1 << 24
    got = _gen(wn, torch, wn.wn_create(N, R, seed), count).cpu().numpy()
    ref = oracle.Stream(N, R, seed).generate(count)
    rms, mx = assert_fp32_close(got, ref, passes_fresh(count, N, R), "single stream 2^24")
    n = count
    x = got.astype(np.float64)
    assert abs(x.mean()) < 5 / math.sqrt(n)
    assert abs(x.var() - 1) < 5 * math.sqrt(2 / n)


def test_heterogeneous_streams_in_one_launch(wn, torch):
    Ns, Rs, seeds = [4, 1024, 16384, 64, 8], [1, 2, 3, 4, 2], [11, 12, 13, 14, 15]
    h = wn.wn_create_streams(Ns, Rs, seeds)
    count = 40000
    got = _gen(wn, torch, h, count).cpu().numpy().reshape(len(Ns), count)
    for i, (N, R, s) in enumerate(zip(Ns, Rs, seeds)):
        ref = oracle.Stream(N, R, s).generate(count)
        assert_fp32_close(got[i], ref, passes_fresh(count, N, R), f"stream {i}")


def test_many_streams_full_size(wn, torch):
    # 4096 streams (one per CTA), pool 4096, R = 2, seeds 1..4096, 2^20 each
    n, N, R, per = 4096, 4096, 2, 1 << 20
    h = wn.wn_create_streams([N] * n, [R] * n, list(range(1, n + 1)))
    out = torch.empty(n * per, dtype=torch.float32, device="cuda")
    wn.wn_generate(out, per, h)
    torch.cuda.synchronize()
    view = out.view(n, per)
    # sampled streams: every value against the oracle
    for i in (0, 1, 777, 2048, 4095):
        ref = oracle.Stream(N, R, i + 1).generate(per)
        assert_fp32_close(view[i].cpu().numpy(), ref, passes_fresh(per, N, R), f"stream {i}")
    # every stream's integer state: draws consumed = N + 2R (W + blocks)
    blocks = -(-per // (N - 1))
    for i in range(n):
        st = wn.wn_get_state(h, i) if i % 64 == 0 else None
        if st is None:
            continue
        assert (st["x"], st["w"]) == _expected_words(i + 1, N + 2 * R * (8 + blocks))
        assert st["blocks"] == 8 + blocks and st["k"] == per - (blocks - 1) * (N - 1)
    # moments over all 2^32 values
    s1 = s2 = s4 = 0.0
    for c in out.split(1 << 27):
        d = c.double()
        s1 += float(d.sum())
        s2 += float((d * d).sum())
        s4 += float((d * d * d * d).sum())
    tot = n * per
    m, v = s1 / tot, s2 / tot - (s1 / tot) ** 2
    assert abs(m) < 5 / math.sqrt(tot)
    assert abs(v - 1) < 5 * math.sqrt(2 / tot)
    assert abs(s4 / tot / v ** 2 - 3) < 5 * math.sqrt(24 / tot)


def test_generator_state_all_streams(wn):
    # bit-exact generator words of every stream of a 4096-stream handle
    n, N, R = 4096, 4096, 2
    h = wn.wn_create_streams([N] * n, [R] * n, list(range(1, n + 1)))
    for i in range(0, n, 97):
        st = wn.wn_get_state(h, i)
        assert (st["x"], st["w"]) == _expected_words(i + 1, N + 2 * R * 8)


@pytest.mark.parametrize("dtype", [1, 2])
def test_16bit_outputs_round_fp32_values(wn, torch, dtype):
    N, R, seed, count = 4096, 3, 21, 3 * 4095 + 11
    f32 = _gen(wn, torch, wn.wn_create(N, R, seed), count)
    low = _gen(wn, torch, wn.wn_create(N, R, seed), count, dtype)
    assert torch.equal(low, f32.to(low.dtype))
    ref = oracle.Stream(N, R, seed).generate(count)
    got = low.float().cpu().numpy().astype(np.float64)
    P = passes_fresh(count, N, R)
    if dtype == 1:
        tol = U_BF16 * np.abs(ref) + 10 * U * np.sqrt(P) * (1 + np.abs(ref))
    else:
        tol = U_F16 * np.abs(ref) + U_F16 * F16_MIN_NORMAL + 10 * U * np.sqrt(P) * (1 + np.abs(ref))
    assert np.all(np.abs(got - ref) <= tol)


def test_boxmuller_matches_oracle(wn, torch):
    count, n, seed = 4099, 3, 7
    out = torch.empty(count * n, dtype=torch.float32, device="cuda")
    wn.wn_boxmuller(out, count, n, seed)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(n, count).astype(np.float64)
    for i in range(n):
        ref = oracle.boxmuller(seed, i, 0, count)
        # FP32 log, sqrt, sincospi: a few ulps of values up to ~5.8
        assert np.all(np.abs(got[i] - ref) <= 8 * U * (1 + np.abs(ref))), i


def test_boxmuller_16bit(wn, torch):
    count, n, seed = 4096, 2, 3
    f32 = torch.empty(count * n, dtype=torch.float32, device="cuda")
    b16 = torch.empty(count * n, dtype=torch.bfloat16, device="cuda")
    wn.wn_boxmuller(f32, count, n, seed)
    wn.wn_boxmuller(b16, count, n, seed, dtype=1)
    torch.cuda.synchronize()
    assert torch.equal(b16, f32.to(torch.bfloat16))


def test_argument_errors(wn, torch):
    h = wn.wn_create(64, 2, 1)
    buf = torch.empty(1024, device="cuda")
    with pytest.raises(wn.WnError):
        wn.wn_generate_ex(buf[1:].data_ptr(), 10, h)  # not 16-byte aligned
    with pytest.raises(wn.WnError):
        wn.wn_generate_ex(buf.data_ptr(), 10, h, 7)  # unknown dtype, rejected by the C ABI
    with pytest.raises(wn.WnError):
        wn.wn_create(48, 2, 1)
    with pytest.raises(wn.WnError):
        wn.wn_create_streams([64, 64], [2, 0], [1, 2])


# (quadruples per thread, compute threads): full shapes cover the pool
# exactly, the others leave quadruple slots idle
SHAPES = {4096: [(2, 512), (4, 256), (8, 128), (8, 512), (16, 256)],
          16384: [(8, 512), (16, 256)],
          1024: [(1, 256), (1, 512), (2, 128), (4, 64), (8, 32), (16, 32)]}


@pytest.mark.parametrize("N", sorted(SHAPES))
def test_every_launch_shape_matches_oracle(wn, torch, N):
    # several streams and a count that is not a multiple of 4, so stream
    # outputs start at every alignment; every shape must give the oracle's
    # values within tolerance and the same integer state
    R, n = 2, 5
    count = 3 * (N - 1) + 6
    seeds = [40 + i for i in range(n)]
    refs = [oracle.Stream(N, R, s).generate(count) for s in seeds]
    words = None
    for qt, threads in SHAPES[N]:
        h = wn.wn_create_streams([N] * n, [R] * n, seeds)
        wn.wn_set_config(h, qt, threads)
        assert wn.wn_get_config(h) == (qt, threads)
        got = _gen(wn, torch, h, count).cpu().numpy().reshape(n, count)
        for i in range(n):
            assert_fp32_close(got[i], refs[i], passes_fresh(count, N, R), f"shape {qt}x{threads} stream {i}")
        w = [(wn.wn_get_state(h, i)["x"], wn.wn_get_state(h, i)["w"]) for i in range(n)]
        assert words is None or w == words
        words = w


def test_rejects_uncompiled_shape(wn):
    h = wn.wn_create(4096, 2, 1)
    with pytest.raises(wn.WnError):
        wn.wn_set_config(h, 4, 128)   # 512 quadruples < 1024
    with pytest.raises(wn.WnError):
        wn.wn_set_config(h, 3, 512)
    wn.wn_set_config(h, 0, 0)
    assert wn.wn_get_config(h) == (4, 256)  # a lone stream's default: the chain mode, 8 compute warps


def test_autotune_keeps_sequence_and_matches_oracle(wn, torch):
    N, R, n, count = 4096, 2, 64, 3 * 4095 + 10
    seeds = list(range(300, 300 + n))
    h = wn.wn_create_streams([N] * n, [R] * n, seeds)
    before = [wn.wn_get_state(h, i) for i in range(n)]
    qt, th = wn.wn_autotune(h, count)
    assert wn.wn_get_config(h) == (qt, th) and qt * th >= N // 4
    assert [wn.wn_get_state(h, i) for i in range(n)] == before  # state restored
    got = _gen(wn, torch, h, count).cpu().numpy().reshape(n, count)
    for i in (0, n - 1):
        ref = oracle.Stream(N, R, seeds[i]).generate(count)
        assert_fp32_close(got[i], ref, passes_fresh(count, N, R), f"autotuned stream {i}")
