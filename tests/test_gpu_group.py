"""Group-mode kernel (WN_CFG_GROUP) against the FP64 oracle.

Every compiled group shape must return each stream's next values within the
FP32 error model, continue the sequence across calls (whole blocks, partial
blocks, requests shorter than the rest of a block), leave the integer state
(generator words, block counts, positions) exactly as the oracle's, and mix
freely with the ordinary kernel on the same handle.  16-bit outputs are the
round-to-nearest conversions of the same FP32 values.
"""
import numpy as np
import pytest

import oracle
from _parity import assert_fp32_close, passes_fresh

pytestmark = pytest.mark.gpu

# (pool N, quadruples per lane, threads) of the compiled group shapes
SHAPES = [(1024, 8, 32), (1024, 2, 128), (2048, 16, 32), (4096, 32, 32), (4096, 16, 64), (4096, 8, 128),
          (4096, 4, 256), (8192, 32, 64), (16384, 32, 128), (16384, 16, 256)]


def _handle(wn, N, R, seeds, shape):
    h = wn.wn_create_streams([N] * len(seeds), [R] * len(seeds), seeds)
    wn.wn_set_config_ex(h, shape[1], shape[2], wn.WN_CFG_GROUP)
    assert wn.wn_get_config_ex(h) == (shape[1], shape[2], wn.WN_CFG_IN_PLACE | wn.WN_CFG_GROUP)
    return h


def _gen(wn, h, count, dtype=0):
    import torch
    tdt = {0: torch.float32, 1: torch.bfloat16, 2: torch.float16}[dtype]
    out = torch.empty(count * h.n, dtype=tdt, device="cuda")
    wn.wn_generate_ex(out, count, h, dtype)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("shape", SHAPES, ids=[f"N{s[0]}_q{s[1]}_t{s[2]}" for s in SHAPES])
def test_group_shapes_match_oracle_across_calls(wn, shape):
    N = shape[0]
    R = 2 if N < 16384 else 3
    seeds = [70 + i for i in range(5)]
    h = _handle(wn, N, R, seeds, shape)
    # a count that is not a multiple of 4 (every stream starts at another
    # alignment), then a call inside one block, then several whole blocks
    counts = [2 * (N - 1) + 7, 5, 3 * (N - 1) + 2]
    refs = [oracle.Stream(N, R, s) for s in seeds]
    done = 0
    for c in counts:
        got = _gen(wn, h, c).cpu().numpy().reshape(len(seeds), c)
        fb = done // (N - 1)
        for i, s in enumerate(refs):
            ref = s.generate(c)
            assert_fp32_close(got[i], ref, passes_fresh(c, N, R, first_block=fb) + R, f"N={N} call {c} stream {i}")
        done += c
    for i, s in enumerate(refs):
        st = wn.wn_get_state(h, i)
        assert (st["x"], st["w"]) == s.gen_state
        assert st["k"] == s.k and st["blocks"] == s.blocks


def test_group_and_ordinary_kernels_interleave(wn):
    # group -> ordinary -> group on one handle: each call continues where the
    # other left the state (pool, reserved value, scale, sum of squares)
    N, R, seeds = 4096, 2, [5, 6, 7]
    h = _handle(wn, N, R, seeds, (4096, 32, 32))
    refs = [oracle.Stream(N, R, s) for s in seeds]
    done = 0
    for c, group in ((9000, True), (7000, False), (12001, True)):
        if group:
            wn.wn_set_config_ex(h, 32, 32, wn.WN_CFG_GROUP)
        else:
            wn.wn_set_config(h, 8, 128)
        got = _gen(wn, h, c).cpu().numpy().reshape(len(seeds), c)
        for i, s in enumerate(refs):
            assert_fp32_close(got[i], s.generate(c), passes_fresh(c, N, R, first_block=done // (N - 1)) + R,
                              f"call of {c} ({'group' if group else 'ordinary'}) stream {i}")
        done += c


def test_group_many_streams_against_ordinary_kernel(wn):
    # 600 streams (several waves at any occupancy): every value within the
    # FP32 tolerance of the ordinary kernel's, and identical integer state
    import torch
    from _parity import C_MAX, U
    N, R, n, count = 4096, 2, 600, 5 * 4095 + 3
    seeds = list(range(1000, 1000 + n))
    hg = _handle(wn, N, R, seeds, (4096, 32, 32))
    ho = wn.wn_create_streams([N] * n, [R] * n, seeds)
    a = _gen(wn, hg, count).double()
    b = _gen(wn, ho, count).double()
    P = torch.from_numpy(passes_fresh(count, N, R).astype(np.float64)).cuda()
    tol = 2 * C_MAX * U * torch.sqrt(P) * (1 + b.view(n, count).abs())
    assert bool(((a - b).view(n, count).abs() <= tol).all())
    for i in range(0, n, 61):
        sg, so = wn.wn_get_state(hg, i), wn.wn_get_state(ho, i)
        assert (sg["x"], sg["w"], sg["k"], sg["blocks"]) == (so["x"], so["w"], so["k"], so["blocks"])
    ref = oracle.Stream(N, R, seeds[-1]).generate(count)
    assert_fp32_close(a.view(n, count)[-1].cpu().numpy(), ref, passes_fresh(count, N, R), "last stream")


@pytest.mark.parametrize("dtype", [1, 2])
def test_group_16bit_outputs_round_fp32_values(wn, dtype):
    N, R, seeds, count = 16384, 3, [3, 4], 2 * 16383 + 9
    f32 = _gen(wn, _handle(wn, N, R, seeds, (16384, 32, 128)), count)
    low = _gen(wn, _handle(wn, N, R, seeds, (16384, 32, 128)), count, dtype)
    assert bool((low == f32.to(low.dtype)).all())


def test_group_rejects_other_shapes_and_variants(wn):
    h = wn.wn_create_streams([4096] * 2, [2] * 2, [1, 2])
    with pytest.raises(wn.WnError):
        wn.wn_set_config_ex(h, 16, 32, wn.WN_CFG_GROUP)   # covers 2048, not 4096
    with pytest.raises(wn.WnError):
        wn.wn_set_config_ex(h, 8, 96, wn.WN_CFG_GROUP)    # three warps: no such compiled shape
    hv = wn.wn_create_ex([4096] * 2, [2] * 2, [1, 2], chi2="a")
    with pytest.raises(wn.WnError):
        wn.wn_set_config_ex(hv, 32, 32, wn.WN_CFG_GROUP)  # variants keep the general kernels
    hm = wn.wn_create_streams([4096, 1024], [2, 2], [1, 2])
    with pytest.raises(wn.WnError):
        wn.wn_set_config_ex(hm, 32, 32, wn.WN_CFG_GROUP)  # mixed pool sizes
