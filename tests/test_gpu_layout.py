"""The in-place pool layout (WN_CFG_IN_PLACE) against the two-buffer layout
and against the FP64 oracle.

In place, a pass gathers all of a CTA's quadruples into registers before
any result overwrites the pool, so with the same shape the arithmetic, and
hence every output bit, equals the two-buffer layout's.  The reserved value
reaches the next block's scale through its own copy, not the pool, so the
cases cover one pass per block (the first pass is also the final one), the
variants that read the pool in the final pass (fastnorm's reserved value),
rotations, decimation, partial blocks across calls and pools of different
sizes in one launch.
"""
import numpy as np
import pytest

import oracle
from _parity import assert_fp32_close, passes_fresh

pytestmark = pytest.mark.gpu


def _pair(wn, N, R, seeds, threads, **ex):
    """Two handles on the same streams: two buffers and in place."""
    hs = []
    for ip in (0, wn.WN_CFG_IN_PLACE):
        h = wn.wn_create_ex([N] * len(seeds), [R] * len(seeds), list(seeds), **ex) if ex else \
            wn.wn_create_streams([N] * len(seeds), [R] * len(seeds), list(seeds))
        wn.wn_set_config_ex(h, 16, threads, ip)
        assert wn.wn_get_config_ex(h) == (16, threads, ip)
        hs.append(h)
    return hs


def _run_both(wn, hs, counts, dtype=0):
    import torch
    tdt = {0: torch.float32, 1: torch.bfloat16, 2: torch.float16}[dtype]
    outs = [[], []]
    for c in counts:
        for i, h in enumerate(hs):
            o = torch.empty(c * h.n, dtype=tdt, device="cuda")
            wn.wn_generate_ex(o, c, h, dtype)
            outs[i].append(o)
    torch.cuda.synchronize()
    return outs


@pytest.mark.parametrize("N,R,threads", [(4096, 1, 64), (4096, 2, 64), (8192, 3, 128), (16384, 1, 256),
                                         (16384, 3, 256)])
def test_in_place_is_bit_identical(wn, N, R, threads):
    import torch
    seeds = list(range(11, 11 + 80))  # more streams than half the SMs: the ordinary kernel
    hs = _pair(wn, N, R, seeds, threads)
    counts = [3 * (N - 1) + 5, N - 7, 1, 2 * (N - 1)]  # partial blocks carried across calls
    a, b = _run_both(wn, hs, counts)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    for i in (0, 17):
        assert wn.wn_get_state(hs[0], i) == wn.wn_get_state(hs[1], i)


@pytest.mark.parametrize("ex", [dict(reserve="current"), dict(chi2="b"), dict(decimate=3), dict(update="rotation"),
                                dict(reserve="current", update="rotation")])
@pytest.mark.parametrize("R", [1, 3])
def test_in_place_variants_bit_identical(wn, ex, R):
    import torch
    N = 8192
    hs = _pair(wn, N, R, list(range(1, 81)), 128, **ex)
    a, b = _run_both(wn, hs, [2 * (N - 1) + 3, N + 1])
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("dtype", [1, 2])
def test_in_place_16bit_outputs(wn, dtype):
    import torch
    hs = _pair(wn, 16384, 3, list(range(1, 97)), 256)
    a, b = _run_both(wn, hs, [5 * 16383 + 9, 16383], dtype)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_in_place_matches_oracle(wn):
    # pool 16384, R = 3 (the 16-bit precision workload's pools) through the
    # in-place layout, FP32 out, against the FP64 oracle
    import torch
    N, R, seeds = 16384, 3, [1, 2, 3]
    h = wn.wn_create_streams([N] * 3, [R] * 3, seeds)
    wn.wn_set_config_ex(h, 16, 256, wn.WN_CFG_IN_PLACE)
    count = 2 * (N - 1) + 100
    out = torch.empty(3 * count, device="cuda")
    wn.wn_generate(out, count, h)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(3, count)
    for i, s in enumerate(seeds):
        ref = oracle.Stream(N, R, s).generate(count)
        assert_fp32_close(got[i], ref, passes_fresh(count, N, R), f"seed {s}")


def test_in_place_mixed_pools(wn):
    # pools of different sizes in one launch (no FULL fast path): every
    # stream's CTA covers the largest pool's quadruples, smaller pools leave
    # compute threads idle
    import torch
    N = np.array([16384, 4096, 8192, 16384, 1024] * 8, dtype=np.uint32)
    R = np.array([3, 2, 1, 2, 3] * 8, dtype=np.uint32)
    seeds = list(range(500, 500 + len(N)))
    count = 9000
    outs = []
    for ip in (0, wn.WN_CFG_IN_PLACE):
        h = wn.wn_create_streams(N, R, seeds)
        wn.wn_set_config_ex(h, 16, 256, ip)
        o = torch.empty(len(N) * count, device="cuda")
        wn.wn_generate(o, count, h)
        outs.append(o)
    torch.cuda.synchronize()
    assert torch.equal(outs[0], outs[1])
    got = outs[1].cpu().numpy().reshape(len(N), count)
    for i in (0, 1, 2, 4):
        ref = oracle.Stream(int(N[i]), int(R[i]), seeds[i]).generate(count)
        assert_fp32_close(got[i], ref, passes_fresh(count, int(N[i]), int(R[i])), f"stream {i}")


def test_in_place_rejected_where_not_compiled(wn):
    h = wn.wn_create_streams([4096] * 2, [2] * 2, [1, 2])
    with pytest.raises(wn.WnError):
        wn.wn_set_config_ex(h, 8, 128, wn.WN_CFG_IN_PLACE)  # no in-place kernel with 8 quadruples per thread
    with pytest.raises(wn.WnError):
        wn.wn_set_config_ex(h, 16, 64, 8)  # unknown flag


def test_default_shapes(wn):
    # many streams of one pool size from 1024 up run the group mode by
    # default (one warp per stream up to 4096, two at 8192, four at 16384);
    # variants and smaller pools keep the ordinary kernel's shapes
    GI = wn.WN_CFG_IN_PLACE | wn.WN_CFG_GROUP
    for N, shape in ((1024, (8, 32, GI)), (4096, (32, 32, GI)), (8192, (32, 64, GI)), (16384, (32, 128, GI))):
        h = wn.wn_create_streams([N] * 100, [2] * 100, list(range(1, 101)), warmup_blocks=0)
        assert wn.wn_get_config_ex(h) == shape, N
    hv = wn.wn_create_ex([16384] * 100, [3] * 100, list(range(1, 101)), warmup_blocks=0, chi2="b")
    assert wn.wn_get_config_ex(hv) == (16, 256, wn.WN_CFG_IN_PLACE)
    h2 = wn.wn_create_ex([4096] * 100, [2] * 100, list(range(1, 101)), warmup_blocks=0, chi2="b")
    assert wn.wn_get_config_ex(h2) == (8, 128, 0)
    h3 = wn.wn_create_streams([256] * 100, [2] * 100, list(range(1, 101)), warmup_blocks=0)
    assert wn.wn_get_config_ex(h3)[2] == 0
