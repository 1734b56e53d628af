"""Checkpoint and resume (wn_save / wn_load) on the GPU.

A loaded handle must continue every stream bit for bit as the saved handle
would have (integers and FP32 values identical, not just within tolerance),
from any position in a block, for mixed pool sizes and pass counts; the
saved bytes round-trip; and the continuation still matches the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from _parity import assert_fp32_close, passes_fresh

pytestmark = pytest.mark.gpu

NS = [1024, 4096, 64, 16384]
RS = [2, 2, 3, 1]
SEEDS = [11, 12, 13, 14]


def _gen(wn, h, count):
    import torch
    out = torch.empty(count * h.n, dtype=torch.float32, device="cuda")
    wn.wn_generate(out, count, h)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(h.n, count)


@pytest.mark.parametrize("first", [0, 1, 4095, 40_000])
def test_resume_is_bit_exact(wn, first):
    h = wn.wn_create_streams(NS, RS, SEEDS)
    if first:
        _gen(wn, h, first)  # leaves some streams mid-block
    buf = wn.wn_save(h)
    more = 3 * 16383 + 17
    a = _gen(wn, h, more)
    h2 = wn.wn_load(buf)
    assert h2.n == len(NS)
    b = _gen(wn, h2, more)
    assert np.array_equal(a, b)
    for i in range(len(NS)):
        assert wn.wn_get_state(h, i) == wn.wn_get_state(h2, i)
        assert np.array_equal(wn.wn_get_pool(h, i, NS[i]), wn.wn_get_pool(h2, i, NS[i]))


def test_saved_bytes_round_trip_and_two_resumes_agree(wn):
    h = wn.wn_create_streams(NS, RS, SEEDS)
    _gen(wn, h, 777)
    buf = wn.wn_save(h)
    h2, h3 = wn.wn_load(buf), wn.wn_load(buf.tobytes())
    assert np.array_equal(wn.wn_save(h2), buf)
    assert np.array_equal(_gen(wn, h2, 5000), _gen(wn, h3, 5000))


def test_save_includes_enqueued_work_and_matches_oracle(wn):
    import torch
    h = wn.wn_create_streams(NS[:2], RS[:2], SEEDS[:2])
    out = torch.empty(2 * 3000, device="cuda")
    wn.wn_generate(out, 3000, h)  # not synchronised: wn_save must wait for it
    buf = wn.wn_save(h)
    got = _gen(wn, wn.wn_load(buf), 2 * 4095 + 3)
    for i in range(2):
        ref = oracle.Stream(NS[i], RS[i], SEEDS[i])
        ref.skip(3000)
        fb = 3000 // (NS[i] - 1)
        assert_fp32_close(got[i], ref.generate(2 * 4095 + 3), passes_fresh(2 * 4095 + 3, NS[i], RS[i], first_block=fb))


def test_save_waits_for_work_on_another_cuda_stream(wn):
    # a call enqueued on a non-blocking stream other than the handle's: the
    # checkpoint must still include it (one lone stream of 2^24 values takes
    # milliseconds, so a save that did not wait would copy the old state)
    import torch
    h = wn.wn_create(1024, 2, 7)
    side = torch.cuda.Stream()
    n = 1 << 24
    out = torch.empty(n, device="cuda")
    with torch.cuda.stream(side):
        wn.wn_generate_ex(out, n, h, wn.WN_F32, side)
    buf = wn.wn_save(h)  # no synchronisation before it
    ref = oracle.Stream(1024, 2, 7)
    ref.skip(n)
    h2 = wn.wn_load(buf)
    st = wn.wn_get_state(h2, 0)
    assert (st["k"], st["blocks"]) == (ref.k, ref.blocks)
    assert (st["x"], st["w"]) == ref.gen_state
    torch.cuda.synchronize()
    assert wn.wn_get_state(h, 0) == st


def test_buffer_too_small_is_rejected(wn):
    import ctypes
    h = wn.wn_create_streams([64], [2], [1])
    need = ctypes.c_uint64(0)
    assert wn._L().wn_save(h.ptr, None, 0, ctypes.byref(need)) == 0
    small = np.empty(need.value - 1, np.uint8)
    assert wn._L().wn_save(h.ptr, small.ctypes.data, small.size, None) == wn.WN_EINVAL
