"""The allocation-free batch entry point, wn_generate_batch_noalloc.

Some callers must not allocate device memory (their device memory belongs to
another allocator, or their serving loop cannot afford cudaMalloc's blocking).
wn_generate_batch_noalloc does the work of wn_generate_batch with its scratch
in a fixed device array compiled into the library.  Here it is called through
the C ABI twice in a row and compared, call by call, with wn_generate_batch on
an identical handle, within the FP32 tolerance the other tests use; the
device's free memory does not move across the calls.  This file is named so
that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from _parity import C_MAX, U, assert_fp32_close, passes_fresh
from paper_1005_2314_gb300.workloads import packed_offsets

pytestmark = pytest.mark.gpu


def _requests():
    rng = np.random.default_rng(2024)
    n = 48
    N = rng.choice(np.array([4, 256, 1024, 4096, 16384], dtype=np.uint32), size=n)
    R = rng.choice(np.array([1, 2, 3], dtype=np.uint32), size=n)
    counts = rng.integers(0, 30000, size=n).astype(np.uint64)
    counts[:4] = [0, 1, 1023, 4095]
    return N, R, counts, np.arange(900, 900 + n)


def test_noalloc_matches_batch_entry_point_twice(wn):
    import torch
    N, R, counts, seeds = _requests()
    offsets = packed_offsets(counts) + 1  # odd start: every output alignment occurs
    total = int(counts.sum()) + 8
    ha = wn.wn_create_streams(N, R, seeds)
    hb = wn.wn_create_streams(N, R, seeds)
    ref = torch.zeros(total, dtype=torch.float32, device="cuda")
    got = torch.zeros(total, dtype=torch.float32, device="cuda")
    # blocks completed before each call bound the values' passes (error model)
    P = np.zeros(total)
    for call in range(2):
        for i in range(len(N)):
            b_end = 8 + (call + 1) * (int(counts[i]) // (int(N[i]) - 1) + 2)
            P[int(offsets[i]): int(offsets[i]) + int(counts[i])] = int(R[i]) * b_end
        wn.wn_generate_batch(ref, counts, offsets, ha)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        wn.wn_generate_batch_noalloc(got, counts, offsets, hb)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before
        r = ref.double().cpu().numpy()
        g = got.double().cpu().numpy()
        tol = C_MAX * U * np.sqrt(np.maximum(P, 1.0)) * (1.0 + np.abs(r))
        assert np.all(np.abs(g - r) <= tol), f"call {call}: {int(np.argmax(np.abs(g - r) - tol))}"
        for i in range(len(N)):
            assert wn.wn_get_state(ha, i)["k"] == wn.wn_get_state(hb, i)["k"]


def test_noalloc_rejects_more_streams_than_its_scratch_holds(wn):
    import torch
    n = wn.WN_NOALLOC_MAX_STREAMS + 1
    h = wn.wn_create_streams([4] * n, [1] * n, np.arange(1, n + 1), warmup_blocks=0)
    out = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(wn.WnError, match="exceed"):
        wn.wn_generate_batch_noalloc(out, np.ones(n, dtype=np.uint64), np.arange(n, dtype=np.uint64), h)


def test_noalloc_matches_the_oracle_directly(wn):
    # the same requests checked against the FP64 oracle itself, not only
    # against the other batch entry point, for streams of every pool size
    import torch
    N, R, counts, seeds = _requests()
    offsets = packed_offsets(counts) + 1
    h = wn.wn_create_streams(N, R, seeds)
    out = torch.zeros(int(counts.sum()) + 8, dtype=torch.float32, device="cuda")
    wn.wn_generate_batch_noalloc(out, counts, offsets, h)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    pick = [int(np.flatnonzero((N == n) & (counts > 0))[0]) for n in np.unique(N)]
    for i in pick + [1, 2]:
        c = int(counts[i])
        ref = oracle.Stream(int(N[i]), int(R[i]), int(seeds[i])).generate(c)
        assert_fp32_close(got[int(offsets[i]): int(offsets[i]) + c], ref, passes_fresh(c, int(N[i]), int(R[i])),
                          f"stream {i} N={N[i]} R={R[i]}")


def test_noalloc_refuses_stream_capture(wn):
    # the call reads host arrays and advances host positions when it is made,
    # so recording it into a CUDA graph is refused (nothing is enqueued)
    import torch
    h = wn.wn_create_streams([64, 64], [1, 1], [1, 2])
    out = torch.zeros(256, dtype=torch.float32, device="cuda")
    x = torch.zeros(4, device="cuda")
    before = [wn.wn_get_state(h, i) for i in range(2)]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=torch.cuda.Stream()):
        x.add_(1.0)
        with pytest.raises(wn.WnError, match="captured"):
            wn.wn_generate_batch_noalloc(out, [10, 10], [0, 128], h)
    torch.cuda.synchronize()
    assert [wn.wn_get_state(h, i) for i in range(2)] == before
