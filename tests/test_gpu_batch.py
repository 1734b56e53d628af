"""Batched uneven requests: persistent kernels per pool size, CUDA graph.

Every stream's slice of the batch output must be the oracle's next values of
that stream (FP32 within the error model), whatever the mix of pool sizes,
passes and lengths, including empty requests and partial blocks, and with
slices packed contiguously so that every alignment occurs.
"""
import numpy as np
import pytest

import oracle
from _parity import assert_fp32_close, passes_fresh
from paper_1005_2314_gb300.workloads import packed_offsets, uneven_batch

pytestmark = pytest.mark.gpu


def _mix(n=36, seed=5):
    rng = np.random.default_rng(seed)
    N = rng.choice(np.array([4, 64, 1024, 4096, 16384], dtype=np.uint32), size=n)
    R = rng.choice(np.array([1, 2, 3, 4], dtype=np.uint32), size=n)
    counts = rng.integers(0, 40000, size=n).astype(np.uint64)
    counts[:6] = [0, 1, 3, 1022, 4095, 16383]
    return N, R, counts


def _check(got_flat, N, R, seeds, counts, offsets, first_blocks=None, prefix=None):
    for i in range(len(N)):
        c = int(counts[i])
        if c == 0:
            continue
        s = oracle.Stream(int(N[i]), int(R[i]), int(seeds[i]))
        fb = 0
        if prefix is not None:
            s.skip(int(prefix[i]))
            fb = int(prefix[i]) // (int(N[i]) - 1)
        ref = s.generate(c)
        got = got_flat[int(offsets[i]): int(offsets[i]) + c]
        # values of a block begun before this call were formed in earlier blocks
        assert_fp32_close(got, ref, passes_fresh(c, int(N[i]), int(R[i]), first_block=fb) + int(R[i]),
                          f"stream {i} N={N[i]} R={R[i]}")


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_oracle_and_continues(wn, use_graph):
    import torch
    N, R, counts = _mix()
    seeds = np.arange(100, 100 + len(N))
    offsets = packed_offsets(counts)
    total = int(counts.sum())
    h = wn.wn_create_streams(N, R, seeds)
    out = torch.zeros(total + 8, dtype=torch.float32, device="cuda")
    wn.wn_generate_batch(out, counts, offsets, h, use_graph=use_graph)
    torch.cuda.synchronize()
    _check(out.cpu().numpy(), N, R, seeds, counts, offsets)
    # a second call (a graph replay when use_graph) continues every stream
    wn.wn_generate_batch(out, counts, offsets, h, use_graph=use_graph)
    torch.cuda.synchronize()
    _check(out.cpu().numpy(), N, R, seeds, counts, offsets, prefix=counts)


def test_graph_recaptures_on_new_arguments(wn):
    import torch
    N, R, counts = _mix(12, seed=9)
    seeds = np.arange(7, 7 + len(N))
    h = wn.wn_create_streams(N, R, seeds)
    off1 = packed_offsets(counts)
    out = torch.zeros(int(counts.sum()) * 2 + 8, dtype=torch.float32, device="cuda")
    wn.wn_generate_batch(out, counts, off1, h, use_graph=True)
    counts2 = counts[::-1].copy()
    off2 = packed_offsets(counts2) + 3  # other lengths, shifted alignment
    wn.wn_generate_batch(out, counts2, off2, h, use_graph=True)
    torch.cuda.synchronize()
    _check(out.cpu().numpy(), N, R, seeds, counts2, off2, prefix=counts)


def test_graph_replay_after_an_eager_call_with_other_arguments(wn):
    # graph(A) -> eager(B) -> graph(A) on one handle: the eager call uploads
    # other descriptors, and the cached graph must still serve A (it reads a
    # copy of its own).  Every range of B lies inside the buffer A uses, so a
    # graph that replayed B's descriptors would give wrong values, not write
    # out of bounds.
    import torch
    N, R, countsA = _mix(14, seed=17)
    seeds = np.arange(300, 300 + len(N))
    offA = packed_offsets(countsA) + 1
    countsB = countsA[::-1].copy()
    offB = packed_offsets(countsB) + 3
    size = int(max(offA[-1] + countsA[-1], offB[-1] + countsB[-1])) + 8
    h = wn.wn_create_streams(N, R, seeds)
    out = torch.zeros(size, dtype=torch.float32, device="cuda")
    wn.wn_generate_batch(out, countsA, offA, h, use_graph=True)
    torch.cuda.synchronize()
    _check(out.cpu().numpy(), N, R, seeds, countsA, offA)
    wn.wn_generate_batch(out, countsB, offB, h, use_graph=False)
    torch.cuda.synchronize()
    _check(out.cpu().numpy(), N, R, seeds, countsB, offB, prefix=countsA)
    out.zero_()
    wn.wn_generate_batch(out, countsA, offA, h, use_graph=True)  # a replay of the first graph
    torch.cuda.synchronize()
    _check(out.cpu().numpy(), N, R, seeds, countsA, offA, prefix=countsA + countsB)
    for i in range(len(N)):
        ref = oracle.Stream(int(N[i]), int(R[i]), int(seeds[i]))
        ref.skip(int(2 * countsA[i] + countsB[i]))
        st = wn.wn_get_state(h, i)
        assert (st["k"], st["blocks"]) == (ref.k, ref.blocks)


def test_batch_arguments_may_be_reused_at_once(wn):
    # counts and offsets are copied before the call returns: overwriting the
    # caller's (page-locked) arrays right after the call changes nothing
    import torch
    N, R, counts = _mix(10, seed=23)
    seeds = np.arange(40, 40 + len(N))
    offsets = packed_offsets(counts)
    tc = torch.from_numpy(counts.astype(np.int64)).pin_memory()
    to = torch.from_numpy(offsets.astype(np.int64)).pin_memory()
    h = wn.wn_create_streams(N, R, seeds)
    out = torch.zeros(int(counts.sum()) + 8, dtype=torch.float32, device="cuda")
    wn._L().wn_generate_batch(out.data_ptr(), tc.data_ptr(), to.data_ptr(), h.ptr, wn.WN_F32, 0,
                              torch.cuda.current_stream().cuda_stream)
    tc.fill_(0)
    to.fill_(0)
    torch.cuda.synchronize()
    _check(out.cpu().numpy(), N, R, seeds, counts, offsets)


def test_autotune_batch_keeps_state(wn):
    import torch
    N, R, counts = _mix(20, seed=11)
    seeds = np.arange(50, 50 + len(N))
    h = wn.wn_create_streams(N, R, seeds)
    offsets = packed_offsets(counts)
    out = torch.zeros(int(counts.sum()) + 8, dtype=torch.float32, device="cuda")
    before = [wn.wn_get_state(h, i) for i in range(len(N))]
    wn.wn_autotune_batch(out, counts, offsets, h)
    assert [wn.wn_get_state(h, i) for i in range(len(N))] == before
    wn.wn_generate_batch(out, counts, offsets, h, use_graph=True)
    torch.cuda.synchronize()
    _check(out.cpu().numpy(), N, R, seeds, counts, offsets)


def test_uneven_recipe_scaled_down(wn):
    # the batched-request recipe (pool from {1024, 4096, 16384}, R from
    # {1, 2, 4}, log-uniform lengths) at 300 streams and lengths 2^10..2^16
    import torch
    N, R, counts = uneven_batch(300, seed=12345, log2_max=16.0)
    seeds = np.arange(1, 301)
    offsets = packed_offsets(counts)
    h = wn.wn_create_streams(N, R, seeds)
    out = torch.zeros(int(counts.sum()) + 8, dtype=torch.float32, device="cuda")
    wn.wn_generate_batch(out, counts, offsets, h, use_graph=True)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    pick = np.arange(0, 300, 37)
    _check(got, N[pick], R[pick], seeds[pick], counts[pick], offsets[pick])


@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_latency_mode_agrees_with_the_ordinary_kernel(wn, R):
    # Few streams run in the latency mode (a table warp, an emitter warp that
    # writes each block while the compute warps run the next, mbarrier
    # hand-offs); many streams run the ordinary kernel.  The passes are the
    # same arithmetic; the sums of squares are added in another order (per
    # emitter lane), so values agree within the FP32 tolerance and the integer
    # state exactly, over calls that stop mid-block.
    import torch
    from _parity import C_MAX, U
    N, shape = 1024, (2, 128)
    n_many = 200  # more than half the SMs: the ordinary kernel
    many = wn.wn_create_streams([N] * n_many, [R] * n_many, list(range(1, n_many + 1)))
    wn.wn_set_config(many, *shape)
    few = wn.wn_create_streams([N] * 3, [R] * 3, [1, 2, 3])
    wn.wn_set_config(few, *shape)
    count = 5 * (N - 1) + 11
    a = torch.empty(n_many * count, device="cuda")
    b = torch.empty(3 * count, device="cuda")
    for call in range(2):  # the second call continues mid-block
        wn.wn_generate(a, count, many)
        wn.wn_generate(b, count, few)
        torch.cuda.synchronize()
        x, y = a.view(n_many, count)[:3].double(), b.view(3, count).double()
        P = torch.from_numpy(passes_fresh(count, N, R, first_block=call * count // (N - 1)) + R).double().cuda()
        assert bool(((x - y).abs() <= 2 * C_MAX * U * P.sqrt() * (1 + x.abs())).all())
        for i in range(3):
            sm, sf = wn.wn_get_state(many, i), wn.wn_get_state(few, i)
            assert (sm["x"], sm["w"], sm["k"], sm["blocks"]) == (sf["x"], sf["w"], sf["k"], sf["blocks"])
        ref = oracle.Stream(N, R, 1)
        ref.skip(call * count)
        assert_fp32_close(y[0].cpu().numpy(), ref.generate(count),
                          passes_fresh(count, N, R, first_block=call * count // (N - 1)) + R, "latency stream 0")


def test_full_batch_recipe_sampled(wn):
    # the batched-request workload at full size (10,000 streams, ~1.76e10 FP32
    # values) in the launch configuration the benchmark times: wn_autotune_batch,
    # then a captured graph, replayed once more (each stream continues); checked
    # on sampled streams -- the longest request of each pool size, a few short
    # and a few random ones -- against the oracle over both calls
    import torch
    N, R, counts = uneven_batch(10000, seed=12345)
    seeds = np.arange(1, 10001)
    offsets = packed_offsets(counts)
    total = int(counts.sum())
    h = wn.wn_create_streams(N, R, seeds)
    out = torch.empty(total, dtype=torch.float32, device="cuda")
    wn.wn_autotune_batch(out, counts, offsets, h)
    rng = np.random.default_rng(3)
    pick = set(rng.choice(10000, size=6, replace=False).tolist())
    for n in (1024, 4096, 16384):
        idx = np.flatnonzero(N == n)
        pick.add(int(idx[np.argmax(counts[idx])]))
        pick.add(int(idx[np.argmin(counts[idx])]))
    pick = sorted(pick)
    for call in range(2):
        wn.wn_generate_batch(out, counts, offsets, h, use_graph=True)
        torch.cuda.synchronize()
        got = {i: out[int(offsets[i]): int(offsets[i] + counts[i])].cpu().numpy() for i in pick}
        for i in pick:
            s = oracle.Stream(int(N[i]), int(R[i]), int(seeds[i]))
            c = int(counts[i])
            fb = 0
            if call:
                s.skip(c)
                fb = c // (int(N[i]) - 1)
            ref = s.generate(c)
            assert_fp32_close(got[i], ref, passes_fresh(c, int(N[i]), int(R[i]), first_block=fb) + int(R[i]),
                              f"call {call} stream {i} N={N[i]} R={R[i]} count={c}")
    del out
    torch.cuda.empty_cache()


def test_batch_plans_change_placement_not_values(wn):
    # chain groups (the longest requests in the latency mode, launched first)
    # at one or two CTAs per SM, or none: the values are the oracle's either way
    import torch
    rng = np.random.default_rng(31)
    n = 40
    N = rng.choice(np.array([1024, 4096], dtype=np.uint32), size=n)
    R = rng.choice(np.array([1, 2, 4], dtype=np.uint32), size=n)
    counts = rng.integers(0, 30000, size=n).astype(np.uint64)
    counts[:4] = [200000, 150000, 120000, 3]  # a few long chains
    R[:3] = 4
    seeds = np.arange(600, 600 + n)
    offsets = packed_offsets(counts) + 2
    out = torch.zeros(int(counts.sum()) + 8, dtype=torch.float32, device="cuda")
    for chains, density in ((0, 1), (3, 1), (5, 2), (-1, 1)):
        h = wn.wn_create_streams(N, R, seeds)
        wn.wn_set_batch_plan(h, chains, density)
        assert wn.wn_get_batch_plan(h) == (chains, density)
        out.zero_()
        wn.wn_generate_batch(out, counts, offsets, h, use_graph=bool(chains % 2))
        torch.cuda.synchronize()
        _check(out.cpu().numpy(), N, R, seeds, counts, offsets)
    with pytest.raises(wn.WnError):
        wn.wn_set_batch_plan(h, -2, 1)
    with pytest.raises(wn.WnError):
        wn.wn_set_batch_plan(h, 4, 0)
