"""Chain-mode kernel (WN_CFG_CHAIN) against the FP64 oracle.

The chain mode runs a stream's passes on compute warps alone, while a draw
warp writes the passes' permutation and sign words blocks ahead, a scale warp
forms each block's scale from the block's sums of squares a block late, and
store warps stage each block's values in the output's 16-byte layout and write
them with bulk copies (pools above 8192: the compute warps store them).  Every compiled shape must return each stream's next values within the
FP32 error model, continue the sequence across calls (whole blocks, partial
blocks, requests shorter than the rest of a block), leave the integer state
exactly as the oracle's, and mix with the other kernels on one handle.  Lone
streams take it without being asked; batches run their longest requests in it
when wn_set_batch_chain_kernel asks for it.
"""
import numpy as np
import pytest

import oracle
from _parity import assert_fp32_close, passes_fresh
from paper_1005_2314_gb300.workloads import packed_offsets

pytestmark = pytest.mark.gpu

# (pool N, quadruples per lane, compute threads) of the compiled chain shapes
SHAPES = [(1024, 2, 128), (1024, 1, 256), (2048, 2, 256), (4096, 4, 256), (8192, 8, 256), (16384, 16, 256)]


def _handle(wn, N, R, seeds, shape):
    h = wn.wn_create_streams([N] * len(seeds), [R] * len(seeds), seeds)
    wn.wn_set_config_ex(h, shape[1], shape[2], wn.WN_CFG_CHAIN)
    assert wn.wn_get_config_ex(h) == (shape[1], shape[2], wn.WN_CFG_CHAIN)
    return h


def _gen(wn, h, count, dtype=0):
    import torch
    tdt = {0: torch.float32, 1: torch.bfloat16, 2: torch.float16}[dtype]
    out = torch.empty(count * h.n, dtype=tdt, device="cuda")
    wn.wn_generate_ex(out, count, h, dtype)
    torch.cuda.synchronize()
    return out


def _run_calls(wn, h, N, R, seeds, counts):
    refs = [oracle.Stream(N, R, s) for s in seeds]
    done = 0
    for c in counts:
        got = _gen(wn, h, c).cpu().numpy().reshape(len(seeds), c)
        fb = done // (N - 1)
        for i, s in enumerate(refs):
            assert_fp32_close(got[i], s.generate(c), passes_fresh(c, N, R, first_block=fb) + R,
                              f"N={N} R={R} call {c} stream {i}")
        done += c
    for i, s in enumerate(refs):
        st = wn.wn_get_state(h, i)
        assert (st["x"], st["w"]) == s.gen_state
        assert st["k"] == s.k and st["blocks"] == s.blocks


@pytest.mark.parametrize("shape", SHAPES, ids=[f"N{s[0]}_q{s[1]}_t{s[2]}" for s in SHAPES])
def test_chain_shapes_match_oracle_across_calls(wn, shape):
    N = shape[0]
    R = 2 if N < 16384 else 3
    seeds = [90 + i for i in range(3)]
    # a count that is not a multiple of 4 (the streams start at other
    # alignments), a call inside one block, one of exactly one block, then
    # several blocks ending in a partial one
    _run_calls(wn, _handle(wn, N, R, seeds, shape), N, R, seeds, [2 * (N - 1) + 7, 5, N - 1, 3 * (N - 1) + 2])


@pytest.mark.parametrize("R", [1, 2, 3, 4, 7])
def test_chain_passes_per_block(wn, R):
    # the barrier pattern depends on R: with one pass the scale hand-over and
    # the block's end share a pass; odd R end blocks in the other buffer
    N, seeds = 1024, [11, 12]
    _run_calls(wn, _handle(wn, N, R, seeds, (1024, 2, 128)), N, R, seeds, [9 * (N - 1) + 3, 1, 4 * (N - 1)])


def test_lone_streams_take_the_chain_mode(wn):
    h = wn.wn_create(1024, 2, 1)
    assert wn.wn_get_config_ex(h)[2] == wn.WN_CFG_CHAIN
    many = wn.wn_create_streams([1024] * 400, [2] * 400, list(range(400)))
    assert wn.wn_get_config_ex(many)[2] != wn.WN_CFG_CHAIN
    mixed = wn.wn_create_streams([1024, 4096], [2, 2], [1, 2])
    assert wn.wn_get_config_ex(mixed)[2] != wn.WN_CFG_CHAIN
    # the default for a lone stream gives the oracle's values (long call:
    # thousands of blocks through the scale hand-over)
    _run_calls(wn, h, 1024, 2, [1], [3000 * 1023 + 17, 2048])


def test_chain_many_streams_and_every_alignment(wn):
    # more streams than SMs (several waves), counts giving each stream's slice
    # another alignment; the last stream against the oracle, all against the
    # group-mode kernel within the FP32 tolerance with identical integer state
    import torch
    from _parity import C_MAX, U
    N, R, n, count = 1024, 4, 300, 7 * 1023 + 3
    seeds = list(range(500, 500 + n))
    hc = _handle(wn, N, R, seeds, (1024, 2, 128))
    hg = wn.wn_create_streams([N] * n, [R] * n, seeds)
    a = _gen(wn, hc, count).double()
    b = _gen(wn, hg, count).double()
    P = torch.from_numpy(passes_fresh(count, N, R).astype(np.float64)).cuda() + R
    tol = 2 * C_MAX * U * torch.sqrt(P) * (1 + b.view(n, count).abs())
    assert bool(((a - b).view(n, count).abs() <= tol).all())
    for i in range(0, n, 37):
        sc, sg = wn.wn_get_state(hc, i), wn.wn_get_state(hg, i)
        assert (sc["x"], sc["w"], sc["k"], sc["blocks"]) == (sg["x"], sg["w"], sg["k"], sg["blocks"])
    assert_fp32_close(a.view(n, count)[-1].cpu().numpy(), oracle.Stream(N, R, seeds[-1]).generate(count),
                      passes_fresh(count, N, R) + R, "last stream")


def test_chain_and_other_kernels_interleave(wn):
    # chain -> group -> ordinary -> chain on one handle: each call continues
    # where the other left the state (pool, reserved value, scale, sum of squares)
    N, R, seeds = 4096, 2, [5, 6]
    h = _handle(wn, N, R, seeds, (4096, 4, 256))
    refs = [oracle.Stream(N, R, s) for s in seeds]
    done = 0
    for c, mode in ((9000, "chain"), (7001, "group"), (5000, "ordinary"), (12001, "chain")):
        if mode == "chain":
            wn.wn_set_config_ex(h, 4, 256, wn.WN_CFG_CHAIN)
        elif mode == "group":
            wn.wn_set_config_ex(h, 32, 32, wn.WN_CFG_GROUP)
        else:
            wn.wn_set_config(h, 8, 128)
        got = _gen(wn, h, c).cpu().numpy().reshape(len(seeds), c)
        for i, s in enumerate(refs):
            assert_fp32_close(got[i], s.generate(c), passes_fresh(c, N, R, first_block=done // (N - 1)) + R,
                              f"call of {c} ({mode}) stream {i}")
        done += c


@pytest.mark.parametrize("dtype", [1, 2])
def test_chain_16bit_outputs_round_fp32_values(wn, dtype):
    N, R, seeds, count = 4096, 3, [3, 4, 5], 3 * 4095 + 9
    f32 = _gen(wn, _handle(wn, N, R, seeds, (4096, 4, 256)), count)
    low = _gen(wn, _handle(wn, N, R, seeds, (4096, 4, 256)), count, dtype)
    assert bool((low == f32.to(low.dtype)).all())


def test_chain_rejects_other_shapes_and_variants(wn):
    h = wn.wn_create_streams([4096] * 2, [2] * 2, [1, 2])
    with pytest.raises(wn.WnError):
        wn.wn_set_config_ex(h, 2, 256, wn.WN_CFG_CHAIN)   # covers 2048, not 4096
    with pytest.raises(wn.WnError):
        wn.wn_set_config_ex(h, 8, 128, wn.WN_CFG_CHAIN)   # four warps: no such compiled shape for 4096
    with pytest.raises(wn.WnError):
        wn.wn_set_config_ex(h, 4, 256, wn.WN_CFG_CHAIN | wn.WN_CFG_GROUP)
    hv = wn.wn_create_ex([4096] * 2, [2] * 2, [1, 2], chi2="a")
    with pytest.raises(wn.WnError):
        wn.wn_set_config_ex(hv, 4, 256, wn.WN_CFG_CHAIN)  # variants keep the general kernels
    hm = wn.wn_create_streams([4096, 1024], [2, 2], [1, 2])
    with pytest.raises(wn.WnError):
        wn.wn_set_config_ex(hm, 4, 256, wn.WN_CFG_CHAIN)  # mixed pool sizes


def test_batch_chain_groups_in_chain_mode(wn):
    # the longest requests of every pool size in chain groups (chain mode,
    # persistent, one to four CTAs per SM), the rest in the throughput groups;
    # packed slices (every alignment), partial blocks, empty requests
    import torch
    rng = np.random.default_rng(77)
    n = 48
    N = rng.choice(np.array([1024, 2048, 4096, 8192, 16384], dtype=np.uint32), size=n)
    R = rng.choice(np.array([1, 2, 3, 4], dtype=np.uint32), size=n)
    counts = rng.integers(0, 50000, size=n).astype(np.uint64)
    counts[:6] = [300000, 260000, 200000, 90000, 0, 1]
    seeds = np.arange(900, 900 + n)
    offsets = packed_offsets(counts) + 3
    out = torch.zeros(int(counts.sum()) + 8, dtype=torch.float32, device="cuda")
    for chains, density, graph in ((12, 1, False), (20, 4, True)):
        h = wn.wn_create_streams(N, R, seeds)
        wn.wn_set_batch_plan(h, chains, density)
        wn.wn_set_batch_chain_kernel(h, True)
        for call in range(2):
            out.zero_()
            wn.wn_generate_batch(out, counts, offsets, h, use_graph=graph)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            for i in range(n):
                c = int(counts[i])
                if c == 0:
                    continue
                s = oracle.Stream(int(N[i]), int(R[i]), int(seeds[i]))
                s.skip(call * c)
                fb = call * c // (int(N[i]) - 1)
                assert_fp32_close(got[int(offsets[i]): int(offsets[i]) + c], s.generate(c),
                                  passes_fresh(c, int(N[i]), int(R[i]), first_block=fb) + int(R[i]),
                                  f"plan ({chains}, {density}) call {call} stream {i} N={N[i]} R={R[i]}")
