"""The method's variants on the GPU against the FP64 oracle (wn_create_ex).

Section 5.5: the chi-squared approximations (a) rann4's, (b) Wilson-Hilferty,
no correction; fastnorm's reserved value taken from the current pool.
Section 5.7: pool decimation (the values of every d-th block).  Section
5.3: rann4's plane rotations in place of the 4x4 update.  Integers
(generator words, block counts) bit-exact; FP32 values within the error
model of tests/_parity.py, where a decimated stream's returned block b has
seen R (W + d (b + 1)) passes.
"""
import numpy as np
import pytest

import oracle
from _parity import assert_fp32_close

pytestmark = pytest.mark.gpu
W = 8


def _gen(wn, h, count, dtype=0):
    import torch
    tdt = {0: torch.float32, 1: torch.bfloat16}[dtype]
    out = torch.empty(count * h.n, dtype=tdt, device="cuda")
    wn.wn_generate_ex(out, count, h, dtype)
    torch.cuda.synchronize()
    return out.float().cpu().numpy().reshape(h.n, count)


def _passes(count, N, R, d=1, first=0):
    b = np.arange(count, dtype=np.int64) // (N - 1) + first
    return R * (W + d * (b + 1))


def _check(wn, N, R, chi2="c", reserve="previous", d=1, seeds=(3, 4), chunks=(None,), update="quad"):
    h = wn.wn_create_ex([N] * len(seeds), [R] * len(seeds), list(seeds), chi2=chi2, reserve=reserve, decimate=d,
                        update=update)
    refs = [oracle.Stream(N, R, s, chi2=chi2, reserve=reserve, decimate=d, update=update) for s in seeds]
    done = 0
    for c in chunks:
        c = c if c is not None else 4 * (N - 1) + 5
        got = _gen(wn, h, c)
        for i, ref in enumerate(refs):
            assert_fp32_close(got[i], ref.generate(c), _passes(c, N, R, d, first=done // (N - 1)),
                              f"N={N} R={R} chi2={chi2} reserve={reserve} d={d} update={update}")
        done += c
    for i, ref in enumerate(refs):
        st = wn.wn_get_state(h, i)
        assert (st["x"], st["w"]) == ref.gen_state
        assert st["blocks"] == ref.blocks and st["k"] == ref.k


@pytest.mark.parametrize("chi2", ["off", "a", "b"])
@pytest.mark.parametrize("N,R", [(1024, 2), (64, 1), (4096, 3)])
def test_chi2_approximations(wn, chi2, N, R):
    _check(wn, N, R, chi2=chi2)


@pytest.mark.parametrize("N,R", [(1024, 2), (256, 1), (4096, 2), (16, 3)])
def test_reserve_from_current_pool(wn, N, R):
    _check(wn, N, R, reserve="current")


@pytest.mark.parametrize("N,R,d", [(1024, 2, 3), (64, 1, 3), (4096, 2, 2), (256, 3, 5)])
def test_pool_decimation(wn, N, R, d):
    # calls cut blocks anywhere: the leftover of a returned block carries over
    _check(wn, N, R, d=d, chunks=(1, N - 2, 3 * (N - 1) + 7, N))


@pytest.mark.parametrize("N,R", [(1024, 4), (64, 3), (4096, 2), (16384, 1), (16, 5)])
def test_rotation_form(wn, N, R):
    _check(wn, N, R, update="rotation", chunks=(N - 2, 3 * (N - 1) + 7))


def test_rotation_with_other_variants(wn):
    _check(wn, 256, 2, update="rotation", chi2="a", d=3)
    _check(wn, 1024, 1, update="rotation", reserve="current", chi2="b")


def test_rotation_batch_equals_per_stream(wn):
    import torch
    Ns, Rs = [1024, 4096, 64], [4, 2, 3]
    counts = np.array([5000, 70_000, 333], dtype=np.uint64)
    offs = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.uint64)
    ha = wn.wn_create_ex(Ns, Rs, [7, 8, 9], update="rotation")
    out = torch.empty(int(counts.sum()), device="cuda")
    wn.wn_generate_batch(out, counts, offs, ha, wn.WN_F32, True)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i in range(3):
        hb = wn.wn_create_ex([Ns[i]], [Rs[i]], [7 + i], update="rotation")
        assert np.array_equal(got[int(offs[i]):int(offs[i] + counts[i])], _gen(wn, hb, int(counts[i]))[0])


def test_variants_combined_and_16bit(wn):
    N, R, d = 1024, 2, 3
    h = wn.wn_create_ex([N] * 2, [R] * 2, [5, 6], chi2="b", reserve="current", decimate=d)
    got = _gen(wn, h, 3 * (N - 1) + 1, dtype=1)
    for i, s in enumerate((5, 6)):
        ref = oracle.Stream(N, R, s, chi2="b", reserve="current", decimate=d).generate(3 * (N - 1) + 1)
        assert np.all(np.abs(got[i] - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5 * (1 + np.abs(ref)))


def test_decimated_batch_equals_per_stream(wn):
    import torch
    Ns, Rs = [1024, 4096, 64], [2, 1, 3]
    counts = np.array([5000, 70_000, 333], dtype=np.uint64)
    offs = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.uint64)
    ha = wn.wn_create_ex(Ns, Rs, [7, 8, 9], decimate=3, chi2="a")
    out = torch.empty(int(counts.sum()), device="cuda")
    wn.wn_generate_batch(out, counts, offs, ha, wn.WN_F32, False)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i in range(3):
        hb = wn.wn_create_ex([Ns[i]], [Rs[i]], [7 + i], decimate=3, chi2="a")
        ref = _gen(wn, hb, int(counts[i]))[0]
        assert np.array_equal(got[int(offs[i]):int(offs[i] + counts[i])], ref)


def test_decimation_resumes_from_checkpoint(wn):
    h = wn.wn_create_ex([1024, 64], [2, 1], [1, 2], decimate=3, reserve="current", chi2="off")
    _gen(wn, h, 1500)
    buf = wn.wn_save(h)
    a = _gen(wn, h, 4000)
    b = _gen(wn, wn.wn_load(buf), 4000)
    assert np.array_equal(a, b)


def test_options_out_of_range_rejected(wn):
    with pytest.raises(wn.WnError):
        wn.wn_create_ex([64], [2], [1], decimate=0)
    with pytest.raises(wn.WnError):
        wn.wn_create_ex([64], [2], [1], decimate=256)
    with pytest.raises(ValueError):
        wn.wn_create_ex([64], [2], [1], chi2="d")
    with pytest.raises(ValueError):
        wn.wn_create_ex([64], [2], [1], update="hex")
