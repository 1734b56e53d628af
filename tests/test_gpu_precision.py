"""Precision form: pool N = 16384, R = 3, outputs in BF16 and FP16.

The pool stays FP32; only the stored values are rounded (round-to-nearest-
even from the FP32 value).  Each 16-bit output's error against the FP64
oracle is bounded by the type's unit roundoff times |x| (plus, for FP16, the
subnormal spacing) plus the FP32 pool error of tests/_parity.py.  The test
prints the measured maximum and mean relative errors.
"""
import math

import numpy as np
import pytest

import oracle
from _parity import F16_MIN_NORMAL, U, U_BF16, U_F16, passes_fresh

pytestmark = pytest.mark.gpu

N, R = 16384, 3
PER = 1 << 20          # first 2^20 values of each checked stream
STREAMS = [1, 2, 777, 2048, 4096]  # seeds (the full workload uses 1..4096)


@pytest.fixture(scope="module")
def refs():
    return {s: oracle.Stream(N, R, s).generate(PER) for s in STREAMS}


@pytest.mark.parametrize("dtype,name", [(1, "bf16"), (2, "f16")])
def test_16bit_error_against_oracle(wn, refs, dtype, name):
    import torch
    tdt = {1: torch.bfloat16, 2: torch.float16}[dtype]
    h = wn.wn_create_streams([N] * len(STREAMS), [R] * len(STREAMS), STREAMS)
    out = torch.empty(len(STREAMS) * PER, dtype=tdt, device="cuda")
    wn.wn_generate_ex(out, PER, h, dtype)
    torch.cuda.synchronize()
    got = out.float().cpu().numpy().astype(np.float64).reshape(len(STREAMS), PER)
    P = passes_fresh(PER, N, R)
    uu = U_BF16 if dtype == 1 else U_F16
    floor = 0.0 if dtype == 1 else U_F16 * F16_MIN_NORMAL
    rel_max, rel_sum, cnt = 0.0, 0.0, 0
    for i, s in enumerate(STREAMS):
        ref = refs[s]
        err = np.abs(got[i] - ref)
        tol = uu * np.abs(ref) + floor + 10 * U * np.sqrt(P) * (1 + np.abs(ref))
        assert np.all(err <= tol), (name, s, int(np.argmax(err - tol)))
        big = np.abs(ref) > 0.1  # where the FP32 pool's absolute error is < 1e-5 relative
        rel = err[big] / np.abs(ref[big])
        rel_max = max(rel_max, float(rel.max()))
        rel_sum += float(rel.sum())
        cnt += rel.size
    print(f"\n{name}: max relative error {rel_max:.3e} (unit roundoff {uu:.3e}), "
          f"mean {rel_sum / cnt:.3e} over {cnt} values with |x| > 0.1")
    assert rel_max <= uu + 10 * U * math.sqrt(P[-1]) * (1 + 1 / 0.1)


def test_fp32_precision_config_matches_oracle(wn, refs):
    import torch
    from _parity import assert_fp32_close
    h = wn.wn_create_streams([N] * 2, [R] * 2, STREAMS[:2])
    out = torch.empty(2 * PER, dtype=torch.float32, device="cuda")
    wn.wn_generate_ex(out, PER, h, 0)
    torch.cuda.synchronize()
    got = out.cpu().numpy().reshape(2, PER)
    for i, s in enumerate(STREAMS[:2]):
        rms, mx = assert_fp32_close(got[i], refs[s], passes_fresh(PER, N, R), f"N=16384 stream {s}")
        print(f"\nFP32 N=16384 R=3 stream {s}: normalised RMS error {rms:.3f}, max {mx:.2f} (units of u sqrt(P))")


def test_full_precision_launch_sampled(wn, refs):
    # the 16-bit workload in the launch configuration the benchmark times:
    # 4096 streams x 2^21 BF16 values in one launch (the default group-mode
    # shape), checked on sampled streams' first 2^20 values
    import torch
    S, per = 4096, 1 << 21
    h = wn.wn_create_streams([N] * S, [R] * S, list(range(1, S + 1)))
    assert wn.wn_get_config_ex(h) == (32, 128, wn.WN_CFG_IN_PLACE | wn.WN_CFG_GROUP)
    out = torch.empty(S * per, dtype=torch.bfloat16, device="cuda")
    wn.wn_generate_ex(out, per, h, 1)
    torch.cuda.synchronize()
    P = passes_fresh(PER, N, R)
    for s in STREAMS:
        got = out[(s - 1) * per:(s - 1) * per + PER].float().cpu().numpy().astype(np.float64)
        ref = refs[s]
        tol = U_BF16 * np.abs(ref) + 10 * U * np.sqrt(P) * (1 + np.abs(ref))
        assert np.all(np.abs(got - ref) <= tol), (s, int(np.argmax(np.abs(got - ref) - tol)))
    # the last value of every stream is finite and the state advanced by per
    tail = out.view(S, per)[:, -1].float()
    assert bool(torch.isfinite(tail).all())
    assert wn.wn_get_state(h, S - 1)["blocks"] == 8 + -(-per // (N - 1))
    del out
    torch.cuda.empty_cache()
