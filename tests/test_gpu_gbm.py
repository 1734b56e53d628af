"""Fused Monte Carlo consumer: geometric Brownian motion driven in-kernel.

Path p of stream c takes value j*ppg + p of the stream's sequence as its
step-j normal (the oracle's definition, oracle.gbm).  Checks: every terminal
price against the FP64 oracle; the stream continues afterwards exactly as if
it had returned steps*ppg values; the closed-form mean and variance of the
lognormal terminal price at 2^20 paths x 252 steps.

Tolerance: the log-return sums steps values in FP32 (sums of magnitude up to
~sqrt(steps) 5, rounding ~1e-6 absolute) and the normals carry the FP32 pool
error (~1e-6); times sigma sqrt(dt) ~ 0.0126 that is ~1e-7 relative in S_T,
plus expf's ~1 ulp: 5e-6 relative is a safe bound.
"""
import math

import numpy as np
import pytest

import oracle
from _parity import assert_fp32_close, passes_fresh

pytestmark = pytest.mark.gpu

S0, MU, SIGMA, STEPS = 100.0, 0.05, 0.2, 252
DT = 1.0 / STEPS


@pytest.mark.parametrize("N,R,ppg", [(4096, 2, 455), (4096, 2, 4095), (4096, 1, 1365), (1024, 2, 341),
                                      (4096, 3, 585)])
def test_gbm_matches_oracle_per_path(wn, N, R, ppg):
    import torch
    G = 5
    h = wn.wn_create_streams([N] * G, [R] * G, list(range(1, G + 1)))
    st = torch.empty(G * ppg, dtype=torch.float32, device="cuda")
    wn.wn_gbm(st, h, ppg, STEPS, S0, MU, SIGMA, DT)
    torch.cuda.synchronize()
    got = st.cpu().numpy().astype(np.float64)
    ref = oracle.gbm(G * ppg, ppg, STEPS, N, R, S0, MU, SIGMA, DT)
    rel = np.abs(got - ref) / ref
    assert rel.max() < 5e-6, float(rel.max())
    # the streams advanced by exactly steps*ppg values
    more = 3 * (N - 1) + 5
    nxt = torch.empty(G * more, dtype=torch.float32, device="cuda")
    wn.wn_generate(nxt, more, h)
    torch.cuda.synchronize()
    nxt = nxt.cpu().numpy().reshape(G, more)
    for c in (0, G - 1):
        s = oracle.Stream(N, R, c + 1)
        s.skip(STEPS * ppg)
        first_block = STEPS * ppg // (N - 1)
        assert_fp32_close(nxt[c], s.generate(more), passes_fresh(more, N, R, first_block=first_block))


def test_gbm_rejects_bad_shapes(wn):
    import torch
    h = wn.wn_create_streams([4096] * 2, [2] * 2, [1, 2])
    st = torch.empty(2 * 4096, dtype=torch.float32, device="cuda")
    with pytest.raises(wn.WnError):
        wn.wn_gbm(st, h, 4096, STEPS, S0, MU, SIGMA, DT)      # does not divide N-1
    with pytest.raises(wn.WnError):
        wn.wn_gbm(st, h, 455, 10, S0, MU, SIGMA, DT)          # 10*455 not whole blocks
    wn.wn_generate(torch.empty(2 * 8, device="cuda"), 7, h)   # leaves a partial block
    with pytest.raises(wn.WnError):
        wn.wn_gbm(st, h, 455, STEPS, S0, MU, SIGMA, DT)


def test_gbm_terminal_moments_full_size(wn):
    # 2^20 paths x 252 steps, pool 4096, R = 2: E S_T = S0 e^{mu}, Var S_T =
    # S0^2 e^{2 mu}(e^{sigma^2} - 1); SE(mean) ~ 0.0207, SE(var) ~ 0.72
    import torch
    N, R, ppg = 4096, 2, 585  # the benchmark's split
    n_paths = 1 << 20
    G = -(-n_paths // ppg)
    h = wn.wn_create_streams([N] * G, [R] * G, list(range(1, G + 1)))
    st = torch.empty(G * ppg, dtype=torch.float32, device="cuda")
    wn.wn_gbm(st, h, ppg, STEPS, S0, MU, SIGMA, DT)
    torch.cuda.synchronize()
    x = st[:n_paths].double().cpu().numpy()
    mean = S0 * math.exp(MU)
    var = S0 ** 2 * math.exp(2 * MU) * (math.exp(SIGMA ** 2) - 1)
    m, v = x.mean(), x.var()
    se_m = x.std() / math.sqrt(n_paths)
    se_v = math.sqrt(np.mean((x - m) ** 4) - v ** 2) / math.sqrt(n_paths)
    assert abs(m - mean) < 5 * se_m, (m, mean, se_m)
    assert abs(v - var) < 5 * se_v, (v, var, se_v)
    # and a sampled set of paths against the oracle
    ref = oracle.gbm(3 * ppg, ppg, STEPS, N, R, S0, MU, SIGMA, DT)
    assert np.max(np.abs(st[: 3 * ppg].double().cpu().numpy() - ref) / ref) < 5e-6
