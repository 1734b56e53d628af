"""Block sum-of-squares statistics of the GPU output (Section 5.5).

The pool's sum of squares is invariant under the orthogonal passes, so
without a correction every block of N-1 returned values would have the same
sum of squares up to the one held-back value.  The chi-squared correction
scales block b so that the pool's sum of squares is a chi-squared_N sample
S_b drawn from the value held back by the previous block; the returned block
then has

    SS_b = (S_b / N) (N - P_{N-1}^2):  mean N - 1,  variance about 2N - 2,

and successive blocks' sums are uncorrelated (S_b depends on block b-1 only
through one value that block b-1 did not return).  With the correction off,
SS_b = N - P_{N-1}^2 has variance Var(x^2) = 2 and never exceeds N.

These run on the launch the many-streams workload uses (more streams than
half the SMs: the ordinary generate kernel), 160 streams x 2500 blocks of
pool 256, so the pooled estimates have standard errors of a few tenths of a
percent.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N, R, STREAMS, BLOCKS = 256, 2, 160, 2500


def _block_sums(wn, **opt):
    import torch
    h = wn.wn_create_ex([N] * STREAMS, [R] * STREAMS, list(range(500, 500 + STREAMS)), **opt)
    count = BLOCKS * (N - 1)
    out = torch.empty(STREAMS * count, dtype=torch.float32, device="cuda")
    wn.wn_generate(out, count, h)
    ss = out.view(STREAMS, BLOCKS, N - 1).double().pow(2).sum(-1)
    torch.cuda.synchronize()
    return ss.cpu().numpy()


def test_block_sums_have_chi_squared_spread_and_no_lag_one_correlation(wn):
    ss = _block_sums(wn)
    n = ss.size
    mean, var = float(ss.mean()), float(ss.var())
    assert abs(mean - (N - 1)) < 5 * math.sqrt(2 * N / n), mean
    assert abs(var / (2 * N - 2) - 1) < 0.03, var
    # lag-1 correlation of successive blocks within each stream, pooled
    a = ss[:, :-1] - ss[:, :-1].mean(axis=1, keepdims=True)
    b = ss[:, 1:] - ss[:, 1:].mean(axis=1, keepdims=True)
    rho = float(np.sum(a * b) / math.sqrt(np.sum(a * a) * np.sum(b * b)))
    assert abs(rho) < 5 / math.sqrt(a.size), rho
    # and no stream on its own shows a correlation beyond 5 sigma
    per = np.sum(a * b, axis=1) / np.sqrt(np.sum(a * a, axis=1) * np.sum(b * b, axis=1))
    assert np.max(np.abs(per)) < 5 / math.sqrt(BLOCKS - 1), float(np.max(np.abs(per)))


def test_block_sums_collapse_without_the_correction(wn):
    ss = _block_sums(wn, chi2="off")
    # N - P^2: at most N (up to the FP32 rounding of the renormalisation),
    # variance Var(x^2) = 2, mean N - 1
    assert float(ss.max()) <= N + 1e-3
    assert abs(float(ss.var()) - 2.0) < 0.1, float(ss.var())
    assert abs(float(ss.mean()) - (N - 1)) < 5 * math.sqrt(2 / ss.size)
