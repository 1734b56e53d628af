"""Pins for the oracle's whole stream: init, blocks, chi-squared correction.

Section 5.1: the output should look iid N(0,1).  Section 5.5: with the pool's
sum of squares invariant, a block's N-1 outputs would have an almost constant
sum of squares; the chi-squared correction restores its spread (variance
about 2N) and, taking the reserved value from the previous pool (fastnorm2),
avoids the negative correlation between the scale and the remaining sum of
squares that fastnorm's current-pool choice causes.
"""
import math

import numpy as np
import pytest

import oracle


def _z(est, mean, se):
    return abs(est - mean) / se


@pytest.mark.parametrize("N", [4, 64, 1024, 16384])
def test_init_pool_integers_scaled_to_sum_N(N):
    s = oracle.Stream(N, 2, seed=77, warmup=0)
    P = s.pool
    assert abs(np.sum(P * P) - N) < 1e-12 * N
    # P = v * sqrt(N / sum v^2) with v even integers in [-262140, 262140]:
    # recover the scale from the generator's draws, which fix v
    d = oracle.draws(77, N)
    v = np.zeros(N)
    for f in range(4):
        v += ((d >> np.uint64(16 * f)) & np.uint64(0xFFFF)).astype(np.float64)
    v = 2 * v - 4 * 65535
    assert np.all(np.abs(v) <= 262140) and np.all(v % 2 == 0)
    scale = math.sqrt(N / float(np.sum(v * v)))
    assert np.array_equal(P, v * scale)
    assert s.k == N - 1 and s.blocks == 0 and s.r == 0.0


def test_generator_advances_two_draws_per_pass():
    # Section 5.8: U ~ 1/n uniforms per normal: N init draws, then 2 per pass.
    N, R, W = 64, 3, 5
    s = oracle.Stream(N, R, seed=9, warmup=W)
    d = oracle.draws(9, N + 2 * R * W + 2 * R)
    x, w = s.gen_state
    assert (x + w) % (1 << 64) == int(d[N + 2 * R * W - 1])
    s.generate(1)
    x, w = s.gen_state
    assert (x + w) % (1 << 64) == int(d[N + 2 * R * W + 2 * R - 1])


@pytest.mark.parametrize("N,R", [(4, 1), (16, 2), (1024, 2), (4096, 3)])
def test_continuation_across_calls(N, R):
    a = oracle.Stream(N, R, seed=5)
    b = oracle.Stream(N, R, seed=5)
    total = 3 * N + 17
    whole = a.generate(total)
    parts = []
    for c in (1, N - 2, 0, N + 5, 3, total - (1 + N - 2 + N + 5 + 3)):
        parts.append(b.generate(c))
    assert np.array_equal(np.concatenate(parts), whole)


@pytest.mark.parametrize("N,R", [(1024, 2), (4096, 2), (16384, 3)])
def test_output_moments(N, R):
    n = 1 << 22
    x = oracle.Stream(N, R, seed=1).generate(n)
    m = x.mean()
    v = x.var()
    kurt = np.mean((x - m) ** 4) / v ** 2
    assert _z(m, 0.0, 1 / math.sqrt(n)) < 5
    assert _z(v, 1.0, math.sqrt(2 / n)) < 5
    assert _z(kurt, 3.0, math.sqrt(24 / n)) < 5
    # third moment
    assert _z(np.mean(x ** 3), 0.0, math.sqrt(15 / n)) < 5


def _block_sums(N, R, nblocks, **kw):
    s = oracle.Stream(N, R, seed=3, **kw)
    x = s.generate(nblocks * (N - 1)).reshape(nblocks, N - 1)
    return np.sum(x * x, axis=1)


def test_block_sum_of_squares_spread_restored():
    N, B = 256, 20000
    ss = _block_sums(N, 2, B)
    # SS_b = (S/N)(N - P_{N-1}^2): mean about N - 1, variance about 2N
    assert _z(ss.mean(), N - 1, math.sqrt(2 * N / B)) < 5
    assert 0.85 < ss.var() / (2 * N) < 1.15
    # successive blocks' sums of squares are uncorrelated
    rho = np.corrcoef(ss[:-1], ss[1:])[0, 1]
    assert abs(rho) < 5 / math.sqrt(B)


def test_block_sum_of_squares_collapses_without_correction():
    # with g = 1 the block sum is N - P_{N-1}^2: variance Var(x^2) = 2
    N, B = 256, 5000
    ss = _block_sums(N, 2, B, chi2="off")
    assert ss.max() <= N + 1e-9
    assert 1.5 < ss.var() < 2.6


def test_current_pool_reserve_correlates_scale_with_remainder():
    # Section 5.5: taking x from the current pool ties a large scale to a
    # small remaining sum of squares; taking it from the previous pool does not.
    N, B = 64, 40000

    def corr(reserve):
        s = oracle.Stream(N, 2, seed=4, reserve=reserve)
        g2 = np.empty(B)
        rem = np.empty(B)
        for b in range(B):
            x = s.generate(N - 1)
            g2[b] = s.g ** 2
            rem[b] = np.sum((x / s.g) ** 2)
        return np.corrcoef(g2, rem)[0, 1]

    # current pool: g^2 = S(x)/N and the remainder is N - x^2 with x the
    # pool's own reserved value, so corr = -Cov(A x^2, x^2)/(sd S sd x^2)
    # = -2A / (sqrt(2N) sqrt(2)) = -A / sqrt(N)
    want = -oracle.chi2_A(N) / math.sqrt(N)
    assert abs(corr("current") - want) < 5 / math.sqrt(B)
    assert abs(corr("previous")) < 5 / math.sqrt(B)


def test_other_chi2_approximations_run():
    for kind in ("a", "b"):
        x = oracle.Stream(1024, 2, seed=2, chi2=kind).generate(1 << 20)
        assert _z(x.var(), 1.0, math.sqrt(2 / x.size)) < 5


def test_invalid_parameters_rejected():
    for N, R in [(0, 1), (3, 1), (12, 1), (1024, 0)]:
        with pytest.raises(ValueError):
            oracle.Stream(N, R, seed=1)


@pytest.mark.parametrize("N,R,d", [(16, 2, 3), (64, 1, 2), (32, 3, 5)])
def test_pool_decimation_returns_every_dth_block(N, R, d):
    # Section 5.7's remedy of keeping only one pool in three.  The decimated stream's
    # j-th returned block is block (j+1) d - 1 of the plain stream with the
    # same seed (the blocks between run in full and return nothing).
    B = 6
    plain = oracle.Stream(N, R, 5).generate(B * d * (N - 1)).reshape(B * d, N - 1)
    dec = oracle.Stream(N, R, 5, decimate=d).generate(B * (N - 1)).reshape(B, N - 1)
    assert np.array_equal(dec, plain[d - 1::d])


def test_pool_decimation_draw_count():
    # each returned block costs d blocks of 2R draws
    N, R, d, seed = 16, 2, 3, 9
    s = oracle.Stream(N, R, seed, decimate=d)
    before = s.gen_state
    s.generate(1)
    ref = oracle.Stream(N, R, seed)
    assert ref.gen_state == before
    ref.generate(d * (N - 1))
    assert s.gen_state == ref.gen_state
    with pytest.raises(ValueError):
        oracle.Stream(N, R, seed, decimate=0)


def test_finite_pool_covariances_match_the_sphere_closed_forms():
    # Section 5.6's effect on the oracle's own stream: a squared value and its
    # next-block descendants (positions fixed by the pass permutations) have
    # the covariances of a pool on the sphere sum P^2 = N -- energy
    # (2N - 2 4^R)/(N+2), one descendant (2N 4^-R - 2)/(N+2), a
    # non-descendant -2/(N+2) -- each within 5 standard errors; here the
    # -2/(N+2) terms exceed 5 standard errors, so a dropped sphere term fails
    from _defects import _draws, energy_covariances, expected_covariances
    N, R, seed, blocks = 256, 1, 31, 60000
    out = oracle.Stream(N, R, seed).generate(blocks * (N - 1)).reshape(blocks, N - 1)
    mean, se = energy_covariances(out, N, R, _draws(N, R, seed, blocks))
    expect = expected_covariances(N, R)
    assert np.all(np.abs(mean - expect) < 5 * se), (mean, se, expect)
    assert abs(mean[2]) > 5 * se[2]
    assert abs(mean[0] - (2.0 - 2.0 * 4.0 ** R / N)) > 5 * se[0] or abs(mean[1] - 2 * 4.0 ** -R) > 5 * se[1]
