"""Pins of the oracle's plane-rotation form (Section 5.3, rann4's update) with
the affine gather of Section 5.4.

The rotation is built from t = tan(theta/2) without trigonometry
(c = (1-t^2)/(1+t^2), s = 2t/(1+t^2)); the tests check it against sin and
cos of theta = 2 atan t, an independent route, plus the structural facts that
fix the pass: orthogonality, an exact inverse, two inputs per output, and the
reach of the mixing.
"""
import math

import numpy as np
import pytest

import oracle


def _cs(w_t):
    th = 2.0 * math.atan(oracle.rot_t(w_t))
    return math.cos(th), math.sin(th)


def test_hand_worked_pass_n4():
    # alpha = 1, gamma = 0 (w_a = 0): pairs (P0, P2) -> slots 0, 1 and (P1, P3) -> slots 2, 3
    w_t = 0x9E3779B97F4A7C15
    c, s = _cs(w_t)
    P = np.array([1.0, 2.0, 3.0, 4.0])
    want = np.array([c * 1 + s * 3, -s * 1 + c * 3, c * 2 + s * 4, -s * 2 + c * 4])
    assert np.allclose(oracle.pass_rot(4, P, 0, w_t), want, rtol=0, atol=1e-14)


def test_t_range_and_symmetry():
    rng = np.random.default_rng(1)
    for w in rng.integers(0, 2**63, size=200, dtype=np.uint64):
        w = int(w) * 2 + 1
        t = oracle.rot_t(w)
        assert -1.0 < t < 1.0
        assert oracle.rot_t(w ^ ((1 << 64) - 1)) == -t  # u -> 2^24 - 1 - u
    assert oracle.rot_t(0) == -1 + 2.0 ** -24 and oracle.rot_t((1 << 64) - 1) == 1 - 2.0 ** -24


@pytest.mark.parametrize("N", [4, 16, 256])
def test_orthogonal_inverse_and_two_inputs_per_output(N):
    rng = np.random.default_rng(N)
    for _ in range(10):
        w_a, w_t = (int(v) for v in rng.integers(0, 2**63, size=2, dtype=np.uint64))
        P = rng.standard_normal(N)
        Q = oracle.pass_rot(N, P, w_a, w_t)
        assert abs(np.dot(Q, Q) - np.dot(P, P)) < 1e-13 * np.dot(P, P)
        assert np.allclose(oracle.pass_rot_inverse(N, Q, w_a, w_t), P, rtol=0, atol=1e-14)
        c, s = _cs(w_t)
        for i in rng.integers(0, N, size=4):
            e = np.zeros(N)
            e[i] = 1.0
            y = oracle.pass_rot(N, e, w_a, w_t)
            nz = np.nonzero(np.abs(y) > 1e-15)[0]
            assert len(nz) <= 2 and nz[0] // 2 == nz[-1] // 2  # one pair of slots
            assert np.allclose(sorted(np.abs(y[nz])), sorted([abs(c), abs(s)])[-len(nz):], atol=1e-14)


def test_mixing_reach_log2_n_passes():
    # after p passes an output depends on at most 2^p inputs; with the
    # transposed write every output depends on every input after log2 N passes
    N, seed = 64, 3
    d = oracle.draws(seed, 64)
    M = np.eye(N)
    for p in range(10):
        M = np.column_stack([oracle.pass_rot(N, M[:, i], int(d[2 * p]), int(d[2 * p + 1])) for i in range(N)])
        dep = np.abs(M) > 1e-12
        assert dep.sum(axis=1).max() <= 2 ** (p + 1)
        if p + 1 == 6:
            assert dep.all()


def test_rotation_stream_moments_and_continuation():
    N, R = 256, 4
    s = oracle.Stream(N, R, 7, update="rotation")
    x = s.generate(400_000)
    n = x.size
    assert abs(x.mean()) < 5 / math.sqrt(n)
    assert abs(x.var() - 1) < 5 * math.sqrt(2 / n)
    k = np.mean(x ** 4) / x.var() ** 2
    assert abs(k - 3) < 5 * math.sqrt(24 / n)
    a = oracle.Stream(N, R, 7, update="rotation")
    parts = np.concatenate([a.generate(c) for c in (1, 254, 3000, 17)])
    assert np.array_equal(parts, oracle.Stream(N, R, 7, update="rotation").generate(parts.size))
    with pytest.raises(ValueError):
        oracle.Stream(N, R, 7, update="other")


def test_warmup_blocks_use_the_rotation_form():
    # the initial pool is the same for both updates; a warm-up block then
    # applies R rotation passes (draws after the N used by the initial pool)
    # and renormalises to sum of squares N
    N, R, seed = 64, 3, 11
    P0 = oracle.Stream(N, R, seed, warmup=0, update="rotation").pool
    assert np.array_equal(P0, oracle.Stream(N, R, seed, warmup=0).pool)
    d = oracle.draws(seed, N + 2 * R)
    P = P0
    for p in range(R):
        P = oracle.pass_rot(N, P, int(d[N + 2 * p]), int(d[N + 2 * p + 1]))
    P = P * math.sqrt(N / np.dot(P, P))
    assert np.allclose(oracle.Stream(N, R, seed, warmup=1, update="rotation").pool, P, rtol=0, atol=1e-13)
    assert not np.allclose(oracle.Stream(N, R, seed, warmup=1).pool, P, atol=1e-3)
