"""Pins for the oracle's pass: y = Q x built from 4x4 orthogonal blocks.

Sections 5.1-5.4: Q orthogonal keeps an iid N(0,1) vector iid N(0,1);
fastnorm's blocks are the printed matrix A_1 and "similar" ones; random signs
decorrelate y from x; the pool is transposed and permuted each pass so that
every value eventually feeds every other.
"""
import math

import numpy as np
import pytest

import oracle
from _golden import fields


def _paper_A1():
    rows = [list(map(int, r[0])) for r in fields("paper_A1.txt")]
    return 0.5 * np.array(rows, dtype=np.float64)


def test_printed_A1_is_orthogonal():
    A1 = _paper_A1()
    assert np.array_equal(A1 @ A1.T, np.eye(4))


def test_update_equals_printed_A1_up_to_rows_and_signs():
    # The oracle's quadruple update with sign nibble 0b1001 (negate outputs 0
    # and 3), read back in the order (2, 1, 0, 3), is exactly A_1 x.  With the
    # identity gather (N = 4, alpha = 1, gamma = 0) the quadruple is the pool.
    A1 = _paper_A1()
    rng = np.random.default_rng(3)
    for _ in range(20):
        x = rng.integers(-1000, 1000, size=4).astype(np.float64)
        y = oracle.pass_(4, x, 0, 0b1001)
        assert np.array_equal(A1 @ x, y[[2, 1, 0, 3]])


def test_hand_worked_n4():
    for pool, draws, want in fields("n4_pass_hand.txt"):
        N = int(pool[0])
        P = np.array([float(v) for v in pool[1:]])
        w_a, w_s = int(draws[0]), int(draws[1])
        got = oracle.pass_(N, P, w_a, w_s)
        assert np.array_equal(got, np.array([float(v) for v in want]))


@pytest.mark.parametrize("N", [4, 8, 64, 1024, 16384])
def test_inverse_pass_restores_pool(N):
    rng = np.random.default_rng(N)
    d = oracle.draws(N + 1, 8)
    # integer inputs keep every intermediate exact in FP64
    P = rng.integers(-2 ** 20, 2 ** 20, size=N).astype(np.float64)
    Q = oracle.pass_(N, P, int(d[0]), int(d[1]))
    assert np.array_equal(oracle.pass_inverse(N, Q, int(d[0]), int(d[1])), P)
    # normal inputs: inverse within rounding
    X = rng.standard_normal(N)
    Y = X
    for p in range(4):
        Y = oracle.pass_(N, Y, int(d[2 * p]), int(d[2 * p + 1]))
    for p in reversed(range(4)):
        Y = oracle.pass_inverse(N, Y, int(d[2 * p]), int(d[2 * p + 1]))
    assert np.max(np.abs(Y - X)) < 1e-14 * math.sqrt(N)


@pytest.mark.parametrize("N", [4, 16, 1024, 4096])
def test_sum_of_squares_preserved(N):
    rng = np.random.default_rng(11 * N)
    d = oracle.draws(N, 64)
    P = rng.standard_normal(N)
    s0 = float(np.sum(P * P))
    for p in range(32):
        P = oracle.pass_(N, P, int(d[2 * p]), int(d[2 * p + 1]))
        assert abs(float(np.sum(P * P)) - s0) < 1e-13 * s0


def test_pass_is_linear_orthogonal_matrix():
    # Build Q column by column from unit vectors: Q^T Q = I exactly (entries
    # are 0 or +-1/2, sums of four products of them).
    N = 64
    d = oracle.draws(5, 2)
    Q = np.stack([oracle.pass_(N, np.eye(N)[j], int(d[0]), int(d[1])) for j in range(N)], axis=1)
    assert np.array_equal(Q.T @ Q, np.eye(N))
    assert set(np.unique(Q)) <= {-0.5, 0.0, 0.5}
    assert np.all(np.count_nonzero(Q, axis=1) == 4)


@pytest.mark.parametrize("N", [16, 64, 1024, 4096])
def test_mixing_reaches_whole_pool(N):
    # Each output depends on 4 inputs, so full dependence needs at least
    # ceil(log4 N) passes; brute force shows the transposed, permuted pass
    # reaches it in exactly that many for the generator's own draws.
    need = math.ceil(math.log(N, 4))
    full = (1 << N) - 1
    for seed in (1, 2, 3):
        d = oracle.draws(seed, 2 * (need + 1))
        dep = [1 << i for i in range(N)]
        for p in range(need):
            sl = oracle.pass_read_slots(N, int(d[2 * p]))
            new = [0] * N
            for q in range(N // 4):
                u = dep[sl[4 * q]] | dep[sl[4 * q + 1]] | dep[sl[4 * q + 2]] | dep[sl[4 * q + 3]]
                for k in range(4):
                    new[4 * q + k] = u
            dep = new
            if p + 1 < need:
                assert any(x != full for x in dep)
        assert all(x == full for x in dep)


def test_read_slots_form_a_bijection_with_odd_alpha():
    for N in (4, 32, 4096):
        for w in oracle.draws(9, 16):
            alpha, gamma = oracle.alpha_gamma(N, int(w))
            assert alpha % 2 == 1 and 0 <= gamma < N
            sl = oracle.pass_read_slots(N, int(w))
            assert sorted(sl.tolist()) == list(range(N))
            # quadruple q reads (alpha*(q + k N/4) + gamma) mod N
            q, k = 3 % (N // 4), 2
            assert sl[4 * q + k] == (alpha * (q + k * N // 4) + gamma) % N


def test_fourth_moment_correlation_closed_form():
    # Section 5.6: squares stay correlated across one update.  For
    # y = ((1/2)J - I) x with x iid N(0,1): E(x_i^2 y_j^2) = 3/2 for every
    # pair (i, j), so Cov(x_i^2, y_j^2) = 1/2.  (With the plane rotation of
    # Section 5.6 the analogous value is 2.)
    rng = np.random.default_rng(21)
    n = 400_000
    X = rng.standard_normal((n, 4))
    # the oracle's update on the first rows, then its (linear) matrix on all
    m = 5_000
    Y0 = np.stack([oracle.pass_(4, X[i], 0, 0) for i in range(m)])
    Q = np.stack([oracle.pass_(4, np.eye(4)[j], 0, 0) for j in range(4)], axis=1)
    assert np.allclose(Y0, X[:m] @ Q.T, rtol=0, atol=1e-12)
    Y = X @ Q.T
    for i in range(4):
        for j in range(4):
            v = X[:, i] ** 2 * Y[:, j] ** 2
            se = np.std(v) / math.sqrt(n)
            assert abs(np.mean(v) - 1.5) < 5 * se, (i, j)
