"""Pins for the oracle's integer generators (Sections 3 and 5.8).

The uniform generator only selects transformations and seeds the pool; the
paper asks for a long period from little state (Section 3) and notes that one
use per pool bounds the normal generator's period below by the uniform one's
(Section 5.8).  Each test checks the oracle against something other than
itself: published known-answer values, or the algebra of the generator.
"""
import decimal

import numpy as np
import pytest

import oracle
from _golden import fields, lines

MASK64 = (1 << 64) - 1


def test_splitmix64_known_answers():
    expected = [int(s, 16) for s in lines("splitmix64_kat.txt")]
    state, got = 0, []
    for _ in expected:
        state, z = oracle.splitmix64(state)
        got.append(z)
    assert got == expected


def test_golden_gamma_and_weyl_constant():
    # SplitMix64's increment is the odd integer nearest 2^64/phi; the Weyl
    # increment is its negation mod 2^64, so it is odd and the Weyl sequence
    # has full period 2^64.
    decimal.getcontext().prec = 60
    phi = (1 + decimal.Decimal(5).sqrt()) / 2
    gamma = int(decimal.Decimal(2 ** 64) / phi)
    assert gamma == 0x9E3779B97F4A7C15 and gamma % 2 == 1
    # the Weyl step: draws(seed) = x_i + w_i with w_i = w_0 + i*omega
    seed = 12345
    s1, x0 = oracle.splitmix64(seed)
    _, w0 = oracle.splitmix64(s1)
    d = oracle.draws(seed, 5)
    x = x0
    omega = (-gamma) & MASK64
    assert omega == 0x61C8864680B583EB
    for i in range(5):
        x = oracle.xorshift64_step(x)
        assert int(d[i]) == (x + w0 + (i + 1) * omega) & MASK64


def test_xorshift_known_answers():
    seq = [int(s) for s in lines("xorshift64_kat.txt")]
    x = seq[0]
    for want in seq[1:]:
        x = oracle.xorshift64_step(x)
        assert x == want


def _gf2_matrix_of(step):
    """Columns of the 64x64 GF(2) matrix of a linear map on 64-bit words."""
    return [step(1 << j) for j in range(64)]


def _gf2_apply(cols, v):
    r = 0
    j = 0
    while v:
        if v & 1:
            r ^= cols[j]
        v >>= 1
        j += 1
    return r


def _gf2_mul(a, b):
    return [_gf2_apply(a, c) for c in b]


def _gf2_pow(a, e):
    result = [1 << j for j in range(64)]
    base = a
    while e:
        if e & 1:
            result = _gf2_mul(result, base)
        base = _gf2_mul(base, base)
        e >>= 1
    return result


def test_xorshift_full_period():
    # The step is linear over GF(2); its period on nonzero states is 2^64 - 1
    # iff T^(2^64-1) = I and T^((2^64-1)/p) != I for every prime p | 2^64-1.
    T = _gf2_matrix_of(oracle.xorshift64_step)
    # linearity check on random words
    rng = np.random.default_rng(7)
    for v in rng.integers(0, 2 ** 63, size=8, dtype=np.int64):
        v = int(v) * 2 + 1
        assert oracle.xorshift64_step(v) == _gf2_apply(T, v)
    ident = [1 << j for j in range(64)]
    order = (1 << 64) - 1
    primes = [3, 5, 17, 257, 641, 65537, 6700417]
    prod = 1
    for p in primes:
        prod *= p
    assert prod == order
    assert _gf2_pow(T, order) == ident
    for p in primes:
        assert _gf2_pow(T, order // p) != ident, p


def test_wrong_shift_triple_fails_period():
    # The period test distinguishes: the triple (13, 7, 16) is not full period.
    def bad(x):
        x ^= (x << 13) & MASK64
        x ^= x >> 7
        x ^= (x << 16) & MASK64
        return x
    T = _gf2_matrix_of(bad)
    ident = [1 << j for j in range(64)]
    order = (1 << 64) - 1
    full = _gf2_pow(T, order) == ident and all(
        _gf2_pow(T, order // p) != ident for p in [3, 5, 17, 257, 641, 65537, 6700417])
    assert not full


def test_philox_known_answers():
    for ctr, key, out in fields("philox4x32_10_kat.txt"):
        got = oracle.philox4x32_10([int(c, 16) for c in ctr], [int(k, 16) for k in key])
        assert got == [int(o, 16) for o in out]
