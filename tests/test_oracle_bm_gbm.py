"""Pins for the oracle's comparison generator and Monte Carlo consumer.

Box-Muller (the conventional method Section 5 compares against): for
u1 in (0,1], u2 in [0,1), (rho cos 2 pi u2, rho sin 2 pi u2) with
rho^2 = -2 ln u1 is a pair of iid N(0,1); rho^2 is exponential with mean 2.
Geometric Brownian motion with the exact log step: S_T is lognormal with
E S_T = S0 e^{mu T} and Var S_T = S0^2 e^{2 mu T}(e^{sigma^2 T} - 1).
"""
import math

import numpy as np

import oracle


def test_boxmuller_pairs_from_philox_words():
    # the first pair of stream 3, seed 11 comes from Philox block 0's words 0, 1
    w = oracle.philox4x32_10([0, 0, 3, 0], [11, 0])
    z = oracle.boxmuller(11, 3, 0, 4)
    for pair in range(2):
        u1 = ((w[2 * pair] >> 8) + 1) / 2 ** 24
        u2 = (w[2 * pair + 1] >> 8) / 2 ** 24
        rho2 = z[2 * pair] ** 2 + z[2 * pair + 1] ** 2
        assert abs(rho2 + 2 * math.log(u1)) < 1e-12 * max(1.0, rho2)
        ang = math.atan2(z[2 * pair + 1], z[2 * pair]) % (2 * math.pi)
        assert abs(ang - 2 * math.pi * u2) < 1e-9 or abs(ang - 2 * math.pi * u2) > 2 * math.pi - 1e-9


def test_boxmuller_offsets_are_consistent():
    a = oracle.boxmuller(5, 7, 0, 1000)
    b = oracle.boxmuller(5, 7, 333, 667)
    assert np.array_equal(a[333:], b)


def test_boxmuller_moments_and_radius_law():
    n = 1 << 21
    z = oracle.boxmuller(1, 0, 0, n)
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / n)
    kurt = np.mean(z ** 4) / z.var() ** 2
    assert abs(kurt - 3) < 5 * math.sqrt(24 / n)
    r2 = z[0::2] ** 2 + z[1::2] ** 2
    for t in (0.5, 2.0, 6.0):
        p = np.mean(r2 > t)
        q = math.exp(-t / 2)
        assert abs(p - q) < 5 * math.sqrt(q * (1 - q) / r2.size)


def test_gbm_terminal_moments_closed_form():
    S0, mu, sigma, T, steps = 100.0, 0.05, 0.2, 1.0, 252
    n = 1 << 16
    ST = oracle.gbm(n, 4095, steps, 4096, 2, S0, mu, sigma, T / steps)
    mean = S0 * math.exp(mu * T)
    var = S0 ** 2 * math.exp(2 * mu * T) * (math.exp(sigma ** 2 * T) - 1)
    assert abs(mean - 105.12710963760242) < 1e-9
    assert abs(var - 451.0288078157963) < 1e-9
    m = ST.mean()
    v = ST.var()
    se_m = ST.std() / math.sqrt(n)
    se_v = math.sqrt(np.mean((ST - m) ** 4) - v ** 2) / math.sqrt(n)
    assert abs(m - mean) < 5 * se_m
    assert abs(v - var) < 5 * se_v
