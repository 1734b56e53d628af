"""Finite-pool statistics of a stream (Sections 5.6 and 5.7): where each pool
value's descendants sit in the next block, and the covariance of a squared
value with its descendants' squares.  Shared by the GPU defect tests and the
CPU test that pins the closed forms on the oracle's own output.
"""
import math

import numpy as np

import oracle

W = 8


def _draws(N, R, seed, blocks):
    return oracle.draws(seed, N + 2 * R * (W + blocks + 1))


def _descendants(N, R, d, b):
    """(N, 4^R) positions in block b+1 that pool position i of block b feeds;
    d: the stream's draws (N for the initial pool, then 2 R per block)."""
    off = N + 2 * R * (W + b + 1)  # block b+1's draws
    desc = np.arange(N)[:, None]
    for p in range(R):
        slots = oracle.pass_read_slots(N, int(d[off + 2 * p]))
        q_of = np.empty(N, dtype=np.int64)
        q_of[slots] = np.arange(N) // 4  # the quadruple that reads position i
        desc = (4 * q_of[desc][..., None] + np.arange(4)).reshape(N, -1)
    return desc


def expected_covariances(N, R):
    """Cov of x_i^2 with (its descendants' energy, one descendant, a
    non-descendant) for a pool on the sphere sum P^2 = N."""
    return np.array([(2.0 * N - 2.0 * 4.0 ** R) / (N + 2), (2.0 * N * 4.0 ** -R - 2.0) / (N + 2), -2.0 / (N + 2)])


def energy_covariances(out, N, R, d, step=2):
    """Mean and standard error of the three covariances over block pairs
    (b, b+1), b = 0, step, 2 step, ...; out: (blocks, N-1) values."""
    stats = []
    for b in range(0, out.shape[0] - 1, step):
        stats.append(_energy_stats(out[b], out[b + 1], _descendants(N, R, d, b)))
    s = np.array(stats)
    return s.mean(axis=0), s.std(axis=0) / math.sqrt(len(s))


def _energy_stats(x, y, desc):
    """Per-block covariances of x_i^2 with the energy of its descendants, with one
    descendant, and with a non-descendant quadruple (positions N-1 excluded)."""
    N1 = x.shape[0]
    ok = np.all(desc < N1, axis=1)[:N1]
    d = desc[:N1][ok]
    x2 = x[ok] ** 2
    y2 = y ** 2
    Y = y2[d].sum(axis=1)
    one = y2[d[:, 0]]
    other = y2[(d[:, 0] // 4 * 4 + 4 * 37) % (N1 - 3)]  # a quadruple that x does not feed
    cov = lambda u, v: float(np.mean(u * v) - np.mean(u) * np.mean(v))
    return cov(x2, Y), cov(x2, one), cov(x2, other)
