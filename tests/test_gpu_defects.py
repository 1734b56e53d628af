"""Finite-pool effects of the method (Sections 5.6 and 5.7), measured on the
GPU stream at more than 10^4 n samples, against closed forms.

Every output y of a pass is a +-1/2 combination of four pool values, so a
pool value x and its descendants in the next block are not independent even
though every value is N(0,1) (the E(x^2 y^2) = 2 effect of Section 5.6):

  * the squared value and the total energy of its 4^R descendants have
    covariance exactly 2 (the quadruple map is orthogonal), each single
    descendant 2 c^2 with c = 2^-R its coefficient on x; values that are not
    descendants have covariance 0;
  * a rare large value is followed by large values among its descendants
    (Section 5.7): for R = 1, P(some descendant |y| > 3 | |x| > 4) is the
    model's value (four outputs of one quadruple holding x), far above the
    unconditional 1 - (1 - P(|N(0,1)| > 3))^4 (|y| > 2 alone would be certain:
    the quadruple's energy is at least x^2 > 16).

Descendant positions come from the pass permutations, which the integer
generator fixes bit-exactly (the oracle's draws and read slots).  The block
scale (Section 5.5) adds a first-order term: the next block is the pool
rescaled by g_{b+1}/g_b and g_b^2 carries x^2/N, so every covariance with a
next-block value is lowered by 2/N (total: 2 - 2 4^R / N).
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
W = 8


def _stream(wn, N, R, seed, blocks):
    import torch
    h = wn.wn_create(N, R, seed)
    n = blocks * (N - 1)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    wn.wn_generate(out, n, h)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64).reshape(blocks, N - 1)


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


@pytest.mark.parametrize("N,R,blocks", [(1024, 1, 12000), (1024, 2, 12000), (256, 1, 48000)])
def test_energy_covariance_with_descendants(wn, N, R, blocks):
    seed = 21 + R
    out = _stream(wn, N, R, seed, blocks)
    d = _draws(N, R, seed, blocks)
    stats = []
    for b in range(0, blocks - 1, 7):  # every 7th block pair: independent, fast
        stats.append(_energy_stats(out[b], out[b + 1], _descendants(N, R, d, b)))
    s = np.array(stats)
    mean, se = s.mean(axis=0), s.std(axis=0) / math.sqrt(len(s))
    expect = np.array([2.0 - 2.0 * 4.0 ** R / N, 2.0 * 4.0 ** -R - 2.0 / N, -2.0 / N])
    print(f"\nN={N} R={R}: cov(x^2, descendants' energy) = {mean[0]:.4f} +- {se[0]:.4f} ({expect[0]:.4f}), "
          f"one descendant {mean[1]:.4f} +- {se[1]:.4f} ({expect[1]:.4f}), "
          f"other {mean[2]:.4f} +- {se[2]:.4f} ({expect[2]:.4f})")
    assert np.all(np.abs(mean - expect) < 5 * se + 0.02), (mean, se, expect)


def test_rare_events_cluster_in_the_next_pool(wn):
    N, R, seed, blocks = 1024, 1, 5, 12000
    out = _stream(wn, N, R, seed, blocks)
    d = _draws(N, R, seed, blocks)
    hits, total = 0, 0
    for b in range(blocks - 1):
        big = np.nonzero(np.abs(out[b]) > 4.0)[0]
        if big.size == 0:
            continue
        desc = _descendants(N, R, d, b)[big]
        keep = np.all(desc < N - 1, axis=1)
        desc = desc[keep]
        total += desc.shape[0]
        hits += int(np.sum(np.any(np.abs(out[b + 1][desc]) > 3.0, axis=1)))
    assert total > 300, total
    frac = hits / total
    # model: x from N(0,1) given |x| > 4, the quadruple's other three inputs
    # N(0,1); each output is s_k (t - a_k) with t half their sum
    from scipy.special import ndtri
    rng = np.random.default_rng(0)
    m = 200_000
    tail = math.erfc(4 / math.sqrt(2)) / 2  # P(x > 4)
    xs = -ndtri(rng.uniform(size=m) * tail) * np.where(rng.uniform(size=m) < 0.5, -1.0, 1.0)
    a = np.column_stack([xs, rng.standard_normal((m, 3))])
    yq = a.sum(axis=1, keepdims=True) / 2 - a
    model = float(np.mean(np.any(np.abs(yq) > 3.0, axis=1)))
    base = 1 - (1 - math.erfc(3 / math.sqrt(2))) ** 4
    se = math.sqrt(model * (1 - model) / total)
    print(f"\nP(descendant |y| > 3 | |x| > 4) = {frac:.3f} over {total} events; model {model:.3f}, "
          f"unconditional {base:.3f}")
    assert abs(frac - model) < 5 * se + 0.02
    assert frac > 3 * base
