"""Finite-pool effects of the method (Sections 5.6 and 5.7), measured on the
GPU stream at more than 10^4 n samples, against closed forms.

Every output y of a pass is a +-1/2 combination of four pool values, so a
pool value x and its descendants in the next block are not independent even
though every value is N(0,1) (the E(x^2 y^2) = 2 effect of Section 5.6):

  * were the pool values independent, the squared value and the total
    energy of its 4^R descendants would have covariance exactly 2 (the
    quadruple map is orthogonal), each single descendant 2 c^2 with c = 2^-R
    its coefficient on x, and values that are not descendants 0 (the pool's
    fixed sum of squares lowers all three by O(1/N), below);
  * a rare large value is followed by large values among its descendants
    (Section 5.7): for R = 1, P(some descendant |y| > 3 | |x| > 4) is the
    model's value (four outputs of one quadruple holding x), far above the
    unconditional 1 - (1 - P(|N(0,1)| > 3))^4 (|y| > 2 alone would be certain:
    the quadruple's energy is at least x^2 > 16).

Descendant positions come from the pass permutations, which the integer
generator fixes bit-exactly (the oracle's draws and read slots).  The exact
values follow from the renormalisation (Section 5.5): the pool lies on the
sphere sum P^2 = N, so its squares are exchangeable with E P^4 = 3N/(N+2)
and Cov(P_i^2, P_k^2) = -2/(N+2), and a next-block value y = sum_k c_k P_k
(sum c_k^2 = 1) has Cov(P_i^2, y^2) = (2 N c_i^2 - 2)/(N + 2).  Hence, with
c_i^2 = 4^-R for each of the 4^R descendants: energy (2N - 2 4^R)/(N+2), one
descendant (2N 4^-R - 2)/(N+2), a non-descendant -2/(N+2).  The block scales
g_b, g_{b+1} have mean-one squares and enter only at O(1/N^2).
"""
import math

import numpy as np
import pytest

import oracle
from _defects import _descendants, _draws, energy_covariances, expected_covariances

pytestmark = pytest.mark.gpu


def _stream(wn, N, R, seed, blocks):
    import torch
    h = wn.wn_create(N, R, seed)
    n = blocks * (N - 1)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    wn.wn_generate(out, n, h)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64).reshape(blocks, N - 1)


@pytest.mark.parametrize("N,R,blocks", [(1024, 1, 12000), (1024, 2, 12000), (256, 1, 96000)])
def test_energy_covariance_with_descendants(wn, N, R, blocks):
    seed = 21 + R
    out = _stream(wn, N, R, seed, blocks)
    d = _draws(N, R, seed, blocks)
    mean, se = energy_covariances(out, N, R, d)  # disjoint block pairs (b, b+1)
    expect = expected_covariances(N, R)
    print(f"\nN={N} R={R}: cov(x^2, descendants' energy) = {mean[0]:.4f} +- {se[0]:.4f} ({expect[0]:.4f}), "
          f"one descendant {mean[1]:.4f} +- {se[1]:.4f} ({expect[1]:.4f}), "
          f"other {mean[2]:.4f} +- {se[2]:.4f} ({expect[2]:.4f})")
    # no absolute slack: each statistic within 5 standard errors of its closed form
    assert np.all(np.abs(mean - expect) < 5 * se), (mean, se, expect)
    if N == 256:
        # here the sphere's -2/(N+2) exceeds 5 standard errors, so the
        # independent-pool values (2 4^-R for one descendant, 0 for a
        # non-descendant) are rejected
        assert 5 * se[2] < 2.0 / (N + 2) and 5 * se[1] < 2.0 / (N + 2), se
        assert abs(mean[2]) > 5 * se[2] and abs(mean[1] - 2.0 * 4.0 ** -R) > 5 * se[1], (mean, se)


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
