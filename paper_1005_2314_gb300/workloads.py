"""Seeded synthetic request mixes for tests and benchmarks.

Recipes only: stream parameters and request lengths.  Nothing here computes
any part of the generator.
"""
from __future__ import annotations

import numpy as np


def uneven_batch(n_streams: int = 10000, seed: int = 12345, pools=(1024, 4096, 16384), passes=(1, 2, 4),
                 log2_min: float = 10.0, log2_max: float = 24.0):
    """Batched uneven requests: pool size and passes uniform over the given
    choices, request length floor(2^U) with U ~ Uniform[log2_min, log2_max]
    (log-uniform), drawn from numpy's PCG64 seeded by `seed`.  Returns
    (pool_N uint32, passes_R uint32, counts uint64)."""
    rng = np.random.default_rng(seed)
    N = rng.choice(np.asarray(pools, dtype=np.uint32), size=n_streams)
    R = rng.choice(np.asarray(passes, dtype=np.uint32), size=n_streams)
    U = rng.uniform(log2_min, log2_max, size=n_streams)
    counts = np.floor(2.0 ** U).astype(np.uint64)
    return N, R, counts


def packed_offsets(counts) -> np.ndarray:
    """Contiguous layout: stream i's values start where stream i-1's end."""
    counts = np.asarray(counts, dtype=np.uint64)
    off = np.zeros_like(counts)
    if counts.size > 1:
        off[1:] = np.cumsum(counts[:-1])
    return off
