"""Tolerances for comparing the FP32 CUDA path with the FP64 oracle.

Error model (derived from the arithmetic; the paper fixes no precision):
a pass computes t = ((a0 + a1) + (a2 + a3)) / 2 and y_k = t - a_k in FP32.
With round-to-nearest (unit roundoff u = 2^-24) and pool values of unit
variance, the four roundings add an error of variance at most
(u^2/3)(|a0+a1|^2/4 + |a2+a3|^2/4 + |2t|^2/4 + |y_k|^2), whose expectation is
u^2.  Every later pass is orthogonal, so earlier errors keep their size and
new ones add in quadrature: after P passes the RMS error of a pool value is
about u sqrt(P).  The output scale is formed in FP64 from an FP64 sum of the
squares and rounded once to FP32, adding O(u).  Hence

    RMS over outputs of |gpu - oracle| / (u sqrt(P))   <=  C_RMS = 2
    every output:  |gpu - oracle| <= C_MAX u sqrt(P) (1 + |oracle|),  C_MAX = 10

(C_MAX covers the largest of up to 2^32 Gaussian-like errors, about 6.7
standard deviations, with margin).  P is the number of passes the value's
block has seen since initialisation: R (W + b + 1) for block b after W
warm-up blocks.  The RMS bound is a statement about many values (their mean
squared error); it is checked from RMS_MIN_VALUES values up, since for a
handful of values it is a bound of 2 standard deviations on each, which
chance alone breaks in a few percent of cases.  The per-value bound holds for
any count.
"""
import math

import numpy as np

U = 2.0 ** -24
C_RMS = 2.0
C_MAX = 10.0
RMS_MIN_VALUES = 32

# round-to-nearest unit roundoffs of the 16-bit output types
U_BF16 = 2.0 ** -8
U_F16 = 2.0 ** -11
F16_MIN_NORMAL = 2.0 ** -14


def passes_fresh(count, N, R, W=8, first_block=0):
    """Passes seen by each of the first `count` values of a stream that has
    returned `first_block` whole blocks after W warm-up blocks."""
    b = np.arange(count, dtype=np.int64) // (N - 1) + first_block
    return R * (W + b + 1)


def assert_fp32_close(gpu, ref, P, what=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    P = np.broadcast_to(np.asarray(P, dtype=np.float64), ref.shape)
    assert gpu.shape == ref.shape
    assert np.all(np.isfinite(gpu)), f"{what}: non-finite output"
    err = np.abs(gpu - ref)
    scale = U * np.sqrt(P)
    tol = C_MAX * scale * (1.0 + np.abs(ref))
    bad = np.flatnonzero(err > tol)
    assert bad.size == 0, (
        f"{what}: {bad.size} values beyond tolerance; first at {bad[0]}: "
        f"gpu={gpu[bad[0]]!r} oracle={ref[bad[0]]!r} err={err[bad[0]]:.3e} tol={tol[bad[0]]:.3e}")
    rms = math.sqrt(float(np.mean((err / scale) ** 2))) if err.size else 0.0
    assert err.size < RMS_MIN_VALUES or rms <= C_RMS, f"{what}: normalised RMS error {rms:.3f} > {C_RMS}"
    return rms, float(np.max(err / scale)) if err.size else 0.0
