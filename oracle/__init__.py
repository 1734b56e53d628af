"""FP64 CPU oracle for Wallace's maximum-entropy normal generator.

TEST INFRASTRUCTURE ONLY.  This package wraps ``wallace_oracle.c`` (a plain,
slow restatement of Brent, arXiv:1005.2314, Section 5, in FP64) for the tests,
the smoke check and the benchmark's CPU-baseline leg.  The CUDA library never
imports it and shares no code with it.

Parity status of each routine (what pins it; see the tests under ``tests/``):

* ``splitmix64``     - published known-answer values (state 0).
* ``xorshift64_step``- full period 2^64 - 1 of its GF(2) matrix; published
                       known-answer values of Marsaglia's xor64 example.
* ``draws``          - Weyl constant = 2^64 - floor(2^64 / phi); definition.
* ``pass_``          - printed matrix A_1 (Section 5.3) up to row order and
                       signs; hand-worked N=4 example; involution; sum of
                       squares preserved; brute-force mixing reach.
* ``pass_rot``       - the rotation form (Section 5.3, rann4): hand-worked
                       N=4 example (t = 1/2: c = 3/5, s = 4/5); c^2+s^2 = 1;
                       sum of squares preserved; exact inverse; each output
                       a combination of exactly two inputs; mixing reach
                       log2 N passes; t's range and symmetry.
* ``chi2``           - closed-form moments (E S = nu, Var S = 2 nu, third
                       central moment 8 nu for approximation (c)); the cubic
                       for A; exact mean of (a) and (b).
* ``Stream``         - output moments, block sum-of-squares statistics,
                       continuation across calls; ``decimate`` (Section 5.7,
                       every d-th pool) returns exactly blocks d-1, 2d-1, ...
                       of the plain stream and advances the generator 2 R d
                       draws per returned block.
* ``philox4x32_10``  - published known-answer vectors (Random123).
* ``boxmuller``      - special angles and radii; output moments.
* ``gbm``            - closed-form mean and variance of the terminal price.

The mixing quality itself (which permutation schedule is "good enough") has
no closed form: parity unpinned, as the paper says only empirical tests exist
(Section 5.4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wallace_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liborc_wallace.so")
_lock = threading.Lock()
_lib = None

CHI2 = {"off": 0, "a": 1, "b": 2, "c": 3}
RESERVE = {"previous": 0, "current": 1}
UPDATE = {"quad": 0, "rotation": 1}

_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_dbl = ctypes.c_double
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE FP64: no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            sig = {
                "orc_splitmix64": (_u64, [ctypes.POINTER(_u64)]),
                "orc_xorshift64_step": (_u64, [_u64]),
                "orc_draws": (None, [_u64, _u64, _p]),
                "orc_pass_read_slots": (None, [_u32, _u64, _p]),
                "orc_pass": (None, [_u32, _p, _p, _u64, _u64]),
                "orc_pass_inverse": (None, [_u32, _p, _p, _u64, _u64]),
                "orc_chi2_A": (_dbl, [_dbl]),
                "orc_chi2": (_dbl, [ctypes.c_int, _dbl, _dbl]),
                "orc_create": (_p, [_u32, _u32, _u64, _u32, ctypes.c_int, ctypes.c_int]),
                "orc_destroy": (None, [_p]),
                "orc_set_decimate": (ctypes.c_int, [_p, _u32]),
                "orc_create_update": (_p, [_u32, _u32, _u64, _u32, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
                "orc_rot_t": (_dbl, [_u64]),
                "orc_pass_rot": (None, [_u32, _p, _p, _u64, _u64]),
                "orc_pass_rot_inverse": (None, [_u32, _p, _p, _u64, _u64]),
                "orc_generate": (None, [_p, _p, _u64]),
                "orc_skip": (_dbl, [_p, _u64]),
                "orc_get_pool": (None, [_p, _p]),
                "orc_get_r": (_dbl, [_p]),
                "orc_get_g": (_dbl, [_p]),
                "orc_get_k": (_u32, [_p]),
                "orc_get_blocks": (_u64, [_p]),
                "orc_get_gen": (None, [_p, _p]),
                "orc_philox4x32_10": (None, [_p, _p, _p]),
                "orc_boxmuller": (None, [_u64, _u32, _u64, _u64, _p]),
                "orc_gbm": (ctypes.c_int, [_u64, _u32, _u32, _u32, _u32, _u32,
                                           _dbl, _dbl, _dbl, _dbl, _p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def splitmix64(state: int) -> tuple[int, int]:
    """One SplitMix64 step: returns (new state, output)."""
    s = _u64(state)
    z = lib().orc_splitmix64(ctypes.byref(s))
    return s.value, z


def xorshift64_step(x: int) -> int:
    return lib().orc_xorshift64_step(x)


def draws(seed: int, n: int) -> np.ndarray:
    """First n 64-bit draws of the stream generator seeded by `seed`."""
    out = np.zeros(n, dtype=np.uint64)
    lib().orc_draws(seed, n, _ptr(out))
    return out


def alpha_gamma(N: int, w_a: int) -> tuple[int, int]:
    """The odd multiplier and offset one pass takes from its draw w_a."""
    return ((w_a >> 32) & (N - 1)) | 1, w_a & (N - 1)


def pass_read_slots(N: int, w_a: int) -> np.ndarray:
    out = np.zeros(N, dtype=np.uint32)
    lib().orc_pass_read_slots(N, w_a, _ptr(out))
    return out


def rot_t(w_t: int) -> float:
    """The rotation parameter t = tan(theta/2) a rotation pass takes from its draw."""
    return lib().orc_rot_t(w_t)


def pass_rot(N: int, P: np.ndarray, w_a: int, w_t: int) -> np.ndarray:
    P = np.ascontiguousarray(P, dtype=np.float64)
    assert P.shape == (N,)
    out = np.empty(N, dtype=np.float64)
    lib().orc_pass_rot(N, _ptr(P), _ptr(out), w_a, w_t)
    return out


def pass_rot_inverse(N: int, Pn: np.ndarray, w_a: int, w_t: int) -> np.ndarray:
    Pn = np.ascontiguousarray(Pn, dtype=np.float64)
    out = np.empty(N, dtype=np.float64)
    lib().orc_pass_rot_inverse(N, _ptr(Pn), _ptr(out), w_a, w_t)
    return out


def pass_(N: int, P: np.ndarray, w_a: int, w_s: int) -> np.ndarray:
    P = np.ascontiguousarray(P, dtype=np.float64)
    assert P.shape == (N,)
    out = np.empty(N, dtype=np.float64)
    lib().orc_pass(N, _ptr(P), _ptr(out), w_a, w_s)
    return out


def pass_inverse(N: int, Pn: np.ndarray, w_a: int, w_s: int) -> np.ndarray:
    Pn = np.ascontiguousarray(Pn, dtype=np.float64)
    assert Pn.shape == (N,)
    out = np.empty(N, dtype=np.float64)
    lib().orc_pass_inverse(N, _ptr(Pn), _ptr(out), w_a, w_s)
    return out


def chi2_A(nu: float) -> float:
    return lib().orc_chi2_A(nu)


def chi2(kind: str, nu: float, x: float) -> float:
    return lib().orc_chi2(CHI2[kind], nu, x)


class Stream:
    """One Wallace stream: pool N, R passes per block, seeded by `seed`."""

    def __init__(self, N: int, R: int, seed: int, warmup: int = 8,
                 chi2: str = "c", reserve: str = "previous", decimate: int = 1, update: str = "quad"):
        self.N, self.R = N, R
        if update not in UPDATE:
            raise ValueError(f"invalid update {update}")
        h = lib().orc_create_update(N, R, seed, warmup, CHI2[chi2], RESERVE[reserve], UPDATE[update])
        if not h:
            raise ValueError(f"invalid stream parameters N={N} R={R}")
        self._h = h
        if lib().orc_set_decimate(h, decimate) != 0:
            raise ValueError(f"invalid decimation {decimate}")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def generate(self, count: int) -> np.ndarray:
        out = np.empty(count, dtype=np.float64)
        if count:
            lib().orc_generate(self._h, _ptr(out), count)
        return out

    def skip(self, count: int) -> float:
        return lib().orc_skip(self._h, count)

    @property
    def pool(self) -> np.ndarray:
        out = np.empty(self.N, dtype=np.float64)
        lib().orc_get_pool(self._h, _ptr(out))
        return out

    @property
    def r(self) -> float:
        return lib().orc_get_r(self._h)

    @property
    def g(self) -> float:
        return lib().orc_get_g(self._h)

    @property
    def k(self) -> int:
        return lib().orc_get_k(self._h)

    @property
    def blocks(self) -> int:
        return lib().orc_get_blocks(self._h)

    @property
    def gen_state(self) -> tuple[int, int]:
        xw = np.zeros(2, dtype=np.uint64)
        lib().orc_get_gen(self._h, _ptr(xw))
        return int(xw[0]), int(xw[1])


def philox4x32_10(ctr, key) -> list[int]:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return [int(v) for v in o]


def boxmuller(seed: int, stream: int, first: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    if count:
        lib().orc_boxmuller(seed, stream, first, count, _ptr(out))
    return out


def gbm(n_paths: int, paths_per_group: int, steps: int, N: int, R: int,
        S0: float, mu: float, sigma: float, dt: float, warmup: int = 8) -> np.ndarray:
    out = np.empty(n_paths, dtype=np.float64)
    rc = lib().orc_gbm(n_paths, paths_per_group, steps, N, R, warmup,
                       S0, mu, sigma, dt, _ptr(out))
    if rc != 0:
        raise RuntimeError(f"orc_gbm failed: {rc}")
    return out
