"""wn_load's validation of a saved state, on the host (no GPU needed: every
check runs before device memory is touched).

The format (include/wallace_gb300.h, wn_save): magic "WNSTATE1", uint32
stream count, uint32 header size 96, the 96-byte per-stream headers, the FP32
pools in stream order, FNV-1a 64 of everything before.  The tests build such
buffers here and corrupt one field at a time.
"""
import struct

import numpy as np
import pytest

HDR = struct.Struct("<QQdddQQfIIIIIdQ")  # the 96-byte per-stream header


def fnv1a64(b: bytes) -> int:
    h = 0xcbf29ce484222325
    for c in b:
        h = ((h ^ c) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def state(Ns=(8, 16), Rs=(2, 1), k=None, x=12345, flags=0, pool=None, magic=b"WNSTATE1", hdr_bytes=96,
          bad_sum=False, extra=b"", variant=3):
    body = magic + struct.pack("<II", len(Ns), hdr_bytes)
    for i, (N, R) in enumerate(zip(Ns, Rs)):
        body += HDR.pack(x, 7, 0.25, 0.66, 1.0, 0, 3, 1.0, (N - 1) if k is None else k, N, R, flags, variant,
                         float(N), 0)
    for N in Ns:
        p = np.linspace(-1, 1, N, dtype=np.float32) if pool is None else np.full(N, pool, np.float32)
        body += p.tobytes()
    s = fnv1a64(body) ^ (1 if bad_sum else 0)
    return body + struct.pack("<Q", s) + extra


@pytest.fixture(scope="module")
def lib():
    import paper_1005_2314_gb300 as wn
    from paper_1005_2314_gb300 import build
    build.build()
    return wn


def test_header_size_is_96():
    assert HDR.size == 96


@pytest.mark.parametrize("buf,why", [
    (b"", "short"),
    (state(magic=b"WNSTATE2"), "magic"),
    (state(hdr_bytes=88), "header"),
    (state(Ns=(12, 16)), "invalid pool size"),
    (state(Ns=(8, 32768)), "invalid pool size"),
    (state(Rs=(0, 1)), "invalid pool size"),
    (state(Rs=(65, 1)), "invalid pool size"),
    (state(k=8), "invalid pool size"),
    (state(x=0), "invalid pool size"),
    (state(flags=1), "invalid pool size"),
    (state(variant=0x10003), "invalid pool size"),
    (state(bad_sum=True), "checksum"),
    (state(extra=b"\0"), "buffer holds"),
    (state()[:-1], "buffer holds"),
    (state(pool=np.nan), "non-finite"),
    (state(pool=np.inf), "non-finite"),
], ids=["empty", "magic", "header-size", "N-not-pow2", "N-too-big", "R-zero", "R-too-big", "k-past-block",
        "x-zero", "flag-set", "variant-bits", "checksum", "trailing-byte", "truncated", "nan-pool", "inf-pool"])
def test_load_rejects_corrupt_state(lib, buf, why):
    with pytest.raises(lib.WnError, match=why):
        lib.wn_load(buf, 0)  # an explicit (legacy default) stream: no torch CUDA call
