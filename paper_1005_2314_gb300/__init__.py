"""GB300 (sm_103a) Wallace maximum-entropy normal generator.

A thin ctypes binding over the C ABI in ``include/wallace_gb300.h``: the
functions here have the same names and only marshal arguments (torch tensors
to device pointers, torch streams to cudaStream_t).  All generation runs in
the CUDA kernels of ``libwallace_gb300.so``; there is no CPU path.  PyTorch
supplies device memory and streams.

The method (Brent, arXiv:1005.2314, Section 5): a pool of N normal values is
renewed pass by pass with random-signed 4x4 orthogonal updates on permuted
quadruples; each block of R passes returns N-1 values scaled so that the
pool's sum of squares is a chi-squared_N sample.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "WN_F32", "WN_BF16", "WN_F16", "WnError",
    "wn_create", "wn_create_streams", "wn_create_ex", "WN_CHI2", "WN_RESERVE", "WN_UPDATE", "wn_destroy", "wn_generate", "wn_generate_ex",
    "wn_generate_host",
    "wn_set_cuda_stream", "wn_set_config", "wn_get_config", "wn_set_config_ex", "wn_get_config_ex",
    "WN_CFG_IN_PLACE", "WN_CFG_GROUP", "WN_CFG_CHAIN", "wn_autotune", "wn_gbm", "wn_generate_batch",
    "wn_autotune_batch", "wn_generate_batch_noalloc", "wn_get_batch_plan", "wn_set_batch_plan", "wn_set_batch_chain_kernel", "wn_num_streams", "wn_get_pool", "wn_get_state",
    "wn_rng_draws", "wn_debug_report", "wn_boxmuller", "wn_save", "wn_load", "wn_last_error", "library_path", "load",
]

WN_F32, WN_BF16, WN_F16 = 0, 1, 2
WN_CFG_IN_PLACE = 1
WN_CFG_GROUP = 2
WN_CFG_CHAIN = 4
WN_OK, WN_EINVAL, WN_ENOMEM, WN_ECUDA, WN_ETIMEOUT = 0, 1, 2, 3, 4
_STATUS = {1: "WN_EINVAL", 2: "WN_ENOMEM", 3: "WN_ECUDA", 4: "WN_ETIMEOUT"}

_u32, _u64, _p, _i = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int


class WnError(RuntimeError):
    """A wn_* call returned an error status."""


def library_path() -> str:
    """The library this binding loads: $WN_LIBRARY if set (e.g. the debug
    build, build.LIB_DEBUG), else the in-tree build."""
    return os.environ.get("WN_LIBRARY") or _build.LIB


def _load() -> ctypes.CDLL:
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(
            f"CUDA library {path} is missing: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    L = ctypes.CDLL(path)
    sig = {
        "wn_create": (_p, [_u32, _u32, _u64]),
        "wn_create_streams": (_p, [_u32, _p, _p, _p, _u32, _p]),
        "wn_create_ex": (_p, [_u32, _p, _p, _p, _u32, _p, _p]),
        "wn_destroy": (None, [_p]),
        "wn_generate": (_i, [_p, _u64, _p]),
        "wn_generate_ex": (_i, [_p, _u64, _p, _i, _p]),
        "wn_generate_host": (_i, [_p, _u64, _p, _i, _p]),
        "wn_set_cuda_stream": (_i, [_p, _p]),
        "wn_set_config": (_i, [_p, _u32, _u32]),
        "wn_get_config": (_i, [_p, _p, _p]),
        "wn_set_config_ex": (_i, [_p, _u32, _u32, _u32]),
        "wn_get_config_ex": (_i, [_p, _p, _p, _p]),
        "wn_autotune": (_i, [_p, _u64, _i, _p, _p, _p]),
        "wn_generate_batch": (_i, [_p, _p, _p, _p, _i, _i, _p]),
        "wn_autotune_batch": (_i, [_p, _p, _p, _p, _i, _p]),
        "wn_generate_batch_noalloc": (_i, [_p, _p, _p, _p, _i, _p]),
        "wn_get_batch_plan": (_i, [_p, _p, _p]),
        "wn_set_batch_plan": (_i, [_p, ctypes.c_int32, _u32]),
        "wn_set_batch_chain_kernel": (_i, [_p, ctypes.c_int32]),
        "wn_gbm": (_i, [_p, _p, _u32, _u32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                        ctypes.c_double, _p]),
        "wn_num_streams": (_u32, [_p]),
        "wn_get_pool": (_i, [_p, _u32, _p]),
        "wn_get_state": (_i, [_p, _u32, _p, _p, _p, _p, _p]),
        "wn_rng_draws": (_i, [_u64, _u64, _p]),
        "wn_debug_report": (_i, [_p, _p, _i]),
        "wn_boxmuller": (_i, [_p, _u64, _u32, _u64, _i, _p]),
        "wn_save": (_i, [_p, _p, _u64, _p]),
        "wn_load": (_p, [_p, _u64, _p]),
        "wn_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


_lib_handle = None


def _L() -> ctypes.CDLL:
    """The loaded library; raises ImportError when it has not been built."""
    global _lib_handle
    if _lib_handle is None:
        _lib_handle = _load()
    return _lib_handle


def load() -> str:
    """Loads the CUDA library now (raises if it is missing); returns its path."""
    _L()
    return library_path()

_DTYPE_BYTES = {WN_F32: 4, WN_BF16: 2, WN_F16: 2}


def _torch_dtype(dt):
    import torch
    m = {WN_F32: torch.float32, WN_BF16: torch.bfloat16, WN_F16: torch.float16}
    if dt not in m:
        raise ValueError(f"unknown wn_dtype {dt}")
    return m[dt]


def _stream_ptr(cuda_stream):
    """cudaStream_t as an int: None -> torch's current stream."""
    if cuda_stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(cuda_stream, int):
        return cuda_stream
    return cuda_stream.cuda_stream


def _out_ptr(out, need_elems: int, dtype: int) -> int:
    """Device pointer of `out` (a CUDA tensor or an int address)."""
    if isinstance(out, int):
        return out
    import torch
    if not isinstance(out, torch.Tensor) or not out.is_cuda:
        raise TypeError("out must be a CUDA tensor or a device address")
    if not out.is_contiguous():
        raise ValueError("out must be contiguous")
    if out.dtype != _torch_dtype(dtype):
        raise TypeError(f"out has dtype {out.dtype}, expected {_torch_dtype(dtype)}")
    if out.numel() < need_elems:
        raise ValueError(f"out holds {out.numel()} elements, the call writes {need_elems}")
    return out.data_ptr()


def _check(st: int, what: str):
    if st != WN_OK:
        msg = _L().wn_last_error().decode(errors="replace")
        raise WnError(f"{what}: {_STATUS.get(st, st)}: {msg}")


def wn_last_error() -> str:
    return _L().wn_last_error().decode(errors="replace")


class Handle:
    """An opaque wn_stream*; freed by wn_destroy (or when collected)."""

    def __init__(self, ptr: int, n: int):
        self.ptr = ptr
        self.n = n

    def __del__(self):
        if getattr(self, "ptr", None):
            _L().wn_destroy(self.ptr)
            self.ptr = None


def wn_create(pool_N: int, passes_R: int, seed: int) -> Handle:
    h = _L().wn_create(pool_N, passes_R, seed)
    if not h:
        raise WnError(f"wn_create: {wn_last_error()}")
    return Handle(h, 1)


def wn_create_streams(pool_N, passes_R, seeds, warmup_blocks: int = 8, cuda_stream=None) -> Handle:
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    n = seeds.size
    N = np.ascontiguousarray(np.broadcast_to(np.asarray(pool_N, dtype=np.uint32), (n,)))
    R = np.ascontiguousarray(np.broadcast_to(np.asarray(passes_R, dtype=np.uint32), (n,)))
    h = _L().wn_create_streams(n, N.ctypes.data, R.ctypes.data, seeds.ctypes.data,
                               warmup_blocks, _stream_ptr(cuda_stream))
    if not h:
        raise WnError(f"wn_create_streams: {wn_last_error()}")
    return Handle(h, n)


class _Options(ctypes.Structure):
    _fields_ = [("chi2", _u32), ("reserve", _u32), ("decimate", _u32), ("update", _u32)]


WN_CHI2 = {"off": 0, "a": 1, "b": 2, "c": 3}
WN_RESERVE = {"previous": 0, "current": 1}
WN_UPDATE = {"quad": 0, "rotation": 1}


def wn_create_ex(pool_N, passes_R, seeds, warmup_blocks: int = 8, chi2: str = "c", reserve: str = "previous",
                 decimate: int = 1, update: str = "quad", cuda_stream=None) -> Handle:
    """wn_create_streams with the method variants of wn_options (names as in WN_CHI2 / WN_RESERVE / WN_UPDATE)."""
    if chi2 not in WN_CHI2 or reserve not in WN_RESERVE or update not in WN_UPDATE:
        raise ValueError(f"chi2 must be one of {list(WN_CHI2)}, reserve one of {list(WN_RESERVE)}, "
                         f"update one of {list(WN_UPDATE)}")
    seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.uint64))
    n = seeds.size
    N = np.ascontiguousarray(np.broadcast_to(np.asarray(pool_N, dtype=np.uint32), (n,)))
    R = np.ascontiguousarray(np.broadcast_to(np.asarray(passes_R, dtype=np.uint32), (n,)))
    opt = _Options(WN_CHI2[chi2], WN_RESERVE[reserve], int(decimate), WN_UPDATE[update])
    h = _L().wn_create_ex(n, N.ctypes.data, R.ctypes.data, seeds.ctypes.data, warmup_blocks, ctypes.byref(opt),
                          _stream_ptr(cuda_stream))
    if not h:
        raise WnError(f"wn_create_ex: {wn_last_error()}")
    return Handle(h, n)


def wn_destroy(h: Handle) -> None:
    if h.ptr:
        _L().wn_destroy(h.ptr)
        h.ptr = None


def wn_generate(out, count: int, h: Handle) -> None:
    _check(_L().wn_generate(_out_ptr(out, count * h.n, WN_F32), count, h.ptr), "wn_generate")


def wn_generate_ex(out, count: int, h: Handle, dtype: int = WN_F32, cuda_stream=None) -> None:
    _check(_L().wn_generate_ex(_out_ptr(out, count * h.n, dtype), count, h.ptr, dtype,
                               _stream_ptr(cuda_stream)), "wn_generate_ex")


def wn_generate_host(host_out, count: int, h: Handle, dtype: int = WN_F32, cuda_stream=None) -> None:
    """host_out: a CPU tensor (pinned for full speed) or a host address."""
    if isinstance(host_out, int):
        ptr = host_out
    else:
        import torch
        if not isinstance(host_out, torch.Tensor) or host_out.is_cuda or not host_out.is_contiguous():
            raise TypeError("host_out must be a contiguous CPU tensor or a host address")
        if host_out.dtype != _torch_dtype(dtype):
            raise TypeError(f"host_out has dtype {host_out.dtype}, expected {_torch_dtype(dtype)}")
        if host_out.numel() < count * h.n:
            raise ValueError(f"host_out holds {host_out.numel()} elements, the call writes {count * h.n}")
        ptr = host_out.data_ptr()
    _check(_L().wn_generate_host(ptr, count, h.ptr, dtype, _stream_ptr(cuda_stream)), "wn_generate_host")


def wn_set_cuda_stream(h: Handle, cuda_stream) -> None:
    _check(_L().wn_set_cuda_stream(h.ptr, _stream_ptr(cuda_stream)), "wn_set_cuda_stream")


def wn_set_config(h: Handle, quads_per_thread: int, threads: int) -> None:
    _check(_L().wn_set_config(h.ptr, quads_per_thread, threads), "wn_set_config")


def wn_get_config(h: Handle) -> tuple[int, int]:
    q = ctypes.c_uint32()
    t = ctypes.c_uint32()
    _check(_L().wn_get_config(h.ptr, ctypes.addressof(q), ctypes.addressof(t)), "wn_get_config")
    return q.value, t.value


def wn_set_config_ex(h: Handle, quads_per_thread: int, threads: int, flags: int = 0) -> None:
    """wn_set_config with layout flags (WN_CFG_IN_PLACE: one pool buffer per CTA;
    WN_CFG_GROUP: the group-mode kernel, threads / 32 warps per stream;
    WN_CFG_CHAIN: the chain-mode kernel, threads / 32 compute warps per stream)."""
    _check(_L().wn_set_config_ex(h.ptr, quads_per_thread, threads, flags), "wn_set_config_ex")


def wn_get_config_ex(h: Handle) -> tuple[int, int, int]:
    """(quadruples per thread, compute threads, layout flags) of the next generate call."""
    q, t, f = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(_L().wn_get_config_ex(h.ptr, ctypes.addressof(q), ctypes.addressof(t), ctypes.addressof(f)),
           "wn_get_config_ex")
    return q.value, t.value, f.value


def wn_autotune(h: Handle, count: int, dtype: int = WN_F32, cuda_stream=None) -> tuple[int, int]:
    """Times the compiled launch shapes on a copy of the state; keeps the best."""
    q = ctypes.c_uint32()
    t = ctypes.c_uint32()
    _check(_L().wn_autotune(h.ptr, count, dtype, _stream_ptr(cuda_stream), ctypes.addressof(q),
                            ctypes.addressof(t)), "wn_autotune")
    return q.value, t.value


def _batch_arrays(h: Handle, counts, offsets):
    counts = np.ascontiguousarray(np.asarray(counts, dtype=np.uint64))
    offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    if counts.shape != (h.n,) or offsets.shape != (h.n,):
        raise ValueError(f"counts and offsets need {h.n} entries")
    need = int(np.max(offsets + counts)) if h.n else 0
    return counts, offsets, need


def wn_generate_batch(out, counts, offsets, h: Handle, dtype: int = WN_F32, use_graph: bool = False,
                      cuda_stream=None) -> None:
    """Stream i's next counts[i] values go to out[offsets[i]:offsets[i]+counts[i]]."""
    counts, offsets, need = _batch_arrays(h, counts, offsets)
    _check(_L().wn_generate_batch(_out_ptr(out, need, dtype), counts.ctypes.data, offsets.ctypes.data, h.ptr,
                                  dtype, int(bool(use_graph)), _stream_ptr(cuda_stream)), "wn_generate_batch")


def wn_generate_batch_noalloc(out, counts, offsets, h: Handle, dtype: int = WN_F32, cuda_stream=None) -> None:
    """As wn_generate_batch without a graph, for callers that must not
    allocate device memory: the library's fixed scratch array holds the
    request descriptors (at most WN_NOALLOC_MAX_STREAMS = 16384 streams)."""
    counts, offsets, need = _batch_arrays(h, counts, offsets)
    _check(_L().wn_generate_batch_noalloc(_out_ptr(out, need, dtype), counts.ctypes.data, offsets.ctypes.data,
                                          h.ptr, dtype, _stream_ptr(cuda_stream)), "wn_generate_batch_noalloc")


WN_NOALLOC_MAX_STREAMS = 16384


def wn_autotune_batch(out, counts, offsets, h: Handle, dtype: int = WN_F32, cuda_stream=None) -> None:
    counts, offsets, need = _batch_arrays(h, counts, offsets)
    _check(_L().wn_autotune_batch(_out_ptr(out, need, dtype), counts.ctypes.data, offsets.ctypes.data, h.ptr,
                                  dtype, _stream_ptr(cuda_stream)), "wn_autotune_batch")


def wn_set_batch_chain_kernel(h: Handle, chain_mode: bool) -> None:
    """Run the batch's chain groups in the chain mode (True) or the latency modes (False, the default)."""
    _check(_L().wn_set_batch_chain_kernel(h.ptr, 1 if chain_mode else 0), "wn_set_batch_chain_kernel")


def wn_get_batch_plan(h: Handle) -> tuple[int, int]:
    """(chains run in the latency mode, chain CTAs per SM) of the handle's batches."""
    k, d = ctypes.c_int32(), ctypes.c_uint32()
    _check(_L().wn_get_batch_plan(h.ptr, ctypes.addressof(k), ctypes.addressof(d)), "wn_get_batch_plan")
    return k.value, d.value


def wn_set_batch_plan(h: Handle, chains: int, density: int = 1) -> None:
    _check(_L().wn_set_batch_plan(h.ptr, chains, density), "wn_set_batch_plan")


def wn_gbm(st_out, h: Handle, paths_per_stream: int, steps: int, S0: float, mu: float, sigma: float,
           dt: float, cuda_stream=None) -> None:
    """st_out: float32 CUDA tensor of h.n * paths_per_stream terminal prices."""
    ptr = _out_ptr(st_out, h.n * paths_per_stream, WN_F32)
    _check(_L().wn_gbm(h.ptr, ptr, paths_per_stream, steps, S0, mu, sigma, dt, _stream_ptr(cuda_stream)),
           "wn_gbm")


def wn_num_streams(h: Handle) -> int:
    return _L().wn_num_streams(h.ptr)


def wn_get_pool(h: Handle, i: int, N: int) -> np.ndarray:
    out = np.empty(N, dtype=np.float32)
    _check(_L().wn_get_pool(h.ptr, i, out.ctypes.data), "wn_get_pool")
    return out


def wn_get_state(h: Handle, i: int) -> dict:
    xw = np.zeros(2, dtype=np.uint64)
    r = ctypes.c_double()
    sc = ctypes.c_float()
    k = ctypes.c_uint32()
    b = ctypes.c_uint64()
    _check(_L().wn_get_state(h.ptr, i, xw.ctypes.data, ctypes.addressof(r), ctypes.addressof(sc),
                             ctypes.addressof(k), ctypes.addressof(b)), "wn_get_state")
    return {"x": int(xw[0]), "w": int(xw[1]), "r": r.value, "scale": sc.value,
            "k": k.value, "blocks": b.value}


def wn_rng_draws(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    _check(_L().wn_rng_draws(seed, n, out.ctypes.data), "wn_rng_draws")
    return out


def wn_debug_report(reset: bool = False) -> tuple[int, int]:
    """(violations, first) of the debug build's bounds record (raises WnError
    on a library built without WN_DEBUG)."""
    v, f = ctypes.c_uint64(), ctypes.c_uint64()
    _check(_L().wn_debug_report(ctypes.addressof(v), ctypes.addressof(f), int(bool(reset))), "wn_debug_report")
    return v.value, f.value


def wn_save(h: Handle) -> np.ndarray:
    """The handle's complete state as a uint8 array (synchronises its CUDA stream)."""
    need = ctypes.c_uint64(0)
    _check(_L().wn_save(h.ptr, None, 0, ctypes.byref(need)), "wn_save")
    buf = np.empty(need.value, dtype=np.uint8)
    _check(_L().wn_save(h.ptr, buf.ctypes.data, buf.size, None), "wn_save")
    return buf


def wn_load(buf, cuda_stream=None) -> Handle:
    """A new handle continuing the streams saved in `buf` (bytes or a uint8 array)."""
    arr = np.ascontiguousarray(np.frombuffer(bytes(buf), dtype=np.uint8) if isinstance(buf, (bytes, bytearray))
                               else np.asarray(buf, dtype=np.uint8))
    p = _L().wn_load(arr.ctypes.data if arr.size else None, arr.size, _stream_ptr(cuda_stream))
    if not p:
        raise WnError(f"wn_load: {wn_last_error()}")
    n = _L().wn_num_streams(p)
    return Handle(p, n)


def wn_boxmuller(out, count: int, n_streams: int, seed: int, dtype: int = WN_F32, cuda_stream=None) -> None:
    _check(_L().wn_boxmuller(_out_ptr(out, count * n_streams, dtype), count, n_streams, seed, dtype,
                             _stream_ptr(cuda_stream)), "wn_boxmuller")
