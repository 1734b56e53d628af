"""In-tree build of the CUDA library (nvcc, sm_103a only).

Compiles every translation unit under csrc/ in parallel and links them into
``_lib/libwallace_gb300.so``.  Used by ``__graft_entry__.build()`` and, when
the library is missing, by the test fixtures.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libwallace_gb300.so")
# the debug build: device bounds checks (-DWN_DEBUG), relocatable device code
# so that every translation unit counts into one violation record
OUT_DIR_DEBUG = os.path.join(PKG, "_lib_debug")
LIB_DEBUG = os.path.join(OUT_DIR_DEBUG, "libwallace_gb300_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return (_sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
            glob.glob(os.path.join(INCLUDE, "*.h")))


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps() + [__file__])


def build(force: bool = False, verbose: bool = False, extra_flags=None, debug: bool = False) -> str:
    """Compile the library if any source is newer than it; returns its path.
    debug=True builds the bounds-checking library (LIB_DEBUG) instead."""
    lib, out_dir = (LIB_DEBUG, OUT_DIR_DEBUG) if debug else (LIB, OUT_DIR)
    if not force and up_to_date(lib):
        return lib
    nvcc = _nvcc()
    os.makedirs(out_dir, exist_ok=True)
    flags = NVCC_FLAGS + list(extra_flags or []) + (["-DWN_DEBUG", "-rdc=true"] if debug else [])
    objs = []
    cmds = []
    for src in _sources():
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        cmds.append([nvcc] + ARCH + flags + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(cmds))) as ex:
        logs = list(ex.map(run, cmds))
    if verbose:
        for log in logs:
            print(log)
    tmp = lib + f".tmp{os.getpid()}"
    run([nvcc] + ARCH + (["-rdc=true"] if debug else []) + ["-shared", "-o", tmp] + objs)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
