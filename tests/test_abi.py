"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/*.h declares.  No compute call is made here."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        # strip comments
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(wn_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1005_2314_gb300 import build
    try:
        return build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("wn_create", "wn_generate", "wn_destroy", "wn_generate_ex",
                     "wn_create_streams", "wn_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _declared() - exported
    assert not missing, missing


def test_library_loads_and_resolves_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert getattr(lib, name) is not None
    lib.wn_last_error.restype = ctypes.c_char_p
    assert lib.wn_last_error() == b""


def test_argument_errors_need_no_gpu(libpath):
    # invalid parameters are rejected on the host before any CUDA call
    lib = ctypes.CDLL(libpath)
    lib.wn_create.restype = ctypes.c_void_p
    lib.wn_create.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64]
    lib.wn_last_error.restype = ctypes.c_char_p
    for N, R in [(0, 1), (3, 2), (12, 2), (32768, 2), (1024, 0), (1024, 65)]:
        assert lib.wn_create(N, R, 1) is None
        assert b"pool_N" in lib.wn_last_error()
    lib.wn_generate.restype = ctypes.c_int
    lib.wn_generate.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
    assert lib.wn_generate(None, 10, None) == 1  # WN_EINVAL
    lib.wn_num_streams.restype = ctypes.c_uint32
    lib.wn_num_streams.argtypes = [ctypes.c_void_p]
    assert lib.wn_num_streams(None) == 0
    lib.wn_destroy.argtypes = [ctypes.c_void_p]
    lib.wn_destroy(None)


def test_python_binding_names_match_abi():
    import paper_1005_2314_gb300 as pkg
    for name in _declared():
        assert hasattr(pkg, name), name
