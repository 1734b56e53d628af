"""Shared test configuration.

Tests marked ``gpu`` need a CUDA device and the compiled CUDA library; all
others run on the CPU (oracle pins, host logic, library exports).
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# the library's tune cache goes to a file of this test session, never to the
# user's cache directory (tests that need another file set their own)
if "WN_TUNE_CACHE" not in os.environ:
    import tempfile
    os.environ["WN_TUNE_CACHE"] = os.path.join(tempfile.mkdtemp(prefix="wn_tests_"), "tune.json")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: long-running statistical test")


@pytest.fixture(scope="session")
def wn():
    """The CUDA library binding; builds it in-tree if needed."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1005_2314_gb300 import build
    build.build()
    import paper_1005_2314_gb300 as pkg
    return pkg
