"""bench.py's arithmetic and argument checks (CPU only).

The roofline figures the benchmark reports come from these helpers, so their
byte and wavefront counts are pinned here against hand-computed values.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_of_the_headline_launch():
    # 4096 streams x (2^20 FP32 values + one read and one write of a 4096-value
    # pool + the 96-byte header twice)
    assert bench._algorithmic_bytes(4096, 1 << 20) == 4096 * (4 * 2**20 + 2 * 4 * 4096 + 2 * 96)
    assert bench._algorithmic_bytes(4096, 1 << 20) == 17_314_873_344
    # 16-bit output, pools of 16384
    assert bench._algorithmic_bytes(2, 10, pool=16384, esize=2) == 2 * (20 + 2 * 4 * 16384 + 192)


def test_l1_roofline_counts():
    r = bench._l1_roofline(1.0e12, 2, 4, 2000.0, 100)
    # per 32 values: 2 passes x (1 gather + 1 store wavefront) + 1 output wavefront
    assert r["wavefronts_per_value"] == pytest.approx(5 / 32)
    assert r["peak"] == pytest.approx(100 * 2000e6 / 1e9)
    assert r["frac"] == pytest.approx(1.0e12 * 5 / 32 / (100 * 2000e6), rel=1e-3)
    r3 = bench._l1_roofline(1.0e12, 3, 2, 2000.0, 100)
    assert r3["wavefronts_per_value"] == pytest.approx(6.5 / 32)
    assert bench._l1_roofline(1.0e12, 2, 4, None, 100) is None


def test_traffic_summary_is_used_only_for_the_current_kernel(monkeypatch):
    t = bench._traffic_per_launch(4096, 1 << 20)
    if t is not None:  # the committed capture matches the kernel sources
        assert 0.9 * bench._algorithmic_bytes(4096, 1 << 20) < t < 1.1 * bench._algorithmic_bytes(4096, 1 << 20)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    assert bench._traffic_per_launch(4096, 1 << 20) is None
    monkeypatch.undo()
    assert bench._traffic_per_launch(4096, 12345) is None  # captured at another per-stream count


def test_other_pools_need_kernel_only():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--pool", "16384"],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 2 and "--kernel-only" in r.stderr
