"""The tune cache: the autotuners' choices kept across processes in a JSON
file.  Each test points the library at a file of its own (WN_TUNE_CACHE is
read at every use)."""
import json
import os

import numpy as np
import pytest

import oracle
from _parity import assert_fp32_close, passes_fresh
from paper_1005_2314_gb300.workloads import packed_offsets

pytestmark = pytest.mark.gpu


@pytest.fixture
def cache_file(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("WN_TUNE_CACHE", str(path))
    return path


def test_autotune_choice_reaches_a_new_handle(wn, cache_file):
    import torch
    N, R, n, count = 1024, 2, 200, 3 * 1023 + 5
    seeds = list(range(70, 70 + n))
    h = wn.wn_create_streams([N] * n, [R] * n, seeds)
    qt, th = wn.wn_autotune(h, count)
    entries = json.loads(cache_file.read_text())
    keys = [k for k in entries if k.startswith("gen|")]
    assert len(keys) == 1 and f"|N={N}|R={R}|" in keys[0] and "|streams=200|dtype=0" in keys[0]
    assert entries[keys[0]].split()[0] == str(qt) and entries[keys[0]].split()[2] == str(th)
    # a new handle of the same workload starts with the tuned shape ...
    h2 = wn.wn_create_streams([N] * n, [R] * n, seeds)
    assert wn.wn_get_config(h2) == (qt, th)
    out = torch.empty(n * count, device="cuda")
    wn.wn_generate(out, count, h2)
    torch.cuda.synchronize()
    ref = oracle.Stream(N, R, seeds[-1]).generate(count)
    assert_fp32_close(out.view(n, count)[-1].cpu().numpy(), ref, passes_fresh(count, N, R), "cached shape")
    # ... and another workload does not
    h3 = wn.wn_create_streams([N] * (n + 1), [R] * (n + 1), seeds + [999])
    assert wn.wn_get_config_ex(h3) == (8, 32, wn.WN_CFG_IN_PLACE | wn.WN_CFG_GROUP)


def test_unusable_cache_entries_are_ignored(wn, cache_file):
    N, R, n = 1024, 2, 150
    h = wn.wn_create_streams([N] * n, [R] * n, list(range(n)))
    wn.wn_autotune(h, 5000)
    entries = json.loads(cache_file.read_text())
    key = next(k for k in entries if k.startswith("gen|"))
    for bad in ("7 99 64 0 0", "32 32 32 1 1", "garbage"):  # no such shape / wrong pool / unparsable
        entries[key] = bad
        cache_file.write_text(json.dumps(entries))
        h2 = wn.wn_create_streams([N] * n, [R] * n, list(range(n)))
        assert wn.wn_get_config_ex(h2) == (8, 32, wn.WN_CFG_IN_PLACE | wn.WN_CFG_GROUP), bad
    cache_file.write_text("{ not json")
    h3 = wn.wn_create_streams([N] * n, [R] * n, list(range(n)))
    assert wn.wn_get_config_ex(h3) == (8, 32, wn.WN_CFG_IN_PLACE | wn.WN_CFG_GROUP)


def test_batch_plan_cached(wn, cache_file):
    import torch
    rng = np.random.default_rng(8)
    n = 60
    N = rng.choice(np.array([1024, 4096], dtype=np.uint32), size=n)
    R = rng.choice(np.array([1, 2, 4], dtype=np.uint32), size=n)
    counts = rng.integers(1, 50000, size=n).astype(np.uint64)
    seeds = np.arange(40, 40 + n)
    offsets = packed_offsets(counts)
    out = torch.zeros(int(counts.sum()) + 8, dtype=torch.float32, device="cuda")
    h = wn.wn_create_streams(N, R, seeds)
    wn.wn_autotune_batch(out, counts, offsets, h)
    plan = wn.wn_get_batch_plan(h)
    assert any(k.startswith("batch|") for k in json.loads(cache_file.read_text()))
    h2 = wn.wn_create_streams(N, R, seeds)
    wn.wn_set_batch_plan(h2, 0, 3)
    wn.wn_autotune_batch(out, counts, offsets, h2)  # from the file, no timing
    assert wn.wn_get_batch_plan(h2) == plan
    wn.wn_generate_batch(out, counts, offsets, h2, use_graph=True)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i in (0, 1, n - 1):
        c = int(counts[i])
        ref = oracle.Stream(int(N[i]), int(R[i]), int(seeds[i])).generate(c)
        assert_fp32_close(got[int(offsets[i]): int(offsets[i]) + c], ref, passes_fresh(c, int(N[i]), int(R[i])),
                          f"stream {i}")


def test_cache_off(wn, tmp_path, monkeypatch):
    monkeypatch.setenv("WN_TUNE_CACHE", "off")
    h = wn.wn_create_streams([1024] * 90, [2] * 90, list(range(90)))
    wn.wn_autotune(h, 3000)
    assert not any(tmp_path.iterdir())
