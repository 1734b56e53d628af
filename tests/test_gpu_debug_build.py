"""The debug build (-DWN_DEBUG): device bounds checks on every pool access of
the generator kernels and every output store, recording violations instead of
trapping.  Tiny pools (N = 4, 8, 16) exercise the index scheme's edge cases
(a pool of four is one quadruple; alpha and gamma wrap at every step), and a
pool of 1024 reaches the group-mode and emitter kernels; every case is checked
against the oracle and the violation record must stay empty.  The checks run
in a child process that loads the debug library (WN_LIBRARY)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
sys.path.insert(0, ROOT); sys.path.insert(0, ROOT + "/tests")
import numpy as np, torch, oracle
import paper_1005_2314_gb300 as wn
from _parity import assert_fp32_close, passes_fresh
from paper_1005_2314_gb300.workloads import packed_offsets
assert wn.library_path().endswith("_debug.so"), wn.library_path()
wn.wn_debug_report(reset=True)
cases = 0

def check(h, N, R, seeds, count, opts=None, calls=2):
    global cases
    refs = [oracle.Stream(N, R, s, **(opts or {})) for s in seeds]
    done = 0
    for _ in range(calls):
        out = torch.empty(len(seeds) * count, device="cuda")
        wn.wn_generate(out, count, h)
        torch.cuda.synchronize()
        got = out.view(len(seeds), count).cpu().numpy()
        for i, s in enumerate(refs):
            assert_fp32_close(got[i], s.generate(count), passes_fresh(count, N, R, first_block=done // (N - 1)) + R,
                              f"N={N} R={R} {opts}")
        done += count
        cases += 1

for N in (4, 8, 16):
    for R in (1, 2, 3):
        count = 7 * (N - 1) + 2
        # few streams: the latency modes; many: the ordinary kernel
        check(wn.wn_create_streams([N] * 3, [R] * 3, [N + R, 2, 3]), N, R, [N + R, 2, 3], count)
        seeds = list(range(10, 10 + 90))
        hm = wn.wn_create_streams([N] * 90, [R] * 90, seeds)
        out = torch.empty(90 * count, device="cuda")
        wn.wn_generate(out, count, hm); torch.cuda.synchronize()
        got = out.view(90, count).cpu().numpy()
        for i in (0, 89):
            assert_fp32_close(got[i], oracle.Stream(N, R, seeds[i]).generate(count), passes_fresh(count, N, R), "many")
        cases += 1
    # the general kernel (method variants), few and many streams
    for opts in ({"chi2": "a"}, {"reserve": "current"}, {"update": "rotation"}, {"decimate": 3}):
        h = wn.wn_create_ex([N] * 3, [2] * 3, [5, 6, 7], **opts)
        check(h, N, 2, [5, 6, 7], 5 * (N - 1) + 3, opts=opts, calls=1)
# pool 1024: group mode (many streams), emitter (few streams, R = 3)
hg = wn.wn_create_streams([1024] * 100, [2] * 100, list(range(100)))
out = torch.empty(100 * 3001, device="cuda")
wn.wn_generate(out, 3001, hg); torch.cuda.synchronize()
assert_fp32_close(out.view(100, 3001)[7].cpu().numpy(), oracle.Stream(1024, 2, 7).generate(3001),
                  passes_fresh(3001, 1024, 2), "group mode")
check(wn.wn_create_streams([1024] * 2, [3] * 2, [3, 4]), 1024, 3, [3, 4], 2 * 1023 + 5)
# batches: persistent ordinary, latency, group and chain kernels
rng = np.random.default_rng(4)
n = 30
N = rng.choice(np.array([4, 8, 16, 1024], dtype=np.uint32), size=n)
R = rng.choice(np.array([1, 2, 3, 4], dtype=np.uint32), size=n)
counts = rng.integers(0, 9000, size=n).astype(np.uint64)
counts[:3] = [60000, 40000, 1]
seeds = np.arange(200, 200 + n)
offsets = packed_offsets(counts) + 1
for chains, density in ((0, 1), (3, 2)):
    h = wn.wn_create_streams(N, R, seeds)
    wn.wn_set_batch_plan(h, chains, density)
    out = torch.zeros(int(counts.sum()) + 8, device="cuda")
    wn.wn_generate_batch(out, counts, offsets, h)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i in range(n):
        c = int(counts[i])
        if c:
            ref = oracle.Stream(int(N[i]), int(R[i]), int(seeds[i])).generate(c)
            assert_fp32_close(got[int(offsets[i]):int(offsets[i]) + c], ref, passes_fresh(c, int(N[i]), int(R[i])),
                              f"batch stream {i}")
    cases += 1
v, first = wn.wn_debug_report()
assert (v, first) == (0, 0), (v, hex(first))
print("debug build ok:", cases, "cases, no bounds violations")
'''


def test_debug_build_tiny_pools_have_no_bounds_violations(wn):
    from paper_1005_2314_gb300 import build
    lib = build.build(debug=True)
    env = dict(os.environ, WN_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "no bounds violations" in r.stdout


def test_release_build_has_no_bounds_record(wn):
    with pytest.raises(wn.WnError, match="WN_DEBUG"):
        wn.wn_debug_report()
