"""CPU model of the latency mode's barrier handshake (no GPU).

In the latency mode (run_stream_lat in csrc/wn_gen.cuh) the compute warps end
every pass on a barrier among themselves (PASS) and, once per block, take the
block's scale and the next block's tables from the two control warps (READY:
the control warps arrive, the compute warps wait) and hand back the block's
partial sums and reserved slot (DONE: the compute warps arrive, the control
warps wait).  A named barrier completes when its thread count has arrived; an
arrival from a later block that lands in an earlier block's generation would
complete that generation early and let a warp read data that is not there,
and a missing arrival hangs the CTA.  This model runs every role's sequence of
barrier operations, as the kernel issues them, under many random
interleavings and checks that every generation holds arrivals of one block
only, that nothing deadlocks and that no arrival is left over.  It also keeps
the reason the handshake has its order: handing the sums back before waiting
for the scale would need two barrier ids per handover.
"""
import itertools
import random

import pytest


def control(nblocks, parity_ids):
    # warp 0 (scale) and warp 1 (tables) issue the same sequence
    for b in range(nblocks):
        if b > 0:
            yield ("sync", "DONE" + (str((b - 1) & 1) if parity_ids else ""), b - 1)
        yield ("arrive", "READY" + (str(b & 1) if parity_ids else ""), b)
    yield ("sync", "ALL", -1)


def compute(nblocks, R, early, parity_ids):
    for b in range(nblocks):
        sfx = str(b & 1) if parity_ids else ""
        for p in range(R):
            if p + 1 == R:  # the final pass of block b
                if early and b + 1 < nblocks:
                    yield ("arrive", "DONE" + sfx, b)
                yield ("sync", "READY" + sfx, b)
                if not early and b + 1 < nblocks:
                    yield ("arrive", "DONE" + sfx, b)
            yield ("sync", "PASS", (b, p))
    yield ("sync", "ALL", -1)


def run(nblocks, R, warps, rng, early=False, parity_ids=False):
    roles = {("ctl", i): control(nblocks, parity_ids) for i in range(2)}
    for w in range(warps):
        roles[("cmp", w)] = compute(nblocks, R, early, parity_ids)
    full = 2 + warps
    need = {"PASS": warps, "ALL": full}
    for name in ("READY", "DONE"):
        need[name] = need[name + "0"] = need[name + "1"] = full
    cur = {k: next(g, None) for k, g in roles.items()}
    arrived = {b: [] for b in need}
    blocked = {b: [] for b in need}
    while True:
        runnable = [k for k in roles if cur[k] is not None and not any(k in blocked[b] for b in need)]
        if not runnable:
            break
        k = rng.choice(runnable)
        kind, bar, tag = cur[k]
        arrived[bar].append((k, tag))
        if kind == "sync":
            blocked[bar].append(k)
        else:
            cur[k] = next(roles[k], None)
        if len(arrived[bar]) == need[bar]:
            tags = {t for _, t in arrived[bar]}
            assert len(tags) == 1, f"{bar} generation mixes blocks {sorted(map(str, tags))}"
            for w in blocked[bar]:
                cur[w] = next(roles[w], None)
            arrived[bar], blocked[bar] = [], []
    left = {k: v for k, v in cur.items() if v is not None}
    assert not left, f"deadlock: {left}"
    for bar in need:
        assert not arrived[bar], f"dangling arrivals at {bar}: {arrived[bar]}"


@pytest.mark.parametrize("warps", [1, 4])
def test_handshake_as_built(warps):
    rng = random.Random(7)
    for nblocks, R in itertools.product(range(0, 7), range(1, 5)):
        for _ in range(100):
            run(nblocks, R, warps, rng)


def test_early_handover_needs_two_ids_per_barrier():
    rng = random.Random(11)
    for nblocks, R in itertools.product(range(0, 7), range(1, 4)):
        for _ in range(60):
            run(nblocks, R, 3, rng, early=True, parity_ids=True)
    failures = 0
    for _ in range(300):
        try:
            run(5, 1, 3, rng, early=True, parity_ids=False)
        except AssertionError:
            failures += 1
    assert failures > 0
