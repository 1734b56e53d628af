"""Model of the latency mode's hand-offs (wn_emit.cuh), checked on the CPU.

The table warp, the emitter warp and the compute warps are actors stepped in
random order.  mbarriers have the hardware's semantics: an arrival counts
towards the current phase, the phase completes at its arrival count, and a
wait on parity P is satisfied once the phase of parity P has completed (the
current phase's parity differs from P).  The compute warps share a named
barrier that completes when all of them arrive.  Every run must finish
(no deadlock), and the buffers must be used in order:

  * the emitter reads E[b mod 2] only after every compute warp wrote block b
    there, and a compute warp writes block b into E[s] only after the
    emitter finished block b-2 there;
  * a pass reads what every compute warp wrote in the pass (or block) before,
    and overwrites a buffer only after every compute warp read it;
  * a block's tables are read only after the table warp wrote them, and
    overwritten only after every compute warp finished that block.
"""
import random

import pytest


class Mbar:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, 0, 0

    def arrive(self):
        self.pending += 1
        assert self.pending <= self.count
        if self.pending == self.count:
            self.pending = 0
            self.phase += 1

    def done(self, parity):
        return (self.phase & 1) != parity


class NamedBarrier:
    def __init__(self, n):
        self.n, self.arrived, self.gen = n, 0, 0

    def arrive(self):
        self.arrived += 1
        g = self.gen
        if self.arrived == self.n:
            self.arrived = 0
            self.gen += 1
        return g


def simulate(nb, R, NC, rng):
    tab_full = [Mbar(1), Mbar(1)]
    tab_empty = [Mbar(NC), Mbar(NC)]
    e_full = [Mbar(NC), Mbar(NC)]
    e_empty = [Mbar(1), Mbar(1)]
    bar = NamedBarrier(NC)
    # buffer contents: which (block, pass) each compute warp's part holds,
    # and which readers are done with the current contents
    E = [[(-1, "final")] * NC, [(-1, "final")] * NC]  # block -1: the stored pool, in E[1]
    E[0] = [None] * NC
    W = [[None] * NC, [None] * NC]
    tables = [None, None]
    emitted = []

    def wait(mb, parity):
        while not mb.done(parity):
            yield

    def sync():
        g = bar.arrive()
        while bar.gen == g:
            yield

    def table_warp():
        for b in range(nb):
            s, k = b & 1, b >> 1
            if k >= 1:
                yield from wait(tab_empty[s], (k - 1) & 1)
            assert tables[s] is None or tables[s] == b - 2
            tables[s] = None
            yield
            tables[s] = b
            tab_full[s].arrive()
            yield

    def emitter():
        for b in range(nb):
            s, k = b & 1, b >> 1
            yield from wait(e_full[s], k & 1)
            assert all(part == (b, "final") for part in E[s]), (b, E[s])
            yield
            emitted.append(b)
            e_empty[s].arrive()
            yield

    def compute(c):
        for b in range(nb):
            s, k = b & 1, b >> 1
            yield from wait(tab_full[s], k & 1)
            if k >= 1:
                yield from wait(e_empty[s], (k - 1) & 1)
            yield from sync()
            for p in range(R):
                assert tables[s] == b
                if p == 0:
                    src = E[s ^ 1]
                    assert all(part == (b - 1, "final") for part in src), (b, src)
                else:
                    src = W[(p - 1) & 1]
                    assert all(part == (b, p - 1) for part in src), (b, p, src)
                yield
                if p + 1 == R:
                    if b >= 2:
                        assert (b - 2) in emitted  # the emitter is done with E[s]
                    E[s][c] = (b, "final")
                else:
                    W[p & 1][c] = (b, p)
                yield
                if p + 1 < R:
                    yield from sync()
            tab_empty[s].arrive()
            e_full[s].arrive()
            yield

    actors = [table_warp(), emitter()] + [compute(c) for c in range(NC)]
    live = list(range(len(actors)))
    steps = 0
    while live:
        i = rng.choice(live)
        try:
            next(actors[i])
        except StopIteration:
            live.remove(i)
        steps += 1
        assert steps < 200000, "no progress: deadlock"
    assert emitted == list(range(nb))


@pytest.mark.parametrize("NC", [1, 2, 4])
@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_protocol_under_random_schedules(NC, R):
    rng = random.Random(1000 * NC + R)
    for trial in range(60):
        simulate(rng.randrange(0, 7), R, NC, rng)


def test_protocol_detects_a_missing_wait():
    # the model is not vacuous: without the compute warps' wait for the
    # emitter, some schedule overwrites an emission buffer too early
    rng = random.Random(7)
    failures = 0
    for trial in range(200):
        try:
            _simulate_without_empty_wait(rng.randrange(3, 7), 2, 2, rng)
        except AssertionError:
            failures += 1
    assert failures > 0


def _simulate_without_empty_wait(nb, R, NC, rng):
    e_full = [Mbar(NC), Mbar(NC)]
    bar = NamedBarrier(NC)
    E = [[None] * NC, [(-1, "final")] * NC]
    emitted = []

    def wait(mb, parity):
        while not mb.done(parity):
            yield

    def sync():
        g = bar.arrive()
        while bar.gen == g:
            yield

    def emitter():
        for b in range(nb):
            s, k = b & 1, b >> 1
            yield from wait(e_full[s], k & 1)
            for _ in range(rng.randrange(1, 6)):
                yield  # a slow emitter
            assert all(part == (b, "final") for part in E[s]), (b, E[s])
            emitted.append(b)
            yield

    def compute(c):
        for b in range(nb):
            s = b & 1
            yield from sync()
            E[s][c] = (b, "final")
            yield
            e_full[s].arrive()
            yield

    actors = [emitter()] + [compute(c) for c in range(NC)]
    live = list(range(len(actors)))
    steps = 0
    while live:
        i = rng.choice(live)
        try:
            next(actors[i])
        except StopIteration:
            live.remove(i)
        steps += 1
        # with no wait, the compute warps can run two uses of a buffer ahead:
        # the emitter's parity wait then never completes
        assert steps < 20000, "no progress"
