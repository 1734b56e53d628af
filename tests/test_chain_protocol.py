"""Model of the chain mode's hand-offs (wn_chain.cuh), checked on the CPU.

The compute warps, the scale warp, the store warps (store warp s takes the
blocks b = s mod NS) and the draw warp are actors stepped in random order.  Named barriers have the hardware's semantics: every arrival
(bar.arrive or bar.sync) counts towards the current phase, the phase
completes at the barrier's count, and a bar.sync returns once the phase it
arrived in has completed.  Bulk copies complete their reads at random later
steps.  Every run must finish (no deadlock), no barrier phase may mix
arrivals of two different hand-overs, and every buffer must be used in
order:

  * a pass reads the pool every compute warp wrote in the pass (or block)
    before, and a buffer is overwritten only after every reader of its
    contents has read them (the compute warps' next pass, and for an
    emission buffer also the store warp);
  * the scale warp reads block b's sums of squares after every compute warp
    wrote them, and they are overwritten only after it read them; likewise
    the scale it hands to the store warp (or, without staging, to the compute
    warps' next emission);
  * a staging buffer is refilled only after the bulk copy that reads it has
    done so.
"""
import random

import pytest


class Barrier:
    """A named barrier: count arrivals complete a phase."""

    def __init__(self, count):
        self.count, self.arrived, self.gen, self.label = count, 0, 0, None

    def arrive(self, label):
        if self.arrived == 0:
            self.label = label
        assert self.label == label, f"one phase mixes {self.label} and {label}"
        self.arrived += 1
        g = self.gen
        if self.arrived == self.count:
            self.arrived = 0
            self.gen += 1
        return g


class Buffer:
    """A pool-sized shared buffer written in G parts (one per compute warp)."""

    def __init__(self, G, content, readers):
        self.parts = [content] * G
        self.pending = {content: set(readers)}  # readers each content still owes

    def write(self, w, content, readers):
        old = self.parts[w]
        assert not self.pending.get(old), f"part {w} of {old} overwritten before {self.pending[old]} read it"
        self.parts[w] = content
        self.pending.setdefault(content, set(readers))

    def read(self, reader, content):
        assert all(p == content for p in self.parts), f"{reader} expected {content}, found {self.parts}"
        self.pending[content].discard(reader)


def simulate(G, R, nb, stage, rng, NS=2, KE=2):
    H = G + 3  # PART, SCALE: the compute warps, the scale warp, one store warp, the draw warp
    KS = KE if stage else 2  # blocks from PART(b) to the compute warps' wait at SCALE(b)
    RK = KS + 2  # slots of the ring of pass words
    MP = max(NS, KS)  # PART and SCALE identifiers
    MSC = 14 - 2 * MP  # SC identifiers
    bars = {"pass": Barrier(G)}
    bars.update({f"P{k}": Barrier(H) for k in range(MP)})
    bars.update({f"S{k}": Barrier(H) for k in range(MP)})
    bars.update({f"SC{k}": Barrier(2) for k in range(MSC)})
    comp = [f"c{w}" for w in range(G)]
    # pool buffers: with staging W0, W1 (work) and E0, E1 (emission, the
    # stored pool in E1); without, two buffers the passes alternate between
    bufs = {"W0": Buffer(G, None, []), "W1": Buffer(G, None, [])}
    bufs.update({f"E{k}": Buffer(G, None, []) for k in range(KS)})
    pool_buf = f"E{KS - 1}" if stage else "W0"
    bufs[pool_buf] = Buffer(G, ("pool",), comp)
    parts = [Buffer(G, None, []) for _ in range(KS)]  # by b mod KS
    K = 2 * NS  # scale slots
    scs = {k: None for k in range(K)}
    scs[0] = ("sc", 0)
    scs_pending = {("sc", 0): {"s0"} if stage else set(comp)}
    bulks = {k: [] for k in range(NS)}  # per store warp: [block, read_done]
    # the ring of pass words: slot -> (block, compute warps yet to read it)
    ring = {}

    def write_words(blk):
        slot = blk % RK
        if slot in ring:
            old, pending = ring[slot]
            assert not pending, f"pass words of block {old} overwritten before {pending} read them"
        ring[slot] = (blk, set(comp))

    def read_words(me, blk):
        got, _ = ring.get(blk % RK, (None, set()))
        assert got == blk, f"{me} expected the pass words of block {blk}, found block {got}"

    def done_words(me, blk):  # the warp's last read of block blk's words is behind it
        got, pending = ring[blk % RK]
        assert got == blk
        pending.discard(me)

    for blk in range(min(nb, KS + 1)):  # before the CTA's first barrier
        write_words(blk)

    def sync(name, label):
        g = bars[name].arrive(label)
        while bars[name].gen == g:
            yield

    def compute(w):
        me = comp[w]
        cur = pool_buf
        if nb > 0:
            read_words(me, 0)
        for b in range(nb):
            for p in range(R):
                rd = cur
                if stage:
                    wr = f"E{b % KS}" if p == R - 1 else f"W{p & 1}"
                else:
                    wr = "W1" if cur == "W0" else "W0"
                prev = ("pool",) if (b == 0 and p == 0) else ((b - 1, R - 1) if p == 0 else (b, p - 1))
                bufs[rd].read(me, prev)
                yield
                if p + 1 < R:  # the next pass's words, loaded during this pass
                    read_words(me, b)
                elif b + 1 < nb:
                    read_words(me, b + 1)
                yield
                if not stage and p == 0 and b > 0:  # the previous block's values, scaled
                    assert scs[(b - 1) % K] == ("sc", b - 1), f"{me} emits block {b - 1} with {scs[(b - 1) % K]}"
                    scs_pending[("sc", b - 1)].discard(me)
                last_pass = p == R - 1
                readers = list(comp) if (b, p) != (nb - 1, R - 1) else []
                if stage and last_pass:
                    readers = readers + [f"s{b % NS}"]
                bufs[wr].write(w, (b, p), readers)
                yield
                if last_pass:
                    done_words(me, b)
                    parts[b % KS].write(w, ("parts", b), ["scale"])
                    bars[f"P{b % MP}"].arrive(("P", b))
                    yield
                    if b + 1 >= KS:
                        yield from sync(f"S{(b + 1 - KS) % MP}", ("S", b + 1 - KS))
                    else:
                        yield from sync("pass", ("pass", b, p))
                else:
                    yield from sync("pass", ("pass", b, p))
                cur = wr
        if not stage and nb > 0:
            assert scs[(nb - 1) % K] == ("sc", nb - 1)
            scs_pending[("sc", nb - 1)].discard(me)

    def scale():
        for b in range(nb):
            yield from sync(f"P{b % MP}", ("P", b))
            parts[b % KS].read("scale", ("parts", b))
            yield
            if stage and b + KS <= nb:  # with staging SCALE(b) only says the sums are read
                bars[f"S{b % MP}"].arrive(("S", b))
                yield
            if b + 1 < nb:
                old = scs[(b + 1) % K]
                assert old is None or not scs_pending[old], f"scale of {old} overwritten before {scs_pending[old]}"
                scs[(b + 1) % K] = ("sc", b + 1)
                scs_pending[("sc", b + 1)] = {f"s{(b + 1) % NS}"} if stage else set(comp)
                yield
                if stage:
                    bars[f"SC{b % MSC}"].arrive(("SC", b))
                else:
                    bars[f"S{b % MP}"].arrive(("S", b))
                yield

    def store(sp):
        me = f"s{sp}"
        for b in range(sp, nb, NS):
            yield from sync(f"P{b % MP}", ("P", b))
            if not stage:
                if b + 1 < nb:
                    bars[f"S{b % MP}"].arrive(("S", b))
                continue
            if b > 0:
                yield from sync(f"SC{(b - 1) % MSC}", ("SC", b - 1))
            assert scs[b % K] == ("sc", b), f"{me} found {scs[b % K]} for block {b}"
            scs_pending[("sc", b)].discard(me)
            # wait_group.read 0: this warp's earlier copy has read T[sp]
            while not all(done for _, done in bulks[sp]):
                yield
            bufs[f"E{b % KS}"].read(me, (b, R - 1))
            yield
            if b + KS <= nb:
                bars[f"S{b % MP}"].arrive(("S", b))
                yield
            bulks[sp].append([b, False])
        while not all(done for _, done in bulks[sp]):  # wait_group 0
            yield

    def drawer():
        for b in range(nb):
            yield from sync(f"P{b % MP}", ("P", b))
            if b + KS + 1 < nb:
                write_words(b + KS + 1)
                yield
            if b + KS <= nb:
                bars[f"S{b % MP}"].arrive(("S", b))
                yield

    actors = [compute(w) for w in range(G)] + [scale()] + [store(k) for k in range(NS)] + [drawer()]
    steps = 0
    while actors:
        # the bulk copies' reads complete at random times
        for lst in bulks.values():
            for bk in lst:
                if not bk[1] and rng.random() < 0.3:
                    bk[1] = True
        a = rng.choice(actors)
        try:
            next(a)
        except StopIteration:
            actors.remove(a)
        steps += 1
        assert steps < 200000, "deadlock"
    for name, bar in bars.items():
        assert bar.arrived == 0, f"barrier {name} left with {bar.arrived} arrivals"


@pytest.mark.parametrize("NS,KE", [(2, 2), (2, 4), (4, 4)])
@pytest.mark.parametrize("stage", [True, False])
@pytest.mark.parametrize("G,R,nb", [(4, 1, 1), (4, 1, 7), (4, 2, 6), (2, 3, 5), (8, 4, 4), (3, 7, 3), (4, 1, 13),
                                    (4, 2, 0)])
def test_chain_protocol_random_schedules(G, R, nb, stage, NS, KE):
    rng = random.Random(1000 * G + 100 * R + nb + stage + 7 * NS + 13 * KE)
    for _ in range(60):
        simulate(G, R, nb, stage, rng, NS, KE)


def test_chain_model_catches_a_missing_wait():
    # the model is not vacuous: without the compute warps' wait at SCALE (each
    # block ending on the pass barrier alone) an emission buffer or the sums
    # of squares get overwritten before a helper read them
    rng = random.Random(5)
    failures = 0
    for _ in range(200):
        try:
            _simulate_without_scale_wait(4, 1, 6, rng)
        except AssertionError:
            failures += 1
    assert failures > 0


def _simulate_without_scale_wait(G, R, nb, rng):
    # as simulate(stage=True) but the compute warps never wait at SCALE; the
    # helpers' arrivals there are dropped so that the barrier counts match
    bars = {"pass": Barrier(G), "P0": Barrier(G + 2), "P1": Barrier(G + 2)}
    bars.update({f"SC{k}": Barrier(2) for k in range(4)})
    comp = [f"c{w}" for w in range(G)]
    bufs = {"E0": Buffer(G, None, []), "E1": Buffer(G, ("pool",), comp)}
    parts = [Buffer(G, None, []), Buffer(G, None, [])]

    def sync(name, label):
        g = bars[name].arrive(label)
        while bars[name].gen == g:
            yield

    def compute(w):
        for b in range(nb):
            par = b & 1
            prev = ("pool",) if b == 0 else (b - 1, R - 1)
            bufs[f"E{par ^ 1}"].read(comp[w], prev)
            yield
            readers = (comp if b < nb - 1 else []) + [f"s{par}"]
            bufs[f"E{par}"].write(w, (b, R - 1), readers)
            parts[par].write(w, ("parts", b), ["scale"])
            bars[f"P{par}"].arrive(("P", b))
            yield
            yield from sync("pass", ("pass", b))

    def scale():
        for b in range(nb):
            yield from sync(f"P{b & 1}", ("P", b))
            for _ in range(rng.randint(0, 30)):
                yield
            parts[b & 1].read("scale", ("parts", b))
            if b + 1 < nb:
                bars[f"SC{b & 3}"].arrive(("SC", b))

    def store(sp):
        for b in range(sp, nb, 2):
            yield from sync(f"P{sp}", ("P", b))
            if b > 0:
                yield from sync(f"SC{(b - 1) & 3}", ("SC", b - 1))
            for _ in range(rng.randint(0, 30)):
                yield
            bufs[f"E{sp}"].read(f"s{sp}", (b, R - 1))

    actors = [compute(w) for w in range(G)] + [scale(), store(0), store(1)]
    steps = 0
    while actors:
        a = rng.choice(actors)
        try:
            next(a)
        except StopIteration:
            actors.remove(a)
        steps += 1
        assert steps < 200000
