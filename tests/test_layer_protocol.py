"""A model of the handoff protocol of the fused message-passing layer
(k_message_tc in csrc/mpnn.cu), run on the CPU under random timing.

The layer's roles share one CTA and hand off through mbarriers only: two
gather groups (even and odd neighbour steps) fill an 8-slot operand ring and
announce their copies three at a time; one thread issues the MMAs into a ring
of four TMEM accumulators; the epilogue releases each accumulator and
finishes each tile. Every wait in the kernel is bounded, so a protocol that
could block for good would surface as a timeout, not a hang; this model
checks that it cannot. Each role is a generator that yields the waits the
kernel makes, with the same barriers, parities, ring sizes, announcement
batching and tile-start flush rule; copies and MMAs complete after random
delays (an MMA commit arrives once every earlier MMA has completed, as
tcgen05.commit does), and a scheduler runs a random ready role at each
tick. A run that stops with every role waiting is a deadlock.

The model counts one arrival per role where the kernel's threads or warps
all arrive together. Two variants must deadlock, which shows that the
checker finds the cycles it is written for: announcing copy groups too late
(four outstanding groups spanning eight steps, the whole ring), and leaving
out the flush at tile starts (a short tile's groups then stay unannounced
while the gather waits for the end of the tile before it)."""
import random

import pytest

NS, ND, QD = 8, 4, 3  # ring slots, TMEM step accumulators, announcement batch


class Bar:
    """An mbarrier with an expected count of one arrival per phase."""

    def __init__(self):
        self.phase = 0

    def arrive(self):
        self.phase += 1

    def done(self, parity):  # try_wait.parity: the phase of that parity has completed
        return (self.phase & 1) != parity


class Model:
    def __init__(self, kmax, rng, qd=QD, batch=QD, flush=True):
        self.kmax, self.rng, self.qd, self.batch, self.flush = kmax, rng, qd, batch, flush
        self.b = {}
        self.copies = {}   # copy group id -> completion tick
        self.mma = []      # issued MMAs: completion ticks, in order
        self.commits = []  # (index of the last MMA it covers, barrier)
        self.tick = 0
        self.next_copy = 0

    def bar(self, name):
        return self.b.setdefault(name, Bar())

    # ---- asynchronous completions ----
    def issue_copy(self):
        cid = self.next_copy
        self.next_copy += 1
        self.copies[cid] = self.tick + self.rng.randint(1, 40)
        return cid

    def copy_done(self, cid):
        return self.copies[cid] <= self.tick

    def issue_mma(self, n=1):
        for _ in range(n):
            last = self.mma[-1] if self.mma else self.tick
            self.mma.append(max(last, self.tick) + self.rng.randint(1, 12))

    def commit(self, name):
        self.commits.append((len(self.mma) - 1, name))

    def advance(self):
        self.tick += 1
        keep = []
        for idx, name in self.commits:
            if idx < 0 or self.mma[idx] <= self.tick:
                self.bar(name).arrive()
            else:
                keep.append((idx, name))
        self.commits = keep

    def pending_async(self):
        return bool(self.commits) or any(t > self.tick for t in self.copies.values())

    # ---- the roles ----
    def gather(self, grp):
        """One gather group (its warps move together)."""
        q = []  # (barrier, copy group) not yet announced, oldest first
        gs0, prev_groups = 0, self.qd

        def wait_copies(keep):  # wait for all but the newest `keep` copy groups
            while not all(self.copy_done(c) for _, c in q[:len(q) - keep]):
                yield ("copies",)

        def announce(n):
            for _ in range(n):
                self.bar(q.pop(0)[0]).arrive()

        def push(name, cid):
            q.append((name, cid))
            if len(q) > self.qd:  # a further group in flight: announce a batch under one fence
                yield from wait_copies(len(q) - self.batch)
                announce(self.batch)

        def flush_to(keep):
            if len(q) > keep:
                yield from wait_copies(keep)
                announce(len(q) - keep)

        for it in range(len(self.kmax) + 1):
            tb = it & 1
            if self.flush:
                yield from flush_to(min(prev_groups, self.qd))
            last = it == len(self.kmax)
            groups = 0
            if grp == 0:
                yield ("wait", ("IFREE", tb), ((it >> 1) & 1) ^ 1)
                self.bar(("IFULL", tb)).arrive()
                if last:
                    break
            else:
                yield ("wait", ("IFULL", tb), (it >> 1) & 1)
                if last:
                    break
                yield ("wait", ("HFREE", tb), ((it >> 1) & 1) ^ 1)
                yield from push(("HFULL", tb), self.issue_copy())
                groups = 1
            km = self.kmax[it]
            for k in range((gs0 ^ grp) & 1, km, 2):
                gs = gs0 + k
                s = gs % NS
                yield ("wait", ("SFREE", s), ((gs // NS) & 1) ^ 1)
                yield from push(("SFULL", s), self.issue_copy())
                groups += 1
            gs0 += km
            prev_groups = groups
        yield from flush_to(0)

    def mma_thread(self):
        gs, nmsg = 0, 0
        for it in range(len(self.kmax) + 1):
            tb = it & 1
            yield ("wait", ("IFULL", tb), (it >> 1) & 1)
            if it == len(self.kmax):
                break
            km = self.kmax[it]
            yield ("wait", ("HFULL", tb), (it >> 1) & 1)
            if km > 0:
                self.issue_mma(4)
                self.commit("PR")
                for _ in range(km):
                    s, d = gs % NS, gs % ND
                    yield ("wait", ("SFULL", s), (gs // NS) & 1)
                    yield ("wait", ("DFREE", d), ((gs // ND) & 1) ^ 1)
                    self.issue_mma(3)
                    self.commit(("DFULL", d))
                    self.commit(("SFREE", s))
                    gs += 1
                yield ("wait", "HL", nmsg & 1)
                nmsg += 1
                self.issue_mma(8)
                self.commit("DM")
            yield ("wait", "M", it & 1)
            self.issue_mma(8)
            self.commit("Z")
            yield ("wait", "ZT", it & 1)
            self.issue_mma(4)
            self.commit("O")
        self.commit("FIN")
        yield ("wait", "FIN", 0)

    def epilogue(self):
        gs, nmsg = 0, 0
        for it in range(len(self.kmax) + 1):
            tb = it & 1
            yield ("wait", ("IFULL", tb), (it >> 1) & 1)
            if self.record_of(it) is None:
                break
            km = self.kmax[it]
            if km > 0:
                yield ("wait", "PR", nmsg & 1)
                for _ in range(km):
                    d = gs % ND
                    yield ("wait", ("DFULL", d), (gs // ND) & 1)
                    self.bar(("DFREE", d)).arrive()
                    gs += 1
                self.bar("HL").arrive()
                yield ("wait", "DM", nmsg & 1)
                nmsg += 1
            self.bar("M").arrive()
            yield ("wait", "Z", it & 1)
            self.bar("ZT").arrive()
            yield ("wait", "O", it & 1)
            self.bar(("HFREE", tb)).arrive()
            self.bar(("IFREE", tb)).arrive()

    def record_of(self, it):
        return None if it == len(self.kmax) else self.kmax[it]

    # ---- the scheduler ----
    def run(self, max_ticks=200000):
        roles = {"g0": self.gather(0), "g1": self.gather(1), "mma": self.mma_thread(), "epi": self.epilogue()}
        waiting = {name: None for name in roles}
        while roles:
            ready = []
            for name, w in waiting.items():
                if w is None:
                    ready.append(name)
                elif w[0] == "copies":
                    ready.append(name)  # re-checked by the generator itself
                elif self.bar(w[1]).done(w[2]):
                    ready.append(name)
            progressed = False
            self.rng.shuffle(ready)
            for name in ready[:self.rng.randint(1, len(ready))] if ready else []:
                w = waiting[name]
                before = w
                try:
                    waiting[name] = next(roles[name])
                except StopIteration:
                    del roles[name], waiting[name]
                    progressed = True
                    continue
                if not (before is not None and before[0] == "copies" and waiting[name][0] == "copies"):
                    progressed = True
            if not progressed and not self.pending_async():
                blocked = {n: w for n, w in waiting.items()}
                return False, blocked
            self.advance()
            if self.tick > max_ticks:
                return False, {"timeout": self.tick}
        return True, None


def _lists(rng):
    """Longest lists of a CTA's tiles: fluid tiles of mixed lengths (empty,
    a few steps, long), then wall tiles (no messages)."""
    kind = rng.choice(["short", "mixed", "long", "empty"])
    nt = rng.randint(1, 9)
    if kind == "short":
        fl = [rng.randint(0, 5) for _ in range(nt)]
    elif kind == "long":
        fl = [rng.randint(20, 40) for _ in range(nt)]
    elif kind == "empty":
        fl = [0] * nt
    else:
        fl = [rng.choice([0, 1, 2, 3, 4, 7, 9, 13, 30]) for _ in range(nt)]
    return fl + [0] * rng.randint(0, 3)


def test_layer_protocol_never_blocks_under_random_timing():
    rng = random.Random(2026)
    for trial in range(400):
        km = _lists(rng)
        ok, blocked = Model(km, random.Random(rng.random())).run()
        assert ok, (trial, km, blocked)


@pytest.mark.parametrize("kmax", [[0], [1], [2, 0, 3], [5] * 6, [40, 0, 1, 40], [8, 8, 8, 8, 8, 8, 8]])
def test_layer_protocol_fixed_cases(kmax):
    for seed in range(20):
        ok, blocked = Model(kmax, random.Random(seed)).run()
        assert ok, (seed, blocked)


def test_the_checker_finds_a_cycle_when_announcements_come_too_late():
    """Keeping four copy groups unannounced lets a thread's pending steps
    span the whole ring of eight: the thread then waits for a slot whose
    MMA waits for that thread's own announcement."""
    rng = random.Random(7)
    found = False
    for trial in range(200):
        km = [rng.randint(10, 30) for _ in range(3)]
        ok, _ = Model(km, random.Random(trial), qd=4, batch=4).run()
        if not ok:
            found = True
            break
    assert found


def test_the_checker_finds_a_cycle_without_the_tile_start_flush():
    found = False
    for trial in range(200):
        ok, _ = Model([1, 0, 0, 2, 0, 0], random.Random(trial), flush=False).run()
        if not ok:
            found = True
            break
    assert found
