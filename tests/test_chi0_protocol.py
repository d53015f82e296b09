"""The mbarrier protocol of the tensor-core chi0 kernel, checked on the CPU.

A random-schedule model of k_chi0_tc's roles: the TMA producer, the A-operand
warps (which also drain the accumulators), two MMA issuers on alternate
accumulation windows, copies that land in any order and MMAs that complete in
issue order.  Barriers follow the mbarrier phase rule (a wait on parity p
returns once the current phase's parity differs from p), so a wait that runs
one phase ahead of its barrier passes early.  Every wait records the event it
stands for; the test asserts that each wait passes only after that event,
that no shared-memory stage or TMEM buffer is overwritten while its MMAs may
still read it, and that every schedule finishes.  The ring depth and window
length are read from the kernel source, so a change to either is re-checked.
A ring of two stages, where an issuer's first wait can pass a phase early, is
the negative control."""
import os
import random
import re

import pytest

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2603_12326_gb300", "csrc", "chi0_tc.cu")


def _constant(name):
    m = re.search(r"constexpr int %s = (\d+);" % name, open(SRC).read())
    assert m, name
    return int(m.group(1))


class _Bar:
    def __init__(self):
        self.done = 0

    def arrive(self):
        self.done += 1

    def passes(self, parity):
        return (self.done & 1) != parity


def _run(kstages, nstage, promote, seed):
    rnd = random.Random(seed)
    full_b = [_Bar() for _ in range(nstage)]
    full_a = [_Bar() for _ in range(nstage)]
    empty = [_Bar() for _ in range(nstage)]
    acc_full = [_Bar(), _Bar()]
    drained = [_Bar(), _Bar()]
    landed, gen_done, mma_done, drain_done = set(), set(), set(), set()
    copies, mmas, errors = [], [], []
    nwin = (kstages + promote - 1) // promote

    def wait(bar, parity, event_happened, what):
        while not bar.passes(parity):
            yield
        if not event_happened():
            errors.append("early pass: " + what)

    def producer():
        for it in range(kstages):
            s, ph = it % nstage, (it // nstage) & 1
            yield from wait(empty[s], ph ^ 1, lambda it=it: it < nstage or (it - nstage) in mma_done,
                            "stage %d free" % it)
            copies.append((it, s))

    def a_warps():
        def drain(wd):
            yield from wait(acc_full[wd & 1], (wd >> 1) & 1, lambda: ("win", wd) in mma_done, "window %d" % wd)
            drain_done.add(wd)
            drained[wd & 1].arrive()

        for it in range(kstages):
            s, ph = it % nstage, (it // nstage) & 1
            yield from wait(full_b[s], ph, lambda it=it: it in landed, "copy %d" % it)
            if it >= nstage and (it - nstage) not in mma_done:
                errors.append("A tile %d overwritten under its MMAs" % it)
            gen_done.add(it)
            full_a[s].arrive()
            if it % promote == promote - 1 and it >= promote:
                yield from drain(it // promote - 1)
        if nwin >= 2 and (kstages - 1) % promote != promote - 1:
            yield from drain(nwin - 2)
        yield from drain(nwin - 1)

    def issuer(par):
        for win in range(par, nwin, 2):
            b = win & 1
            if win >= 2:
                yield from wait(drained[b], ((win - 2) >> 1) & 1, lambda w=win: (w - 2) in drain_done,
                                "buffer of window %d drained" % win)
            for it in range(win * promote, min((win + 1) * promote, kstages)):
                s = it % nstage
                yield from wait(full_a[s], (it // nstage) & 1, lambda it=it: it in gen_done, "A tile %d" % it)
                if it not in landed:
                    errors.append("MMA %d before its copy landed" % it)
                mmas.append((it, [empty[s]]))
                yield
            mmas.append((("win", win), [acc_full[b]]))
            yield

    actors = [producer(), a_warps(), issuer(0), issuer(1)]
    alive = [True] * len(actors)
    for _ in range(400000):
        if not any(alive) and not copies and not mmas:
            return errors, (len(gen_done), len(drain_done))
        r = rnd.random()
        if r < 0.2 and copies:
            it, s = copies.pop(rnd.randrange(len(copies)))       # copies land in any order
            landed.add(it)
            full_b[s].arrive()
        elif r < 0.4 and mmas:
            key, bars = mmas.pop(0)                               # MMAs complete in issue order
            mma_done.add(key)
            for bar in bars:
                bar.arrive()
        else:
            live = [i for i, a in enumerate(alive) if a]
            if live:
                i = rnd.choice(live)
                try:
                    next(actors[i])
                except StopIteration:
                    alive[i] = False
    return errors + ["no progress (deadlock)"], None


@pytest.mark.parametrize("kstages", [1, 2, 3, 5, 8, 63])
def test_kernel_protocol_holds_under_random_schedules(kstages):
    nstage, promote = _constant("NSTAGE"), _constant("PROMOTE")
    for seed in range(60):
        errors, counts = _run(kstages, nstage, promote, seed)
        assert not errors, (nstage, promote, kstages, seed, errors[:3])
        nwin = (kstages + promote - 1) // promote
        assert counts == (kstages, nwin)


def test_two_stage_ring_is_caught():
    """With two stages the second issuer's first wait (stage 2, the second use
    of its barrier) can pass before stage 0's tile exists."""
    bad = sum(bool(_run(16, 2, 2, seed)[0]) for seed in range(40))
    assert bad > 0
