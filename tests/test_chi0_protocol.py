"""The mbarrier protocol of the tensor-core chi0 kernels, checked on the CPU.

A random-schedule model of the roles of k_chi0_tc (one tile per CTA) and of
the persistent k_chi0_tc_batch (a list of tiles per CTA, stage and window
counters running on across tiles): the TMA producer, the A-operand
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

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2603_12326_gb300", "csrc")


def _constant(name, src="chi0_tc.cu"):
    m = re.search(r"constexpr int %s = (\d+);" % name, open(os.path.join(CSRC, src)).read())
    assert m, (src, name)
    return int(m.group(1))


class _Bar:
    def __init__(self):
        self.done = 0

    def arrive(self):
        self.done += 1

    def passes(self, parity):
        return (self.done & 1) != parity


def _run(kstages, nstage, promote, seed, ntile=1):
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

    ntot = ntile * kstages                       # stages of all tiles of the CTA, in order

    def producer():
        for gs in range(ntot):
            s, ph = gs % nstage, (gs // nstage) & 1
            yield from wait(empty[s], ph ^ 1, lambda gs=gs: gs < nstage or (gs - nstage) in mma_done,
                            "stage %d free" % gs)
            copies.append((gs, s))

    def a_warps():
        def drain(gw):
            yield from wait(acc_full[gw & 1], (gw >> 1) & 1, lambda: ("win", gw) in mma_done, "window %d" % gw)
            drain_done.add(gw)
            drained[gw & 1].arrive()

        for lt in range(ntile):
            for it in range(kstages):
                gs = lt * kstages + it
                s, ph = gs % nstage, (gs // nstage) & 1
                yield from wait(full_b[s], ph, lambda gs=gs: gs in landed, "copy %d" % gs)
                if gs >= nstage and (gs - nstage) not in mma_done:
                    errors.append("A tile %d overwritten under its MMAs" % gs)
                gen_done.add(gs)
                full_a[s].arrive()
                # drain the previous window after the last stage of a window; at the tile's end the rest
                wd0, wd1 = nwin, -1
                if it % promote == promote - 1 and it >= promote:
                    wd0 = wd1 = it // promote - 1
                if it + 1 == kstages:
                    wd0 = min(wd0, it // promote - 1 if (it % promote == promote - 1 and it >= promote)
                              else max(nwin - 2, 0))
                    wd1 = nwin - 1
                for wd in range(wd0, wd1 + 1):
                    yield from drain(lt * nwin + wd)

    def issuer(par):
        for lt in range(ntile):
            for wd in range(nwin):
                gw = lt * nwin + wd
                if (gw & 1) != par:
                    continue
                b = gw & 1
                if gw >= 2:
                    yield from wait(drained[b], ((gw - 2) >> 1) & 1, lambda g=gw: (g - 2) in drain_done,
                                    "buffer of window %d drained" % gw)
                for it in range(wd * promote, min((wd + 1) * promote, kstages)):
                    gs = lt * kstages + it
                    s = gs % nstage
                    yield from wait(full_a[s], (gs // nstage) & 1, lambda gs=gs: gs in gen_done, "A tile %d" % gs)
                    if gs not in landed:
                        errors.append("MMA %d before its copy landed" % gs)
                    mmas.append((gs, [empty[s]]))
                    yield
                mmas.append((("win", gw), [acc_full[b]]))
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


@pytest.mark.parametrize("kstages,ntile", [(1, 5), (2, 4), (3, 3), (5, 3), (8, 2), (13, 3)])
def test_batch_kernel_protocol_across_tiles(kstages, ntile):
    """The persistent batch kernel runs the same roles over a list of tiles with
    the stage and window counters continuing across tiles."""
    nstage, promote = _constant("NSTAGE", "chi0_tc_batch.cu"), _constant("PROMOTE", "chi0_tc_batch.cu")
    for seed in range(40):
        errors, counts = _run(kstages, nstage, promote, seed, ntile=ntile)
        assert not errors, (kstages, ntile, seed, errors[:3])
        nwin = (kstages + promote - 1) // promote
        assert counts == (kstages * ntile, nwin * ntile)


def test_two_stage_ring_is_caught():
    """With two stages the second issuer's first wait (stage 2, the second use
    of its barrier) can pass before stage 0's tile exists."""
    bad = sum(bool(_run(16, 2, 2, seed)[0]) for seed in range(40))
    assert bad > 0
