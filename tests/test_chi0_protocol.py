"""The mbarrier protocol of the tensor-core chi0 kernels, checked on the CPU.

A random-schedule model of the roles of k_chi0_tc (one tile per CTA) and of
the persistent k_chi0_tc_batch (a list of tiles per CTA, stage and window
counters running on across tiles): the TMA producer, every A-operand warp
(eight warps that all take every K stage; in the batch kernel they also drain
the accumulators, in the per-q kernel eight separate warps drain them; groups
of four warps taking every fourth stage are a layout the model also checks),
two MMA issuers on alternate accumulation windows, copies that
land in any order and MMAs that complete in issue order.  A barrier completes
a phase when its expected number of arrivals is in (each A warp arrives on its
own), and a wait on parity p returns once the completed-phase count's parity
differs from p, so a wait that runs one phase ahead of its barrier passes
early.  Every wait records the event it stands for; the test asserts that each
wait passes only after that event, that no shared-memory stage or TMEM buffer
is overwritten while its MMAs may still read it, that every schedule finishes,
and that when the producer leaves no copy is in flight and when TMEM is freed
no MMA is.  The same model runs with waits that give up (a wait limit that
runs out, or copies withheld so that nothing completes): the abort must still
end every role with its copies landed and its MMAs finished.  Ring depth and
window length are read from the kernel sources (four stages, windows of two
for both kernels).  The copy and A-tile barriers are indexed by the stage
modulo (number of A groups, at least two) x ring depth, so a barrier's
previous phase always belongs to the same A-warp group and lies two windows
back for an issuer.  A ring shorter than the window, where an issuer's wait
can pass a phase early, is the negative control."""
import os
import random
import re

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2603_12326_gb300", "csrc")


def _src(name):
    return open(os.path.join(CSRC, name)).read()


def _constant(name, src):
    m = re.search(r"constexpr int %s = (\d+);" % name, _src(src))
    assert m, (src, name)
    return int(m.group(1))


class _Bar:
    def __init__(self, count):
        self.count, self.pending, self.done = count, 0, 0

    def arrive(self):
        self.pending += 1
        assert self.pending <= self.count
        if self.pending == self.count:
            self.pending = 0
            self.done += 1

    def passes(self, parity):
        return (self.done & 1) != parity


def _run(kstages, nstage, promote, seed, ngroups=4, ntile=1, timeouts=False, withhold=False, drain_warps=0):
    """One random schedule.  ngroups = 4: 16 A warps in groups of four, group g
    forms stages g, g+4, ...; a warp drains the windows before wd after its
    group's last stage of window wd; ngroups = 1: 8 A warps, every stage; with
    drain_warps = 0 (the batch kernel) they drain the previous window after a
    window's last stage, with drain_warps = n (the per-q kernel) n other warps
    drain every window in order and the A warps only form A tiles."""
    rnd = random.Random(seed)
    wpg = 4 if ngroups > 1 else 8                 # warps per group
    nwarp = wpg * ngroups
    nb = max(2, ngroups) * nstage                 # copy and A-tile barriers: stage modulo nb
    full_b = [_Bar(1) for _ in range(nb)]
    full_a = [_Bar(wpg) for _ in range(nb)]
    empty = [_Bar(1) for _ in range(nstage)]
    acc_full = [_Bar(1), _Bar(1)]
    ndrain = drain_warps or nwarp
    drained = [_Bar(ndrain), _Bar(ndrain)]
    mma_done_bar = _Bar(2)
    landed, gen_done, mma_done, drain_done = set(), {}, set(), {}
    copies, mmas, errors = [], [], []
    issued = []
    state = {"abort": False, "producer_left": False}
    nwin = (kstages + promote - 1) // promote
    ntot = ntile * kstages

    def wait(bar, parity, event_happened, what, honour_abort=True):
        spins = 0
        while not bar.passes(parity):
            if honour_abort and state["abort"]:
                return False
            spins += 1
            if honour_abort and timeouts and spins > 8 and rnd.random() < 0.01:
                state["abort"] = True             # the wait limit ran out
                return False
            yield
        if not event_happened():
            errors.append("early pass: " + what)
        return True

    def producer():
        for gs in range(0 if withhold else ntot):
            s, ph = gs % nstage, (gs // nstage) & 1
            ok = yield from wait(empty[s], ph ^ 1, lambda gs=gs: gs < nstage or (gs - nstage) in mma_done,
                                 "stage %d free" % gs)
            if not ok:
                break
            copies.append((gs, gs % nb))
            issued.append(gs)
        for gs in issued[-nstage:]:              # let the copies in flight land
            yield from wait(full_b[gs % nb], (gs // nb) & 1, lambda gs=gs: gs in landed,
                            "copy %d" % gs, honour_abort=False)
        if [c for c in copies]:
            errors.append("producer left with copies in flight")
        state["producer_left"] = True

    def a_warp(w):
        grp = w // wpg
        drained_upto = 0

        def drain(gw):
            ok = yield from wait(acc_full[gw & 1], (gw >> 1) & 1, lambda: ("win", gw) in mma_done, "window %d" % gw)
            if ok:
                drain_done[gw] = drain_done.get(gw, 0) + 1
                drained[gw & 1].arrive()
            return ok

        for lt in range(ntile):
            stages = range(grp, kstages, ngroups)
            nxt = 0
            for it in stages:
                gs = lt * kstages + it
                s, ph = gs % nb, (gs // nb) & 1
                ok = yield from wait(full_b[s], ph, lambda gs=gs: gs in landed, "copy %d" % gs)
                if not ok:
                    return
                if gs >= nstage and (gs - nstage) not in mma_done:
                    errors.append("A tile %d overwritten under its MMAs" % gs)
                gen_done[gs] = gen_done.get(gs, 0) + 1
                full_a[s].arrive()
                if drain_warps:
                    nxt = nwin
                elif ngroups > 1:
                    wd = it // promote
                    if it + ngroups >= min((wd + 1) * promote, kstages):
                        while nxt < wd:
                            ok = yield from drain(lt * nwin + nxt)
                            nxt += 1
                            if not ok:
                                return
                else:
                    wd0, wd1 = nwin, -1
                    if it % promote == promote - 1 and it >= promote:
                        wd0 = wd1 = it // promote - 1
                    if it + 1 == kstages:
                        wd0 = min(wd0, it // promote - 1 if (it % promote == promote - 1 and it >= promote)
                                  else max(nwin - 2, 0))
                        wd1 = nwin - 1
                    for wd in range(wd0, wd1 + 1):
                        ok = yield from drain(lt * nwin + wd)
                        if not ok:
                            return
                    nxt = nwin
            while nxt < nwin:
                ok = yield from drain(lt * nwin + nxt)
                nxt += 1
                if not ok:
                    return

    def drain_warp():
        for gw in range(ntile * nwin):
            ok = yield from wait(acc_full[gw & 1], (gw >> 1) & 1, lambda gw=gw: ("win", gw) in mma_done,
                                 "window %d" % gw)
            if not ok:
                return
            drain_done[gw] = drain_done.get(gw, 0) + 1
            drained[gw & 1].arrive()

    def issuer(par):
        ok = True
        for lt in range(ntile):
            for wd in range(nwin):
                gw = lt * nwin + wd
                if (gw & 1) != par or not ok:
                    continue
                b = gw & 1
                if gw >= 2:
                    ok = yield from wait(drained[b], ((gw - 2) >> 1) & 1,
                                         lambda g=gw: drain_done.get(g - 2, 0) == ndrain,
                                         "buffer of window %d drained" % gw)
                    if not ok:
                        break
                for it in range(wd * promote, min((wd + 1) * promote, kstages)):
                    gs = lt * kstages + it
                    s2 = gs % nb
                    ok = yield from wait(full_a[s2], (gs // nb) & 1,
                                         lambda gs=gs: gen_done.get(gs, 0) == wpg, "A tile %d" % gs)
                    if not ok:
                        break
                    if gs not in landed:
                        errors.append("MMA %d before its copy landed" % gs)
                    mmas.append((gs, [empty[gs % nstage]]))
                    yield
                if ok:
                    mmas.append((("win", gw), [acc_full[b]]))
                yield
        mmas.append((("done", par), [mma_done_bar]))
        yield from wait(mma_done_bar, 0, lambda: ("done", 0) in mma_done and ("done", 1) in mma_done,
                        "every MMA finished", honour_abort=False)

    actors = [producer(), issuer(0), issuer(1)] + [a_warp(w) for w in range(nwarp)]
    actors += [drain_warp() for _ in range(drain_warps)]
    alive = [True] * len(actors)
    for _ in range(2000000):
        if not any(alive):
            if mmas:
                errors.append("TMEM freed with MMAs in flight")
            if not state["abort"] and (len(gen_done) != ntot or len(drain_done) != ntile * nwin):
                errors.append("work missing without an abort")
            if withhold and not state["abort"]:
                errors.append("withheld copies did not abort the kernel")
            return errors, state["abort"]
        r = rnd.random()
        if r < 0.15 and copies:
            gs, s2 = copies.pop(rnd.randrange(len(copies)))      # copies land in any order
            landed.add(gs)
            full_b[s2].arrive()
        elif r < 0.3 and mmas:
            key, bars = mmas.pop(0)                               # MMAs complete in issue order
            mma_done.add(key)
            for bar in bars:
                bar.arrive()
        else:
            live = [i for i, a in enumerate(alive) if a]
            i = rnd.choice(live)
            try:
                next(actors[i])
            except StopIteration:
                alive[i] = False
    return errors + ["no progress (deadlock)"], None


def test_model_matches_the_kernel_sources():
    """The constants and counts the model assumes are those of the kernels."""
    for name in ("chi0_tc.cu", "chi0_tc_batch.cu"):
        src = _src(name)
        assert _constant("NSTAGE", name) == 4, name
        assert "mbar_init(&full_a[s], 8)" in src and "mbar_init(&drained[b], 8)" in src, name
        assert "mbar_init(&full_a[s + NSTAGE], 8)" in src, name
        assert src.count("% (2 * NSTAGE)") >= 4, name
    # the per-q kernel: eight A warps (warps 4-11) and eight drain warps (12-19)
    assert _constant("AGEN_WARP0", "chi0_tc.cu") == 4 and _constant("DRAIN_WARP0", "chi0_tc.cu") == 12
    assert _constant("NTHREADS", "chi0_tc.cu") == 640
    assert _constant("PROMOTE", "chi0_tc.cu") == 2
    assert "a.promote = 2;" in _src("chi0_tc_batch.cu")
    assert "for (int it = max(0, last - NSTAGE + 1); it <= last; ++it)" in _src("chi0_tc.cu")


@pytest.mark.parametrize("kstages", [1, 2, 3, 5, 8, 13, 40])
def test_kernel_protocol_holds_under_random_schedules(kstages):
    nstage, promote = _constant("NSTAGE", "chi0_tc.cu"), _constant("PROMOTE", "chi0_tc.cu")
    for seed in range(20):
        errors, aborted = _run(kstages, nstage, promote, seed, ngroups=1, drain_warps=8)
        assert not errors and not aborted, (nstage, kstages, seed, errors[:3])


@pytest.mark.parametrize("nstage,promote,ngroups,drain_warps",
                         [(4, 2, 1, 8), (3, 2, 1, 0), (4, 2, 1, 0), (4, 4, 4, 0), (5, 4, 4, 0), (7, 4, 4, 0)])
def test_kernel_abort_path_drains_copies_and_mmas(nstage, promote, ngroups, drain_warps):
    """Waits that give up at random points (or copies withheld, so that the
    first waits run out): every role ends, the producer leaves no copy in
    flight and no MMA runs when TMEM is freed.  Also for rings of four A-warp
    groups (a layout the model keeps for comparison)."""
    n_abort = 0
    for seed in range(30):
        errors, aborted = _run(24, nstage, promote, seed, ngroups=ngroups, timeouts=True, drain_warps=drain_warps)
        assert not errors, (seed, errors[:3])
        n_abort += bool(aborted)
        errors, aborted = _run(9, nstage, promote, seed, ngroups=ngroups, timeouts=True, withhold=True,
                               drain_warps=drain_warps)
        assert not errors and aborted, (seed, errors[:3])
    assert n_abort > 0


@pytest.mark.parametrize("kstages,ntile", [(1, 5), (2, 4), (3, 3), (5, 3), (8, 2), (13, 3)])
def test_batch_kernel_protocol_across_tiles(kstages, ntile):
    """The persistent batch kernel runs the same roles over a list of tiles with
    the stage and window counters continuing across tiles."""
    nstage = _constant("NSTAGE", "chi0_tc_batch.cu")
    for seed in range(10):
        errors, aborted = _run(kstages, nstage, 2, seed, ngroups=1, ntile=ntile)
        assert not errors and not aborted, (kstages, ntile, seed, errors[:3])
    for seed in range(10):
        errors, aborted = _run(kstages, nstage, 2, seed, ngroups=1, ntile=ntile, timeouts=True)
        assert not errors, (kstages, ntile, seed, errors[:3])


def _run_spec(kstages, nstage, promote, seed, timeouts=False, withhold=False):
    """One random schedule of k_spec_kk_tc: both operands come by TMA, so the
    issuers wait on the copies themselves, and eight warps only drain the
    windows in order."""
    rnd = random.Random(seed)
    nwarp = 8
    nb = 2 * nstage
    full = [_Bar(1) for _ in range(nb)]
    empty = [_Bar(1) for _ in range(nstage)]
    acc_full = [_Bar(1), _Bar(1)]
    drained = [_Bar(nwarp), _Bar(nwarp)]
    mma_done_bar = _Bar(2)
    landed, mma_done, drain_done = set(), set(), {}
    copies, mmas, errors, issued = [], [], [], []
    state = {"abort": False}
    nwin = (kstages + promote - 1) // promote

    def wait(bar, parity, event_happened, what, honour_abort=True):
        spins = 0
        while not bar.passes(parity):
            if honour_abort and state["abort"]:
                return False
            spins += 1
            if honour_abort and timeouts and spins > 8 and rnd.random() < 0.01:
                state["abort"] = True
                return False
            yield
        if not event_happened():
            errors.append("early pass: " + what)
        return True

    def producer():
        for gs in range(0 if withhold else kstages):
            s, ph = gs % nstage, (gs // nstage) & 1
            ok = yield from wait(empty[s], ph ^ 1, lambda gs=gs: gs < nstage or (gs - nstage) in mma_done,
                                 "stage %d free" % gs)
            if not ok:
                break
            copies.append((gs, gs % nb))
            issued.append(gs)
        for gs in issued[-nstage:]:
            yield from wait(full[gs % nb], (gs // nb) & 1, lambda gs=gs: gs in landed, "copy %d" % gs,
                            honour_abort=False)
        if copies:
            errors.append("producer left with copies in flight")

    def drainer():
        for wd in range(nwin):
            ok = yield from wait(acc_full[wd & 1], (wd >> 1) & 1, lambda wd=wd: ("win", wd) in mma_done,
                                 "window %d" % wd)
            if not ok:
                return
            drain_done[wd] = drain_done.get(wd, 0) + 1
            drained[wd & 1].arrive()

    def drain_warp():
        for gw in range(ntile * nwin):
            ok = yield from wait(acc_full[gw & 1], (gw >> 1) & 1, lambda gw=gw: ("win", gw) in mma_done,
                                 "window %d" % gw)
            if not ok:
                return
            drain_done[gw] = drain_done.get(gw, 0) + 1
            drained[gw & 1].arrive()

    def issuer(par):
        ok = True
        for wd in range(par, nwin, 2):
            b = wd & 1
            if wd >= 2:
                ok = yield from wait(drained[b], ((wd - 2) >> 1) & 1, lambda w=wd: drain_done.get(w - 2, 0) == nwarp,
                                     "buffer of window %d drained" % wd)
                if not ok:
                    break
            for gs in range(wd * promote, min((wd + 1) * promote, kstages)):
                ok = yield from wait(full[gs % nb], (gs // nb) & 1, lambda gs=gs: gs in landed, "copy %d" % gs)
                if not ok:
                    break
                mmas.append((gs, [empty[gs % nstage]]))
                yield
            if not ok:
                break
            mmas.append((("win", wd), [acc_full[b]]))
            yield
        mmas.append((("done", par), [mma_done_bar]))
        yield from wait(mma_done_bar, 0, lambda: ("done", 0) in mma_done and ("done", 1) in mma_done,
                        "every MMA finished", honour_abort=False)

    actors = [producer(), issuer(0), issuer(1)] + [drainer() for _ in range(nwarp)]
    alive = [True] * len(actors)
    for _ in range(2000000):
        if not any(alive):
            if mmas:
                errors.append("TMEM freed with MMAs in flight")
            if not state["abort"] and len(drain_done) != nwin:
                errors.append("work missing without an abort")
            if withhold and not state["abort"]:
                errors.append("withheld copies did not abort the kernel")
            return errors, state["abort"]
        r = rnd.random()
        if r < 0.15 and copies:
            gs, s2 = copies.pop(rnd.randrange(len(copies)))
            landed.add(gs)
            full[s2].arrive()
        elif r < 0.3 and mmas:
            key, bars = mmas.pop(0)
            mma_done.add(key)
            for bar in bars:
                bar.arrive()
        else:
            live = [i for i, a in enumerate(alive) if a]
            i = rnd.choice(live)
            try:
                next(actors[i])
            except StopIteration:
                alive[i] = False
    return errors + ["no progress (deadlock)"], None


@pytest.mark.parametrize("kstages", [1, 2, 3, 5, 8, 13, 40, 128])
def test_spectral_kernel_protocol(kstages):
    """k_spec_kk_tc (the spectral route's contraction): ring depth, window and
    barrier counts read from its source; random schedules with and without
    waits that give up, and with the copies withheld."""
    src = _src("spectral_tc.cu")
    nstage, promote = _constant("SK_NSTAGE", "spectral_tc.cu"), _constant("SK_PROMOTE", "spectral_tc.cu")
    assert "mbar_init(&drained[b], 8)" in src and src.count("% (2 * SK_NSTAGE)") >= 3
    assert "for (int it = max(0, last - SK_NSTAGE + 1); it <= last; ++it)" in src
    for seed in range(15):
        errors, aborted = _run_spec(kstages, nstage, promote, seed)
        assert not errors and not aborted, (kstages, seed, errors[:3])
        errors, _ = _run_spec(kstages, nstage, promote, seed, timeouts=True)
        assert not errors, (kstages, seed, errors[:3])
        errors, aborted = _run_spec(kstages, nstage, promote, seed, timeouts=True, withhold=True)
        assert not errors and aborted, (kstages, seed, errors[:3])


def test_short_ring_is_caught():
    """A window longer than the ring (five stages per window on a ring of
    two) lets an issuer's wait on an A-tile barrier pass one phase early."""
    bad = sum(bool(_run(20, 2, 5, seed, ngroups=1)[0]) for seed in range(20))
    assert bad > 0


def test_warpgroup_register_budgets_fit_the_launch():
    """k_chi0_tc trades registers between its warpgroups with setmaxnreg: one control warpgroup, two
    A-generation and two drain warpgroups.  An increase waits until other warpgroups give registers
    back, so the budgets must sum to at most the block's launch allocation (threads x registers per
    thread at launch, 65536 / 640 rounded down to 8), or the drain warps would wait forever; the host
    refuses to launch a build whose register count differs from LAUNCH_REGS."""
    src = _src("chi0_tc.cu")
    m = re.search(r"constexpr int REG_CTRL = (\d+), REG_AGEN = (\d+), REG_DRAIN = (\d+);", src)
    assert m
    ctrl, agen, drain = (int(x) for x in m.groups())
    nthreads, launch = _constant("NTHREADS", "chi0_tc.cu"), _constant("LAUNCH_REGS", "chi0_tc.cu")
    assert launch == (65536 // nthreads) // 8 * 8
    assert 128 * ctrl + 256 * agen + 256 * drain <= nthreads * launch
    for r in (ctrl, agen, drain):
        assert r % 8 == 0 and 24 <= r <= 256          # setmaxnreg's range and granule
    assert "if (fa.numRegs != LAUNCH_REGS) return cudaErrorNotSupported;" in src
    # every warp of a warpgroup takes the same budget: the roles split at warpgroup boundaries
    assert _constant("AGEN_WARP0", "chi0_tc.cu") % 4 == 0 and _constant("DRAIN_WARP0", "chi0_tc.cu") % 4 == 0
