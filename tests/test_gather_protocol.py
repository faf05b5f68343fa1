"""Model of the gather kernel's pipelined round protocol (two FFT buffers per CTA).

The kernel (paper_1411_3656_gb300/csrc/ppf_gather.cuh, tiles named ":db") runs, on
each of the P CTAs of a cluster: FIR of round 0; then for every round k, the FIR of
round k+1 and the FFT of round k.  Round g uses FFT buffer b = g mod 2 of every owner;
each buffer has a "full" mbarrier (one local arrival with the expected bytes, plus the
P slices other CTAs store into it, counted as transaction bytes) and a "free"
mbarrier (P arrivals, one per owner after its last FFT-pass loads of that buffer).
A sender waits for phase (g-2)/2 of its own "free" barrier of buffer b before
storing round g; an owner waits for phase g/2 of its "full" barrier before
transforming round g.  Waits use the parity of the phase, so the model also checks
that no barrier is ever more than one phase ahead of the phase waited for.

Random interleavings of the CTAs must never deadlock, never let a slice of round g
land in a buffer an owner still reads for round g-2, and give every FFT exactly the P
slices of its own round.  Host-only: no GPU.
"""
import random

import pytest


class Barrier:
    """An mbarrier phase counter: a phase completes after `count` arrivals and,
    for the 'full' barriers, `tx` transaction units."""

    def __init__(self, count, tx=0):
        self.count, self.tx_needed = count, tx
        self.completed = 0
        self.arrivals = 0
        self.tx = 0

    def _maybe_complete(self):
        if self.arrivals == self.count and self.tx == self.tx_needed:
            self.completed += 1
            self.arrivals = 0
            self.tx = 0

    def arrive(self):
        self.arrivals += 1
        assert self.arrivals <= self.count
        self._maybe_complete()

    def complete_tx(self):
        self.tx += 1
        assert self.tx <= self.tx_needed
        self._maybe_complete()

    def wait_ready(self, phase):
        # parity wait for phase `phase`: true once that phase has completed; the
        # barrier must not have run a further phase (its parity would match again)
        assert self.completed <= phase + 1, "barrier ran two phases ahead of a waiter"
        return self.completed == phase + 1


class CTA:
    def __init__(self, rank, P):
        self.rank, self.P = rank, P
        self.full = [Barrier(1, P), Barrier(1, P)]
        self.free = [Barrier(P), Barrier(P), ]
        self.buf = [dict(), dict()]      # buffer b: {sender rank: round}
        self.reading = [None, None]      # round being transformed in buffer b
        self.done_rounds = []


def cta_program(me, ctas, nr, skip_free_wait=False, free_before_read=False):
    P = len(ctas)

    def fir(g):
        b = g & 1
        # the local arrival with the expected bytes belongs to phase g/2
        assert me.full[b].completed == g >> 1
        me.full[b].arrive()
        yield None  # the FIR arithmetic
        if g >= 2 and not skip_free_wait:
            while not me.free[b].wait_ready((g - 2) >> 1):
                yield "wait"
        for owner in ctas:
            # the owner may not still be reading round g-2 from this buffer
            assert owner.reading[b] != g - 2, "slice stored into a buffer still being read"
            assert owner.full[b].completed == g >> 1
            owner.buf[b][me.rank] = g
            owner.full[b].complete_tx()
            yield None

    def fft(g):
        b = g & 1
        while not me.full[b].wait_ready(g >> 1):
            yield "wait"
        if free_before_read:
            for peer in ctas:
                peer.free[b].arrive()
            yield None
        assert me.buf[b] == {r: g for r in range(P)}, "FFT input is not exactly round g's slices"
        me.reading[b] = g
        yield None  # the passes' loads
        me.reading[b] = None
        if not free_before_read:
            for peer in ctas:
                peer.free[b].arrive()
        yield None  # the rest of the passes and the stores
        me.done_rounds.append(g)

    if nr > 0:
        yield from fir(0)
    for k in range(nr):
        if k + 1 < nr:
            yield from fir(k + 1)
        yield from fft(k)


@pytest.mark.parametrize("P,nr,seed", [(2, 1, 0), (2, 2, 1), (2, 9, 2), (4, 7, 3), (8, 12, 4), (8, 3, 5), (3, 10, 6)])
def test_pipelined_rounds_complete_without_overwrites(P, nr, seed):
    run_gather_model(P, nr, seed)


@pytest.mark.parametrize("mistake", ["skip_free_wait", "free_before_read"])
def test_pipelined_planted_mistakes_fail(mistake):
    """The sender's wait for the buffer's release left out, or an owner freeing a
    buffer before reading it, is caught in some interleaving."""
    with pytest.raises(AssertionError):
        for seed in range(30):
            run_gather_model(4, 8, 200 + seed, trials=20, **{mistake: True})


def run_gather_model(P, nr, seed, trials=40, **mistake):
    rng = random.Random(seed)
    for trial in range(trials):
        ctas = [CTA(r, P) for r in range(P)]
        progs = {r: cta_program(ctas[r], ctas, nr, **mistake) for r in range(P)}
        blocked = {r: False for r in range(P)}
        live = set(range(P))
        steps = 0
        while live:
            steps += 1
            assert steps < 100000
            r = rng.choice(sorted(live))
            try:
                st = next(progs[r])
            except StopIteration:
                live.discard(r)
                continue
            blocked[r] = st == "wait"
            if live and all(blocked[q] for q in live):
                # every live CTA is waiting: one more round of polls must free one
                progressed = False
                for q in sorted(live):
                    try:
                        st = next(progs[q])
                    except StopIteration:
                        live.discard(q)
                        progressed = True
                        continue
                    if st != "wait":
                        blocked[q] = False
                        progressed = True
                assert progressed or not live, f"deadlock (P={P}, rounds={nr}, trial={trial})"
        for c in ctas:
            assert c.done_rounds == list(range(nr))


# --------------------------------------------------------------------------
# The warp-specialised gather kernel (paper_1411_3656_gb300/csrc/ppf_gws.cuh):
# every CTA runs two programs at once, a FIR role and an FFT role, over the
# same rounds.  Round g uses buffer b = g mod NXB (NXB = 1 or 2 FFT buffers per
# CTA), phase g // NXB of that buffer's barriers.  The FIR role filters round g,
# then (g >= NXB) waits for phase (g - NXB) // NXB of its "free" barrier of b,
# only then makes the local arrival (expected bytes) on its own "full" barrier
# of b, and stores its slice into every owner's buffer b.  The FFT role waits
# for phase g // NXB of its "full" barrier of b, reads the buffer, arrives on
# every CTA's "free" barrier of b and stores the spectra.  The FIR role may run
# ahead of its own FFT role; the model checks that the local arrival never
# lands on a phase that has not completed yet.


def gws_programs(me, ctas, nr, nxb, arrive_before_free_wait=False, skip_free_wait=False):
    P = len(ctas)

    def fir_role():
        for g in range(nr):
            b = g % nxb
            yield None  # the FIR arithmetic of round g
            if arrive_before_free_wait:
                me.full[b].arrive()
            if g >= nxb and not skip_free_wait:
                while not me.free[b].wait_ready((g - nxb) // nxb):
                    yield "wait"
            if not arrive_before_free_wait:
                # the earlier phase of this buffer has completed
                assert me.full[b].completed == g // nxb, "local arrival on a phase still open"
                me.full[b].arrive()
            for owner in ctas:
                assert owner.reading[b] != g - nxb, "slice stored into a buffer still being read"
                assert owner.full[b].completed == g // nxb, "slice of round g counted in another phase"
                owner.buf[b][me.rank] = g
                owner.full[b].complete_tx()
                yield None

    def fft_role():
        for g in range(nr):
            b = g % nxb
            while not me.full[b].wait_ready(g // nxb):
                yield "wait"
            assert me.buf[b] == {r: g for r in range(P)}, "FFT input is not exactly round g's slices"
            me.reading[b] = g
            yield None  # the passes' loads
            me.reading[b] = None
            for peer in ctas:
                peer.free[b].arrive()
            yield None  # the rest of the passes and the stores
            me.done_rounds.append(g)

    return fir_role(), fft_role()


def run_gws_model(P, nr, nxb, seed, trials=40, **mistake):
    rng = random.Random(seed)
    for trial in range(trials):
        ctas = [CTA(r, P) for r in range(P)]
        progs = {}
        for r in range(P):
            progs[(r, "fir")], progs[(r, "fft")] = gws_programs(ctas[r], ctas, nr, nxb, **mistake)
        blocked = {k: False for k in progs}
        live = set(progs)
        steps = 0
        while live:
            steps += 1
            assert steps < 200000
            k = rng.choice(sorted(live))
            try:
                st = next(progs[k])
            except StopIteration:
                live.discard(k)
                continue
            blocked[k] = st == "wait"
            if live and all(blocked[q] for q in live):
                progressed = False
                for q in sorted(live):
                    try:
                        st = next(progs[q])
                    except StopIteration:
                        live.discard(q)
                        progressed = True
                        continue
                    if st != "wait":
                        blocked[q] = False
                        progressed = True
                assert progressed or not live, f"deadlock (P={P}, rounds={nr}, NXB={nxb}, trial={trial})"
        for c in ctas:
            assert c.done_rounds == list(range(nr))


@pytest.mark.parametrize("nxb", [1, 2])
@pytest.mark.parametrize("P,nr,seed", [(2, 1, 10), (2, 7, 11), (4, 9, 12), (8, 12, 13), (3, 10, 14)])
def test_warp_specialised_rounds_complete_without_overwrites(P, nr, nxb, seed):
    run_gws_model(P, nr, nxb, seed)


@pytest.mark.parametrize("mistake", ["arrive_before_free_wait", "skip_free_wait"])
@pytest.mark.parametrize("nxb", [1, 2])
def test_warp_specialised_planted_mistakes_fail(mistake, nxb):
    """The local arrival made before the wait for the buffer's release, or the
    release wait left out, is caught in some interleaving."""
    with pytest.raises(AssertionError):
        for seed in range(30):
            run_gws_model(4, 8, nxb, 100 + seed, trials=20, **{mistake: True})
