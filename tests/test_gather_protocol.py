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


# --------------------------------------------------------------------------
# The ring of input chunks in the gather-type kernels: NCH shared-memory slots
# of ROWS rows each, one mbarrier per slot (the copy of chunk c lands in slot
# c mod NCH and completes phase c // NCH of its barrier).  A round k reads the
# window of rows k*ROWS .. k*ROWS + ROWS + T - 2, i.e. chunks k .. k + KO.
#   After the round (the normal form) every FIR thread has waited for all of
#   them at the round's start; a barrier after the round's reads lets thread 0
#   copy chunk k + NCH into the slot of chunk k.
#   With the early refill (the ":er" tiles) a thread waits for chunk k + w
#   right before its window reaches row w*ROWS, and the barrier sits right
#   after the window's first ROWS rows, so the refill of chunk k's slot is
#   issued mid-round.
# Copies land after random delays.  The model checks that every row is read
# from a slot holding the chunk it belongs to, after that chunk's copy landed,
# that no parity wait sees its barrier two phases ahead, and that every
# interleaving finishes; planting the barrier one row too early, or letting
# thread 0 refill without the barrier, fails.


class Ring:
    def __init__(self, nch):
        self.content = [None] * nch     # chunk whose copy has landed in the slot
        self.pending = [None] * nch     # chunk whose copy is in flight into the slot
        self.bars = [Barrier(1) for _ in range(nch)]


def ring_programs(nthr, nch, rows, T, nr, early, rng, refill_row=None, no_barrier=False):
    ko = (T - 2) // rows + 1 if T >= 2 else 0
    window = rows + T - 1
    nchunks = (nr * rows + T - 1 + rows - 1) // rows
    refill_row = rows if refill_row is None else refill_row
    ring = Ring(nch)
    state = {"issued": 0, "arrived": [0] * (nr + 1), "inflight": []}

    def issue(c):
        s = c % nch
        assert ring.pending[s] is None
        ring.pending[s] = c
        state["inflight"].append(s)

    def copier():
        # lands in-flight copies one at a time, in random order
        while True:
            if state["inflight"]:
                s = state["inflight"].pop(rng.randrange(len(state["inflight"])))
                ring.content[s] = ring.pending[s]
                ring.pending[s] = None
                ring.bars[s].arrive()
            yield None

    def wait_chunk(c):
        s = c % nch
        while not ring.bars[s].wait_ready(c // nch):
            yield "wait"

    def read_row(k, u):
        c = k + u // rows
        if c < nchunks:
            assert ring.content[c % nch] == c, f"row of chunk {c} read from a slot holding {ring.content[c % nch]}"

    def barrier(k, tid):
        state["arrived"][k] += 1
        while state["arrived"][k] < nthr:
            yield "wait"

    def refill(k, tid):
        if not no_barrier:
            yield from barrier(k, tid)
        if tid == 0 and state["issued"] < nchunks and state["issued"] == k + nch:
            issue(state["issued"])
            state["issued"] += 1

    def thread(tid):
        if tid == 0:
            first = min(nch, nchunks)
            for c in range(first):
                issue(c)
            state["issued"] = first
        waited = 0
        for k in range(nr):
            if not early:
                need = min(k + ko, nchunks - 1) + 1
                while waited < need:
                    yield from wait_chunk(waited)
                    waited += 1
            for u in range(window):
                if early:
                    if u % rows == 0:
                        need = min(k + u // rows, nchunks - 1) + 1
                        while waited < need:
                            yield from wait_chunk(waited)
                            waited += 1
                    if u == refill_row:
                        yield from refill(k, tid)
                read_row(k, u)
                yield None
            if not early:
                yield from refill(k, tid)

    return [thread(t) for t in range(nthr)], copier()


def run_ring_model(nthr, nch, rows, T, nr, early, seed, trials=30, **mistake):
    rng = random.Random(seed)
    for trial in range(trials):
        threads, copier = ring_programs(nthr, nch, rows, T, nr, early, rng, **mistake)
        live = set(range(nthr))
        steps = 0
        while live:
            steps += 1
            assert steps < 400000, "ring model did not finish"
            if rng.random() < 0.3:
                next(copier)
            t = rng.choice(sorted(live))
            try:
                next(threads[t])
            except StopIteration:
                live.discard(t)


@pytest.mark.parametrize("early", [False, True])
@pytest.mark.parametrize("nthr,nch,rows,T,nr,seed", [(3, 6, 8, 32, 9, 1), (2, 5, 8, 32, 6, 2), (3, 4, 4, 8, 11, 3),
                                                     (4, 6, 2, 8, 7, 4), (2, 3, 4, 4, 9, 5)])
def test_ring_refill_reads_only_landed_chunks(nthr, nch, rows, T, nr, early, seed):
    run_ring_model(nthr, nch, rows, T, nr, early, seed)


@pytest.mark.parametrize("mistake", [{"refill_row": 7}, {"no_barrier": True}])
def test_early_refill_planted_mistakes_fail(mistake):
    """The mid-round barrier placed one row before the window leaves its first
    chunk, or thread 0 refilling without waiting for the others, is caught."""
    with pytest.raises(AssertionError, match="read from a slot holding"):
        for seed in range(30):
            run_ring_model(3, 6, 8, 32, 9, True, 300 + seed, trials=20, **mistake)


def test_ring_shorter_than_the_window_never_finishes():
    """The kernels' static check (NCH >= KO + 1 chunks) is needed: with a ring
    one chunk shorter than a round's window the model stalls."""
    with pytest.raises(AssertionError, match="did not finish"):
        run_ring_model(2, 4, 2, 8, 5, False, 7, trials=1)
