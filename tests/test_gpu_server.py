"""Serving (ppf_server_*): continuous batching of many streams.

The defining property: a stream's spectra are the same alone and in the mix
(bitwise: every spectrum is computed by the same kernel from the same inputs),
and equal to ppf_execute on the stream's concatenated samples.  Each stream's
served spectra are also compared with the FP64 oracle (relative L2 <= 1e-5,
reduced-precision streams on their stored values with the FP16 coefficients
the device uses): the first spectrum after admission, every spectrum whose
window straddles a chunk boundary (history spliced onto a chunk head by the
tick's copy segments), the last, and a seeded sample.
"""
import numpy as np
import pytest

import oracle
from paper_1411_3656_gb300 import synth

TOL32 = 1e-5

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppf():
    import torch
    from paper_1411_3656_gb300 import build, ppf as mod
    build.build()
    mod.load()
    assert torch.cuda.is_available()
    return mod


class Feed:
    """A stream: plan, its whole sample sequence on the device, cut into chunks."""

    def __init__(self, ppf, N, T, dtype, total, seed, chunks):
        import torch
        g = np.random.default_rng(seed)
        self.h = g.standard_normal(N * T).astype(np.float32)
        x = synth.stream(total, N, seed + 1)
        if dtype == "ci8":
            x = synth.int8_iq(total, seed + 2)
        elif dtype == "c16":
            x = synth.to_fp16_iq(x)
        self.plan = ppf.Plan(N, T, self.h, dtype)
        self.x_host = x
        self.h_dev = self.h if dtype == "c32" else self.h.astype(np.float16).astype(np.float32)
        self.x = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        self.N, self.T, self.dtype, self.total = N, T, dtype, total
        cuts = np.sort(g.choice(np.arange(1, total), size=chunks - 1, replace=False))
        self.bounds = list(zip([0, *cuts], [*cuts, total]))
        self.outs = []

    def chunk(self, i):
        a, b = self.bounds[i]
        return self.x[a:b]

    def batch_reference(self):
        return self.plan(self.x)

    def oracle_rows(self):
        """First, last, straddling and sampled spectra of the whole stream."""
        N, T = self.N, self.T
        S = max(0, self.total // N - T + 1)
        rows = {0, S - 1} | set(synth.sample_rows(S, 64).tolist())
        for a, _ in self.bounds[1:]:  # chunk boundary at sample a
            lo = max(0, -(-(a - T * N + 1) // N))
            hi = min(S - 1, (a - 1) // N)
            rows |= set(range(lo, hi + 1))
        return np.asarray(sorted(r for r in rows if 0 <= r < S), dtype=np.int64)

    def check_oracle(self, got):
        rows = self.oracle_rows()
        ref = oracle.ppf_rows(self.x_host, self.h_dev, self.N, self.T, rows)
        g = got.cpu().numpy()[rows]
        err = synth.rel_l2(g, ref)
        assert err <= TOL32, (self.N, self.T, self.dtype, err, synth.worst_spectrum_rel_l2(g, ref))


def _serve(ppf, feeds, schedule, max_chunk, stats=None):
    """schedule: list of ticks, each a list of (feed index, chunk index)."""
    import torch
    srv = ppf.Server(max_streams=16, memory_budget_bytes=8 << 30)
    slots = [srv.admit(f.plan, max_chunk) for f in feeds]
    outs = [[] for _ in feeds]
    keep = []
    for tick in schedule:
        queued = [0] * len(feeds)
        for fi, ci in tick:
            f = feeds[fi]
            c = f.chunk(ci)
            n = c.shape[0]
            k = srv.expected(slots[fi], queued[fi], n)
            out = torch.empty((k, f.N), dtype=torch.complex64, device="cuda")
            assert srv.submit(slots[fi], c, out) == 0
            queued[fi] += n
            outs[fi].append(out)
            keep.append(c)
        srv.tick()
    torch.cuda.synchronize()
    res = [torch.cat(o) if o else None for o in outs]
    if stats is not None:
        stats["ticks"] = sum(1 for t in schedule if t)  # a tick with nothing queued launches nothing
        stats["graph_ticks"] = srv.graph_ticks
        stats["launches"] = srv.info()["last_tick_launches"]
    srv.close()
    return res


def test_alone_equals_mix_equals_batch(ppf):
    import torch
    rng = np.random.default_rng(3)
    A = Feed(ppf, 1024, 8, "c32", 1024 * 300 + 77, 11, 23)
    others = [Feed(ppf, 256, 16, "c32", 256 * 900 + 5, 21, 17), Feed(ppf, 4096, 16, "c32", 4096 * 60 + 999, 31, 9),
              Feed(ppf, 512, 4, "ci8", 512 * 500 + 3, 41, 13), Feed(ppf, 2048, 8, "c16", 2048 * 100 + 1, 51, 11),
              Feed(ppf, 64, 3, "c32", 64 * 700, 61, 7)]
    max_chunk = max(b - a for f in [A, *others] for a, b in f.bounds)
    # alone: A's chunks, one or two per tick
    sched_alone, i = [], 0
    while i < len(A.bounds):
        k = 1 + int(rng.integers(0, 4))
        sched_alone.append([(0, j) for j in range(i, min(i + k, len(A.bounds)))])
        i += k
    alone = _serve(ppf, [A], sched_alone, max_chunk)[0]
    # mix: every stream's chunks interleaved at random over ticks
    feeds = [A, *others]
    nxt = [0] * len(feeds)
    sched_mix = []
    while any(nxt[f] < len(feeds[f].bounds) for f in range(len(feeds))):
        tick = []
        for f in range(len(feeds)):
            k = int(rng.integers(0, 5))
            for _ in range(k):
                if nxt[f] < len(feeds[f].bounds):
                    tick.append((f, nxt[f]))
                    nxt[f] += 1
        sched_mix.append(tick)
    mixed = _serve(ppf, feeds, sched_mix, max_chunk)
    torch.cuda.synchronize()
    assert torch.equal(alone, mixed[0])
    A.check_oracle(alone)
    for f, got in zip(feeds, mixed):
        f.check_oracle(got)
    for f, got in zip(feeds, mixed):
        ref = f.batch_reference()
        torch.cuda.synchronize()
        assert got.shape == ref.shape
        assert torch.equal(got, ref), (f.N, f.T, f.dtype)


def test_admission_by_memory_and_slots(ppf):
    N, T = 1024, 8
    h = np.ones(N * T, np.float32)
    plan = ppf.Plan(N, T, h)
    chunk = 1 << 20
    per_slot = 2 * (8 * T * N + 4 * chunk + 2 * N) * 8
    srv = ppf.Server(max_streams=3, memory_budget_bytes=2 * per_slot + 100)
    a = srv.admit(plan, chunk)
    b = srv.admit(plan, chunk)
    with pytest.raises(ppf.PPFError) as e:
        srv.admit(plan, chunk)
    assert e.value.status == 4  # PPF_ERR_OUT_OF_MEMORY: budget exhausted
    srv.release(a)
    c = srv.admit(plan, chunk)
    assert srv.info()["streams"] == 2
    srv.close()
    srv = ppf.Server(max_streams=1, memory_budget_bytes=1 << 40)
    srv.admit(plan, 1024)
    with pytest.raises(ppf.PPFError) as e:
        srv.admit(plan, 1024)
    assert e.value.status == 7  # PPF_ERR_BUSY: no free slot
    srv.close()


def test_submit_errors(ppf):
    import torch
    N, T = 256, 4
    plan = ppf.Plan(N, T, np.ones(N * T, np.float32))
    srv = ppf.Server(max_streams=2, memory_budget_bytes=1 << 30)
    s = srv.admit(plan, 4 * N)
    x = torch.zeros(20 * N, dtype=torch.complex64, device="cuda")
    small = torch.empty((0, N), dtype=torch.complex64, device="cuda")
    assert srv.submit(s, x[:8 * N], small, 8 * N) == 1          # more than max_chunk
    assert srv.submit(s, x[:4 * N], small, 4 * N) == 1          # completes 1 spectrum, no room
    out = torch.empty((1, N), dtype=torch.complex64, device="cuda")
    assert srv.submit(s, x[:4 * N], out, 4 * N) == 0
    with pytest.raises(ppf.PPFError):
        srv.release(s)                                          # chunk still queued
    assert srv.tick() == 1
    srv.release(s)
    srv.close()


def test_tick_is_a_graph_replay(ppf):
    """Streams that all have a work-list kernel (every window that fits one SM
    on the mixed-shape kernel, N*T = 64K complex64 on its cluster kernel,
    int8 on its ring kernel): every tick replays the captured graph (gather
    copy, mixed kernel, the other groups' work lists, carry copy) with only
    the uploaded tables changing.  Each stream's spectra equal its own
    ppf_execute bitwise and the FP64 oracle within 1e-5."""
    import torch
    rng = np.random.default_rng(8)
    feeds = [Feed(ppf, 1024, 8, "c32", 1024 * 400 + 77, 111, 19), Feed(ppf, 256, 16, "c32", 256 * 900 + 5, 121, 15),
             Feed(ppf, 4096, 16, "c32", 4096 * 60 + 999, 131, 9), Feed(ppf, 512, 4, "ci8", 512 * 500 + 3, 141, 13),
             Feed(ppf, 128, 32, "c32", 128 * 2000 + 9, 151, 11), Feed(ppf, 2048, 4, "c32", 2048 * 150 + 1, 161, 7)]
    max_chunk = max(b - a for f in feeds for a, b in f.bounds)
    nxt = [0] * len(feeds)
    sched = []
    while any(nxt[f] < len(feeds[f].bounds) for f in range(len(feeds))):
        tick = []
        for f in range(len(feeds)):
            for _ in range(int(rng.integers(0, 4))):
                if nxt[f] < len(feeds[f].bounds):
                    tick.append((f, nxt[f]))
                    nxt[f] += 1
        sched.append(tick)
    stats = {}
    got = _serve(ppf, feeds, sched, max_chunk, stats)
    assert stats["graph_ticks"] == stats["ticks"], stats
    # gather copy, mixed kernel, cluster kernel group, int8 ring group, carry copy
    assert stats["launches"] == 5, stats
    for f, y in zip(feeds, got):
        f.check_oracle(y)
        ref = f.batch_reference()
        torch.cuda.synchronize()
        assert torch.equal(y, ref), (f.N, f.T, f.dtype)


def test_graph_recaptured_after_admit_and_release(ppf):
    """Releasing a stream and admitting another between ticks re-captures the
    graph; the streams that stay keep producing their exact spectra."""
    import torch
    A = Feed(ppf, 512, 8, "c32", 512 * 600 + 11, 171, 12)
    B = Feed(ppf, 1024, 16, "c32", 1024 * 200 + 3, 181, 6)
    C = Feed(ppf, 256, 4, "c32", 256 * 700 + 1, 191, 6)
    max_chunk = max(b - a for f in (A, B, C) for a, b in f.bounds)
    srv = ppf.Server(max_streams=4, memory_budget_bytes=8 << 30)
    sa, sb = srv.admit(A.plan, max_chunk), srv.admit(B.plan, max_chunk)
    outs = {0: [], 1: [], 2: []}
    keep = []

    def push(slot, f, i, key):
        c = f.chunk(i)
        k = srv.expected(slot, 0, c.shape[0])
        out = torch.empty((k, f.N), dtype=torch.complex64, device="cuda")
        assert srv.submit(slot, c, out) == 0
        outs[key].append(out)
        keep.append(c)

    for i in range(6):
        push(sa, A, i, 0)
        push(sb, B, i, 1)
        srv.tick()
    torch.cuda.synchronize()
    srv.release(sb)
    sc = srv.admit(C.plan, max_chunk)
    for i in range(6):
        push(sa, A, 6 + i, 0)
        push(sc, C, i, 2)
        srv.tick()
    torch.cuda.synchronize()
    assert srv.graph_ticks == 12
    srv.close()
    for key, f in ((0, A), (1, B), (2, C)):
        y = torch.cat(outs[key])
        ref = f.batch_reference()
        torch.cuda.synchronize()
        assert torch.equal(y, ref[: y.shape[0]]), (f.N, f.T)
        f.check_oracle(torch.cat([y, ref[y.shape[0]:]]))
