"""Real-time serving driver for many PPF streams on one GPU.

Each stream is one sensor channel producing complex samples at the paper's
real-time rate, 6.5 GB/s (Section 1, Section 3): 8.125e8 complex64 samples per
second.  Chunks of ``chunk_ms`` milliseconds of data arrive as a Poisson
process with mean inter-arrival time ``chunk_ms``, so every stream averages
the real-time rate.  The driver runs in wall-clock time: whatever has arrived
is submitted to a :class:`~paper_1411_3656_gb300.ppf.Server` and one tick runs
it all (continuous batching).  A chunk's latency is the time from its arrival
to the completion of the tick that processed it (CUDA events on the serving
stream, aligned to the host clock by an event recorded at start).

The sample data are synthetic and resident in device memory before the run
(a pool the chunks point into), so the measurement is the paper's streaming
mode M_c: no host-device transfer inside the loop.
"""
from __future__ import annotations

import gc
import time

import numpy as np

REALTIME_SAMPLES_PER_S = 8.125e8


def poisson_arrivals(n_streams: int, chunk_ms: float, duration_s: float, seed: int):
    """Sorted (time_s, stream) arrivals: per stream, exponential gaps of mean chunk_ms."""
    g = np.random.default_rng(seed)
    out = []
    mean = chunk_ms / 1e3
    for s in range(n_streams):
        t = g.exponential(mean)
        while t < duration_s:
            out.append((t, s))
            t += g.exponential(mean)
    out.sort()
    return out


# chunks are drawn from a device pool at least four times the 129 MB L2, so
# a chunk's samples come from HBM, not from lines an earlier chunk left in L2
L2_BYTES = 129 * 2**20
POOL_MIN_BYTES = 4 * L2_BYTES


def run(n_streams: int, chunk_ms: float, shapes, dtype: str = "c32", duration_s: float = 10.0,
        warmup_s: float = 0.3, seed: int = 1411_3656, memory_budget: int | None = None,
        pool_bytes: int = POOL_MIN_BYTES):
    """Serve ``n_streams`` real-time streams for ``duration_s`` seconds.

    ``shapes`` is a list of (N, T); stream i uses shapes[i % len(shapes)].
    Chunks point at random 64-byte-aligned offsets of a device pool of at
    least ``pool_bytes`` (default four times L2).
    Returns a dict with chunk latency percentiles, throughput, backlog and
    whether the run was sustained: every stream admitted and p99 latency
    <= chunk_ms (chunks a full stream buffer defers are retried next tick
    and keep their arrival time, so a growing backlog shows as latency).
    """
    import torch

    from . import ppf, synth

    dev = torch.device("cuda")
    chunk = int(round(REALTIME_SAMPLES_PER_S * chunk_ms / 1e3))
    bps = ppf.SAMPLE_BYTES[dtype]
    plans = {}
    for N, T in set(shapes):
        plans[(N, T)] = ppf.Plan(N, T, synth.hamming_sinc(N, T), dtype)
    free, total = torch.cuda.mem_get_info()
    budget = memory_budget if memory_budget is not None else int(0.6 * free)
    srv = ppf.Server(max_streams=n_streams, memory_budget_bytes=budget)
    # device-resident sample pool (contents do not affect timing), larger
    # than L2 so that chunk reads come from HBM
    pool_samples = max(4 * chunk + (1 << 20), -(-int(pool_bytes) // bps))
    if dtype == "c32":
        pool = torch.randn(pool_samples, dtype=torch.complex64, device=dev)
    elif dtype == "c16":
        pool = torch.randn(pool_samples, 2, dtype=torch.float16, device=dev)
    else:
        pool = torch.randint(-100, 100, (pool_samples, 2), dtype=torch.int8, device=dev)
    slots, outs, shp = [], [], []
    bps = ppf.SAMPLE_BYTES[dtype]
    refused_admission = 0
    for i in range(n_streams):
        N, T = shapes[i % len(shapes)]
        try:
            slots.append(srv.admit(plans[(N, T)], chunk))
        except ppf.PPFError:
            refused_admission += 1
            continue
        shp.append((N, T))
        # output ring: room for two chunks' spectra
        outs.append(torch.empty((2 * (chunk // N + 2), N), dtype=torch.complex64, device=dev))
    n_live = len(slots)
    arrivals = poisson_arrivals(n_live, chunk_ms, warmup_s + duration_s, seed)
    arr_t = np.array([a[0] for a in arrivals])
    arr_s = np.array([a[1] for a in arrivals], dtype=np.int64)
    Ns = np.array([n for n, _ in shp], dtype=np.int64)
    Ts = np.array([t for _, t in shp], dtype=np.int64)
    slot_arr = np.array(slots, dtype=np.int32)
    out_base = np.array([o.data_ptr() for o in outs], dtype=np.uint64)
    out_rows = np.array([o.shape[0] // 2 for o in outs], dtype=np.int64)
    pushed = np.zeros(n_live, dtype=np.int64)
    half = np.zeros(n_live, dtype=np.int64)
    pool_ptr = pool.data_ptr()
    stream = torch.cuda.current_stream(dev)
    rng = np.random.default_rng(seed + 1)
    start_ev = torch.cuda.Event(enable_timing=True)
    start_ev.record(stream)
    torch.cuda.synchronize()
    gc_was = gc.isenabled()
    gc.disable()   # no collector pauses inside the real-time loop
    t0 = time.perf_counter()
    pending_events = []   # (event, arrival times of the chunks it completes)
    latencies = []
    refused = 0
    ai = 0
    ticks = 0
    n_arr = len(arrivals)
    host_tick_s = 0.0
    tick_events = []
    chunks_per_tick = []
    back_s = np.zeros(0, dtype=np.int64)   # chunks a full stream buffer refused: retried next tick
    back_t = np.zeros(0)
    max_backlog = 0
    while ai < n_arr or back_s.size:
        now = time.perf_counter() - t0
        hi = int(np.searchsorted(arr_t, now, side="right"))
        if hi <= ai and not back_s.size:
            _retire(pending_events, start_ev, latencies, warmup_s, block=False)
            continue
        s_idx = np.concatenate([back_s, arr_s[ai:hi]])
        t_idx = np.concatenate([back_t, arr_t[ai:hi]])
        ai = max(ai, hi)
        offs = rng.integers(0, (pool_samples - chunk) // 8, size=s_idx.shape[0]) * 8
        chunk_ptrs = pool_ptr + offs.astype(np.uint64) * np.uint64(bps)
        outp = out_base[s_idx] + (half[s_idx] * out_rows[s_idx] * Ns[s_idx] * 8).astype(np.uint64)
        caps = out_rows[s_idx]
        st = srv.submit_many(slot_arr[s_idx], chunk_ptrs, np.full(s_idx.shape[0], chunk, np.int64), outp, caps)
        ok = st == 0
        np.bitwise_xor.at(half, s_idx[ok], 1)
        back_s, back_t = s_idx[~ok], t_idx[~ok]
        max_backlog = max(max_backlog, int(back_s.size))
        refused += int((~ok).sum())
        np.add.at(pushed, s_idx[ok], chunk)
        if ok.any():
            th = time.perf_counter()
            srv.tick(stream)
            host_tick_s += time.perf_counter() - th
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            pending_events.append((ev, t_idx[ok]))
            tick_events.append(ev)
            chunks_per_tick.append(int(ok.sum()))
            ticks += 1
        _retire(pending_events, start_ev, latencies, warmup_s, block=False)
    _retire(pending_events, start_ev, latencies, warmup_s, block=True)
    wall = time.perf_counter() - t0
    if gc_was:
        gc.enable()
    gaps = [tick_events[i - 1].elapsed_time(tick_events[i]) for i in range(1, len(tick_events))]
    lat = np.concatenate(latencies) * 1e3 if latencies else np.array([np.nan])
    measured = int(lat.shape[0]) if latencies else 0
    info = srv.info()
    srv.close()
    samples = measured * chunk
    p99 = float(np.percentile(lat, 99))
    return {
        "streams": n_streams, "admitted": n_live, "refused_admission": refused_admission,
        "chunk_ms": chunk_ms, "chunk_samples": chunk, "dtype": dtype,
        "chunks": measured, "deferred_chunks": refused, "max_backlog": max_backlog, "ticks": ticks,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": p99, "max_ms": float(np.max(lat)),
        "Msamples_s": samples / duration_s / 1e6,
        "x_realtime_total": samples / duration_s / REALTIME_SAMPLES_PER_S,
        "sustained": bool(refused_admission == 0 and p99 <= chunk_ms),
        "wall_s": wall, "reserved_GB": info["reserved_bytes"] / 1e9,
        "in_bytes_per_sample": bps, "pool_GB": pool_samples * bps / 1e9, "duration_s": duration_s,
        "host_ms_per_tick": 1e3 * host_tick_s / max(1, ticks),
        "gpu_ms_between_ticks_p50": float(np.percentile(gaps, 50)) if gaps else None,
        "chunks_per_tick_mean": float(np.mean(chunks_per_tick)) if chunks_per_tick else 0.0,
    }


def _retire(pending, start_ev, latencies, warmup_s, block):
    """Record latencies of completed ticks (arrival -> tick completion)."""
    while pending:
        ev, arr = pending[0]
        if not block and not ev.query():
            return
        ev.synchronize()
        done_s = start_ev.elapsed_time(ev) / 1e3
        arr = np.asarray(arr)
        arr = arr[arr >= warmup_s]
        if arr.size:
            latencies.append(done_s - arr)
        pending.pop(0)


__all__ = ["run", "poisson_arrivals", "REALTIME_SAMPLES_PER_S"]
