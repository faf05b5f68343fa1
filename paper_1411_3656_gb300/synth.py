"""Seeded synthetic inputs for the polyphase filter bank.

This module generates input data only.  It contains none of the filter-bank
arithmetic (no FIR, no DFT); the CUDA path and the CPU oracle both consume
what it produces, and neither shares any other code.

The inputs stand in for the paper's workload: a single-channel complex
voltage stream of the SKA Low Frequency Aperture Array at 6.5 GB/s
(Section 1 and Section 3).  Samples are complex64 (8 bytes), so one second of
data is 8.125e8 samples.  Values are Gaussian noise (I and Q independent
N(0, sigma^2)) plus unit-amplitude tones centred on DFT bins.

Every generator is deterministic in its seed and independent of the number
of worker threads: the stream is cut into fixed-size chunks and chunk i draws
from child i of the seed's ``numpy.random.SeedSequence``.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

#: 6.5 GB/s of complex64 samples, the paper's real-time rate (Section 1, Section 3).
REALTIME_BYTES_PER_S = 6.5e9
REALTIME_SAMPLES_PER_S = REALTIME_BYTES_PER_S / 8.0   # 8.125e8
BASE_SEED = 1411_3656
_CHUNK = 1 << 22


def _workers() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def complex_gaussian(n: int, seed: int, sigma: float = 1.0) -> np.ndarray:
    """n complex64 samples with I, Q ~ N(0, sigma^2), chunk-seeded."""
    n = int(n)
    out = np.empty(n, dtype=np.complex64)
    if n == 0:
        return out
    f = out.view(np.float32)
    nchunks = (n + _CHUNK - 1) // _CHUNK
    children = np.random.SeedSequence(seed).spawn(nchunks)

    def fill(i):
        lo = i * _CHUNK
        hi = min(n, lo + _CHUNK)
        g = np.random.Generator(np.random.PCG64(children[i]))
        v = g.standard_normal(2 * (hi - lo), dtype=np.float32)
        if sigma != 1.0:
            v *= np.float32(sigma)
        f[2 * lo:2 * hi] = v

    if nchunks == 1:
        fill(0)
    else:
        with ThreadPoolExecutor(_workers()) as ex:
            list(ex.map(fill, range(nchunks)))
    return out


def add_tones(x: np.ndarray, N: int, bins, amplitude: float = 1.0, start: int = 0) -> np.ndarray:
    """Add amplitude * exp(2*pi*i*k*n/N) for each bin k to complex64 ``x`` in place.

    The phase k*n mod N is reduced exactly in integers before the angle is
    formed, so the tone is exact at any stream length.  ``start`` is the
    global index of x[0].
    """
    n = x.shape[0]
    bins = [int(b) % N for b in bins]
    if n == 0 or not bins:
        return x
    # One period of each tone, then tile it: exp(2 pi i k n / N) has period N.
    idx = np.arange(N, dtype=np.int64)
    table = np.zeros(N, dtype=np.complex128)
    for k in bins:
        m = (k * idx) % N
        table += amplitude * np.exp(2j * np.pi * m / N)
    table64 = table.astype(np.complex64)
    nchunks = (n + _CHUNK - 1) // _CHUNK

    def fill(i):
        lo = i * _CHUNK
        hi = min(n, lo + _CHUNK)
        ph = (np.arange(lo, hi, dtype=np.int64) + start) % N
        x[lo:hi] += table64[ph]

    if nchunks == 1:
        fill(0)
    else:
        with ThreadPoolExecutor(_workers()) as ex:
            list(ex.map(fill, range(nchunks)))
    return x


def hamming_sinc(N: int, T: int) -> np.ndarray:
    """Prototype filter: sinc with cutoff 1/N, Hamming-windowed, float32 [N*T].

    The paper designs the coefficients as a sampled sinc (the inverse DFT of an
    ideal rectangular band), truncated and windowed (Section 2).  Length
    L = N*T, h[n] = sinc((n - (L-1)/2) / N) * (0.54 - 0.46*cos(2*pi*n/(L-1))),
    sinc(u) = sin(pi*u)/(pi*u), no normalisation.  Coefficient index n = t*N + c
    is tap t of channel c.
    """
    L = N * T
    n = np.arange(L, dtype=np.float64)
    u = (n - (L - 1) / 2.0) / N
    s = np.sinc(u)
    w = 0.54 - 0.46 * np.cos(2.0 * np.pi * n / (L - 1)) if L > 1 else np.ones(1)
    return (s * w).astype(np.float32)


def kaiser_sinc(N: int, T: int, beta: float = 8.0) -> np.ndarray:
    """Sinc prototype with the Kaiser window the paper names (Section 2), float32 [N*T].

    w[n] = I0(beta * sqrt(1 - (2n/(L-1) - 1)^2)) / I0(beta); ``beta`` is not
    given in the paper, 8.0 is a common choice for ~80 dB sidelobes.
    """
    L = N * T
    n = np.arange(L, dtype=np.float64)
    u = (n - (L - 1) / 2.0) / N
    s = np.sinc(u)
    if L > 1:
        r = 2.0 * n / (L - 1) - 1.0
        w = np.i0(beta * np.sqrt(np.clip(1.0 - r * r, 0.0, None))) / np.i0(beta)
    else:
        w = np.ones(1)
    return (s * w).astype(np.float32)


def tone_bins(N: int, count: int, seed: int) -> list[int]:
    """``count`` distinct seeded bins in [1, N)."""
    g = np.random.Generator(np.random.PCG64(seed))
    count = min(count, N - 1)
    return sorted(int(b) for b in g.choice(np.arange(1, N), size=count, replace=False))


def stream(n_samples: int, N: int, seed: int, n_tones: int = 3, sigma: float = 1.0) -> np.ndarray:
    """Gaussian noise plus ``n_tones`` unit tones at seeded bin centres, complex64."""
    x = complex_gaussian(n_samples, seed, sigma)
    add_tones(x, N, tone_bins(N, n_tones, seed + 7), 1.0)
    return x


def samples_for(n_spectra: int, N: int, T: int) -> int:
    """Input samples a batch of n_spectra spectra reads: (n_spectra + T - 1) * N."""
    return (int(n_spectra) + T - 1) * N if n_spectra > 0 else 0


def spectra_for(n_samples: int, N: int, T: int) -> int:
    """Complete spectra in a contiguous stream of n_samples: max(0, floor(n/N) - T + 1)."""
    return max(0, int(n_samples) // N - T + 1)


# -- the named workloads ------------------------------------------------------

def plain_config(seed: int = BASE_SEED + 1):
    """Plain PPF: N=256, T=8, 1024 spectra, complex64 noise + 3 bin-centred tones.

    Returns (x complex64[(1024+7)*256], h float32[2048], N, T, S).
    """
    N, T, S = 256, 8, 1024
    x = stream(samples_for(S, N, T), N, seed, n_tones=3)
    return x, hamming_sinc(N, T), N, T, S


def realtime_second_config(N: int, T: int, seconds: float = 1.0, seed: int = BASE_SEED + 2):
    """One SKA-LFAA-like stream: ``seconds`` of 6.5 GB/s complex64 at (N, T).

    S = floor(8.125e8 * seconds / N) - T + 1 spectra; the input holds exactly
    (S + T - 1) * N samples.  Returns (x, h, N, T, S).
    """
    n_total = int(REALTIME_SAMPLES_PER_S * seconds)
    S = spectra_for(n_total, N, T)
    x = stream(samples_for(S, N, T), N, seed + 97 * N + T, n_tones=3)
    return x, hamming_sinc(N, T), N, T, S


def to_fp16_iq(x: np.ndarray) -> np.ndarray:
    """Store complex64 samples as float16 (I, Q) pairs: float16 [n, 2]."""
    return x.view(np.float32).reshape(-1, 2).astype(np.float16)


def int8_iq(n_samples: int, seed: int, sigma: float = 20.0) -> np.ndarray:
    """int8 (I, Q) pairs: clip(round(N(0, sigma^2)), -127, 127), int8 [n, 2]."""
    g = complex_gaussian(n_samples, seed, sigma).view(np.float32).reshape(-1, 2)
    return np.clip(np.rint(g), -127, 127).astype(np.int8)


def sample_rows(S: int, count: int = 1024, seed: int = BASE_SEED + 5, edge: int = 8) -> np.ndarray:
    """Spectra to check at full size: the first and last ``edge`` plus ``count`` seeded."""
    S = int(S)
    if S <= 2 * edge + count:
        return np.arange(S, dtype=np.int64)
    g = np.random.Generator(np.random.PCG64(seed))
    mid = g.choice(np.arange(edge, S - edge), size=count, replace=False)
    rows = np.concatenate([np.arange(edge), np.sort(mid), np.arange(S - edge, S)])
    return rows.astype(np.int64)


def rel_l2(a, b) -> float:
    """Relative L2 error ||a - b|| / ||b|| in FP64 (0 when both are empty or zero)."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    den = float(np.sqrt(np.sum(np.abs(b) ** 2)))
    num = float(np.sqrt(np.sum(np.abs(a - b) ** 2)))
    if den == 0.0:
        return num
    return num / den



def worst_spectrum_rel_l2(a, b) -> float:
    """Largest per-spectrum relative L2 error over the rows of [S, N] arrays
    (each row's ||a_s - b_s|| / ||b_s||; rows with ||b_s|| = 0 count their
    absolute error).  A diagnostic beside the whole-array figure."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    if a.size == 0:
        return 0.0
    a = a.reshape(-1, a.shape[-1])
    b = b.reshape(-1, b.shape[-1])
    num = np.sqrt(np.sum(np.abs(a - b) ** 2, axis=1))
    den = np.sqrt(np.sum(np.abs(b) ** 2, axis=1))
    return float(np.max(np.where(den > 0, num / np.where(den > 0, den, 1.0), num)))
