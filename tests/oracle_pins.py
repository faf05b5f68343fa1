"""Pins for the FP64 oracle: facts fixed by the paper and by mathematics.

Each pin takes an oracle-like object with ``fir(x, h, N, T, n)`` and
``ppf(x, h, N, T, n)`` (see ``oracle``) and raises AssertionError when the
oracle disagrees.  They are written so that a plausible mistake anywhere in
the oracle (a dropped tap, a reversed or transposed index, a wrong DFT sign
or a wrong angle) fails at least one of them; ``test_oracle_mutants`` plants
exactly such mistakes in a copy of the oracle and checks that it does.

None of the expected values comes from the oracle itself.
"""
from __future__ import annotations

import numpy as np


def _rand_h(N, T, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(N * T).astype(np.float32)


def _rand_x(n, seed):
    g = np.random.default_rng(seed)
    return (g.standard_normal(n) + 1j * g.standard_normal(n)).astype(np.complex64)


def pin_impulse(orc, N=16, T=4, S=12, atol=1e-12):
    """Impulse response reproduces h (Eq. 1: the response of a FIR to a pulse is its coefficients).

    x = delta at sample m = r*N + c0.  Then spectrum s sees the pulse in tap
    t = r - s of channel c0, so Y[s][k] = h[(r-s)*N + c0] * exp(-2*pi*i*k*c0/N)
    for r-T+1 <= s <= r and 0 elsewhere.  Sweeping c0 recovers every tap of
    every channel, which also fixes which end of h weights the oldest row.
    """
    h = _rand_h(N, T, 11)
    k = np.arange(N)
    for r, c0 in [(T - 1, 0), (T + 2, 3), (S - 1, N - 1), (T, N // 2 + 1), (0, 5 % N)]:
        x = np.zeros((S + T - 1) * N, dtype=np.complex64)
        x[r * N + c0] = 1.0
        Y = orc.ppf(x, h, N, T, S)
        want = np.zeros((S, N), dtype=np.complex128)
        for s in range(S):
            t = r - s
            if 0 <= t < T:
                want[s] = float(h[t * N + c0]) * np.exp(-2j * np.pi * k * c0 / N)
        assert np.allclose(Y, want, rtol=0, atol=atol), f"impulse at r={r}, c0={c0}"


def pin_tone_boxcar(orc, N=32, T=4, S=5):
    """A bin-centred tone through an all-ones filter lands entirely in its bin.

    x[n] = exp(2*pi*i*k0*n/N) gives y[s][c] = T*exp(2*pi*i*k0*c/N) for every
    s, whose forward DFT is T*N at k = k0 and exactly 0 elsewhere (the
    bandpass role of the PPF, Section 2; forward sign convention).
    """
    h = np.ones(N * T, dtype=np.float32)
    for k0 in (0, 1, 5, N - 3):
        n = np.arange((S + T - 1) * N)
        x = np.exp(2j * np.pi * ((k0 * n) % N) / N)
        Y = orc.ppf(x, h, N, T, S)
        want = np.zeros((S, N), dtype=np.complex128)
        want[:, k0] = T * N
        assert np.allclose(Y, want, rtol=0, atol=1e-9 * T * N), f"boxcar tone k0={k0}"


def pin_tone_general(orc, N=64, T=8, S=6):
    """Bin-centred tone with a general filter: closed form via the channel gains.

    y[s][c] = H_c * exp(2*pi*i*k0*c/N) with H_c = sum_t h[t*N + c], so
    Y[s][k] = sum_c H_c * exp(-2*pi*i*(k-k0)*c/N) = DFT(H)[(k - k0) mod N],
    the same for every s.  DFT(H) is taken from numpy.fft, not the oracle.
    """
    h = _rand_h(N, T, 23)
    H = h.astype(np.float64).reshape(T, N).sum(axis=0)
    FH = np.fft.fft(H)
    for k0 in (3, N // 2 + 7):
        n = np.arange((S + T - 1) * N)
        x = np.exp(2j * np.pi * ((k0 * n) % N) / N)
        Y = orc.ppf(x, h, N, T, S)
        want = FH[(np.arange(N) - k0) % N]
        assert np.allclose(Y, np.broadcast_to(want, Y.shape), rtol=0, atol=1e-10 * np.abs(FH).max())


def pin_linearity(orc, N=32, T=5, S=9):
    """The PPF is linear (Section 2: a linear filter followed by a DFT)."""
    h = _rand_h(N, T, 31)
    x1 = _rand_x((S + T - 1) * N, 1)
    x2 = _rand_x((S + T - 1) * N, 2)
    a, b = 0.75 - 0.5j, -1.25 + 2.0j
    lhs = orc.ppf(a * x1.astype(np.complex128) + b * x2.astype(np.complex128), h, N, T, S)
    rhs = a * orc.ppf(x1, h, N, T, S) + b * orc.ppf(x2, h, N, T, S)
    assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-11)


def pin_parseval(orc, N=64, T=4, S=7):
    """Parseval on the DFT stage: sum_k |Y[s][k]|^2 = N * sum_c |y[s][c]|^2."""
    h = _rand_h(N, T, 41)
    x = _rand_x((S + T - 1) * N, 3)
    y = orc.fir(x, h, N, T, S)
    Y = orc.ppf(x, h, N, T, S)
    lhs = np.sum(np.abs(Y) ** 2, axis=1)
    rhs = N * np.sum(np.abs(y) ** 2, axis=1)
    assert np.allclose(lhs, rhs, rtol=1e-12)


def pin_fir_direct(orc, N=8, T=3, S=5):
    """FIR stage against Eq. 1 evaluated per output sample of each channel.

    Channel c sees the sub-stream u_c[m] = x[m*N + c].  Eq. 1 with T taps
    b_i gives v_c[n] = sum_i u_c[n-i] b_i; our convention is b_i = h[(T-1-i)*N + c]
    and y[s][c] = v_c[s + T - 1].  Evaluated with numpy.convolve (a library
    routine for Eq. 1), one channel at a time.
    """
    h = _rand_h(N, T, 53)
    x = _rand_x((S + T - 1) * N, 4)
    y = orc.fir(x, h, N, T, S)
    for c in range(N):
        u = x[c::N].astype(np.complex128)
        b = np.array([h[(T - 1 - i) * N + c] for i in range(T)], dtype=np.float64)
        v = np.convolve(u, b)            # v[n] = sum_i u[n-i] b[i]
        assert np.allclose(y[:, c], v[T - 1:T - 1 + S], rtol=1e-12, atol=1e-12), f"channel {c}"


def pin_t1_blockwise_fft(orc, N=128, S=6):
    """T = 1, h = 1: the PPF reduces to a blockwise forward FFT (numpy.fft)."""
    h = np.ones(N, dtype=np.float32)
    x = _rand_x(S * N, 5)
    Y = orc.ppf(x, h, N, 1, S)
    want = np.fft.fft(x.astype(np.complex128).reshape(S, N), axis=1)
    assert np.allclose(Y, want, rtol=1e-12, atol=1e-10)


# exact 4-point DFT matrix: W_4^m = exp(-2*pi*i*m/4) = 1, -i, -1, i
_W4 = [1, -1j, -1, 1j]


def pin_exact_n4(orc):
    """Gaussian-integer inputs, N = 4, T = 2: the result is exact integers.

    The 4-point forward DFT has entries W^m in {1, -i, -1, i}, so with integer
    h and Gaussian-integer x every output is a Gaussian integer, computed here
    in exact Python integer arithmetic by the defining double sum.
    """
    N, T, S = 4, 2, 3
    h = [2, -1, 3, 1, 1, 4, -2, 5]            # h[t*N + c]
    xs = [complex(a, b) for a, b in [(1, 0), (0, 2), (-3, 1), (2, 2), (1, -1), (4, 0), (0, -2),
                                        (3, 3), (-1, 1), (2, -3), (1, 1), (0, 0), (5, -1), (-2, 2),
                                        (1, 4), (3, -2)]]
    want = np.zeros((S, N), dtype=np.complex128)
    for s in range(S):
        y = [sum(h[t * N + c] * xs[(s + t) * N + c] for t in range(T)) for c in range(N)]
        for k in range(N):
            want[s, k] = sum(y[c] * _W4[(k * c) % 4] for c in range(N))
    Y = orc.ppf(np.array(xs, dtype=np.complex64), np.array(h, dtype=np.float32), N, T, S)
    assert np.allclose(Y, want, rtol=0, atol=1e-12), (Y, want)


def pin_brute_small(orc):
    """Brute force at N <= 16: the defining triple sum, evaluated term by term."""
    for N, T, S in [(2, 1, 3), (4, 3, 4), (8, 2, 5), (16, 4, 3), (16, 1, 2)]:
        h = _rand_h(N, T, 60 + N)
        x = _rand_x((S + T - 1) * N, 70 + N)
        Y = orc.ppf(x, h, N, T, S)
        for s in range(S):
            for k in range(N):
                acc = 0j
                for t in range(T):
                    for c in range(N):
                        acc += float(h[t * N + c]) * complex(x[(s + t) * N + c]) * \
                            np.exp(-2j * np.pi * k * c / N)
                assert abs(Y[s, k] - acc) <= 1e-12 * max(1.0, abs(acc)), (N, T, s, k)


ALL_PINS = [pin_impulse, pin_tone_boxcar, pin_tone_general, pin_linearity, pin_parseval,
            pin_fir_direct, pin_t1_blockwise_fft, pin_exact_n4, pin_brute_small]
