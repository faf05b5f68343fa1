"""The second CPU path (FIR + iterative radix-2 FFT) against the naive oracle,
numpy's FFT and every oracle pin; planted mistakes in a copy of it are caught.

It is pinned independently of the naive DFT: an O(N log N) transform built
from butterflies that reaches the O(N^2) definition to FP64 rounding (about
1e-13 relative L2 up to N = 4096) can only be the same transform.
"""
import os
import tempfile

import numpy as np
import pytest

import oracle
from tests import oracle_pins

SIZES = [4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096]
SRC2 = os.path.join(os.path.dirname(oracle.__file__), "ppf_cpu_radix2.c")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda p: p.__name__)
def test_radix2_passes_every_oracle_pin(pin):
    pin(oracle.radix2())


@pytest.mark.parametrize("N", SIZES)
def test_radix2_fft_equals_naive_dft(N):
    g = np.random.default_rng(N)
    y = g.standard_normal((7, N)) + 1j * g.standard_normal((7, N))
    got = oracle.radix2().dft(y, N)
    assert _rel(got, oracle.dft(y, N)) <= 1e-13
    assert _rel(got, np.fft.fft(y, axis=1)) <= 1e-13


@pytest.mark.parametrize("N,T,S", [(4, 3, 20), (64, 8, 17), (1024, 16, 5), (4096, 4, 3)])
def test_radix2_ppf_equals_oracle(N, T, S):
    g = np.random.default_rng(N + T)
    n = (S + T - 1) * N
    x = (g.standard_normal(n) + 1j * g.standard_normal(n)).astype(np.complex64)
    h = g.standard_normal(N * T).astype(np.float32)
    r2 = oracle.radix2()
    assert _rel(r2.ppf(x, h, N, T, S), oracle.ppf(x, h, N, T, S)) <= 1e-13
    assert np.array_equal(r2.fir(x, h, N, T, S), oracle.fir(x, h, N, T, S))
    rows = np.array([0, S // 2, S - 1])
    assert _rel(r2.ppf_rows(x, h, N, T, rows), oracle.ppf_rows(x, h, N, T, rows)) <= 1e-13


def test_radix2_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        oracle.radix2().dft(np.zeros((1, 12), np.complex128), 12)


MUTANTS = {
    "no_bit_reversal": ("if (i < j) {", "if (0) {"),
    "flipped_twiddle_sign": ("tw[2 * m + 1] = -sin(ang);", "tw[2 * m + 1] = sin(ang);"),
    "wrong_twiddle_step": ("const int half = L / 2, step = N / L;", "const int half = L / 2, step = N / half / 4;"),
    "swapped_butterfly_outputs": ("v[0] = u[0] - vr;", "v[0] = u[0] + vr;"),
}


def _caught(orc):
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(orc)
        except AssertionError:
            return True
    g = np.random.default_rng(1)
    for N in (8, 64, 512):
        y = g.standard_normal((3, N)) + 1j * g.standard_normal((3, N))
        if _rel(orc.dft(y, N), oracle.dft(y, N)) > 1e-13:
            return True
    return False


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_radix2_mutant_is_caught(name):
    old, new = MUTANTS[name]
    src = open(SRC2).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "mutant.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        lib = oracle._compile(path, os.path.join(d, "libmutant.so"))
        assert _caught(oracle.Radix2(lib)), f"nothing catches the planted mistake '{name}'"
