"""The FP64 oracle against facts fixed by the paper and by mathematics."""
import numpy as np
import pytest

import oracle
from tests import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin):
    pin(oracle.default())


def test_rows_equals_contiguous():
    """Gathered windows give the same spectra as the contiguous stream."""
    g = np.random.default_rng(9)
    N, T, S = 32, 6, 40
    x = (g.standard_normal((S + T - 1) * N) + 1j * g.standard_normal((S + T - 1) * N)).astype(np.complex64)
    h = g.standard_normal(N * T).astype(np.float32)
    full = oracle.ppf(x, h, N, T, S)
    rows = np.array([0, 3, 17, S - 1])
    assert np.array_equal(oracle.ppf_rows(x, h, N, T, rows), full[rows])


def test_stored_int8_and_fp16_exact():
    """Stored int8 / float16 I/Q pairs are read exactly (no rounding in the oracle)."""
    g = np.random.default_rng(3)
    N, T, S = 16, 3, 5
    n = (S + T - 1) * N
    q = np.clip(np.rint(g.standard_normal((n, 2)) * 20), -127, 127).astype(np.int8)
    h = g.standard_normal(N * T).astype(np.float32)
    as_c = q[:, 0].astype(np.float64) + 1j * q[:, 1].astype(np.float64)
    assert np.array_equal(oracle.ppf(q, h, N, T, S), oracle.ppf(as_c, h, N, T, S))
    f16 = g.standard_normal((n, 2)).astype(np.float16)
    as_c = f16[:, 0].astype(np.float64) + 1j * f16[:, 1].astype(np.float64)
    assert np.array_equal(oracle.ppf(f16, h, N, T, S), oracle.ppf(as_c, h, N, T, S))


def test_invalid_arguments():
    with pytest.raises(ValueError):
        oracle.ppf(np.zeros(10, np.complex64), np.ones(3, np.float32), 4, 2, 5)
