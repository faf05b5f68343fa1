"""Prototype filter design (Section 2: windowed, truncated sinc) against numpy.

ppf_design_coeffs is host code in the library; these tests load it without a
GPU.  numpy's window routines (np.hamming, np.kaiser, np.sinc) are independent
implementations of the same textbook definitions.
"""
import numpy as np
import pytest

from paper_1411_3656_gb300 import build, ppf, synth

INVALID = 1  # PPF_ERR_INVALID_ARG


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ppf.load()


def _numpy_design(N, T, window, beta):
    L = N * T
    n = np.arange(L, dtype=np.float64)
    w = np.hamming(L) if window == "hamming" else np.kaiser(L, beta)
    return np.sinc((n - (L - 1) / 2) / N) * w


@pytest.mark.parametrize("N,T", [(4, 1), (16, 4), (256, 8), (1024, 16), (4096, 32)])
@pytest.mark.parametrize("window,beta", [("hamming", 0.0), ("kaiser", 0.0), ("kaiser", 5.0), ("kaiser", 8.6)])
def test_matches_numpy_windows(lib, N, T, window, beta):
    h = ppf.ppf_design_coeffs(N, T, window, beta)
    ref = _numpy_design(N, T, window, beta)
    assert h.dtype == np.float32 and h.shape == (N * T,)
    # FP64 design rounded once to FP32: within one FP32 rounding of numpy's FP64 value
    np.testing.assert_allclose(h, ref, rtol=2e-7, atol=1e-12)


def test_hamming_matches_fixture(lib):
    np.testing.assert_allclose(ppf.ppf_design_coeffs(256, 8, "hamming"), synth.hamming_sinc(256, 8),
                               rtol=2e-7, atol=1e-12)


def test_kaiser_beta_zero_is_rectangular(lib):
    # I0(0) = 1: the Kaiser window with beta = 0 is the boxcar, leaving the bare sinc
    N, T = 64, 4
    n = np.arange(N * T)
    np.testing.assert_allclose(ppf.ppf_design_coeffs(N, T, "kaiser", 0.0),
                               np.sinc((n - (N * T - 1) / 2) / N), rtol=2e-7, atol=1e-12)


def test_symmetric_and_peak(lib):
    # the prototype is symmetric about (L-1)/2; with even L the two centre taps are the largest
    h = ppf.ppf_design_coeffs(128, 8, "kaiser", 8.0)
    np.testing.assert_array_equal(h, h[::-1])
    assert np.argmax(h) in (h.size // 2 - 1, h.size // 2)


def test_argument_errors(lib):
    import ctypes
    buf = (ctypes.c_float * 16)()
    f = lib.ppf_design_coeffs
    assert f(4, 4, 0, 0.0, None) == INVALID
    assert f(0, 4, 0, 0.0, buf) == INVALID
    assert f(4, 0, 0, 0.0, buf) == INVALID
    assert f(4, 4, 7, 0.0, buf) == INVALID
    assert f(4, 4, 1, -1.0, buf) == INVALID
    assert f(4, 4, 1, float("nan"), buf) == INVALID
    assert f(4, 4, 1, 8.0, buf) == 0
