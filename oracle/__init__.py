"""FP64 CPU oracle for the polyphase filter bank (arXiv 1411.3656).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
library never loads it and has no CPU fallback.

The arithmetic lives in ``ppf_oracle.c`` (plain C, FP64, OpenMP over spectra):

* FIR stage, Section 2 Eq. 1 in the loop order of Algorithm 1, with the index
  convention y[s][c] = sum_t h[t*N+c] * x[(s+t)*N+c];
* DFT stage, a naive O(N^2) forward DFT, unnormalised, natural bin order
  (Section 3: the DFT is a standard library FFT).

A second, independent CPU path lives in ``ppf_cpu_radix2.c`` (its own
library): the same FIR followed by an iterative radix-2 FFT.  It is pinned to
the naive DFT (FP64 rounding, ~1e-13) and to every oracle pin, and it is the
faster CPU baseline, standing in for the paper's CPU code with a library FFT
(Section 3).  ``radix2()`` returns it with the same methods as the oracle.

Inputs are converted exactly to FP64 from the values as stored (float32,
float16, int8 and float32 coefficients are all exactly representable), so the
oracle sees precisely what the GPU path sees.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppf_oracle.c")
_LIB = os.path.join(_HERE, "libppf_oracle.so")
_SRC2 = os.path.join(_HERE, "ppf_cpu_radix2.c")
_LIB2 = os.path.join(_HERE, "libppf_cpu_radix2.so")
_lock = threading.Lock()
_default = None
_radix2 = None


def _compile(src: str, out: str) -> str:
    base = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC", "-std=c11"]
    tmp = out + f".{os.getpid()}.tmp"
    try:
        subprocess.run(base + ["-fopenmp", src, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        # No OpenMP runtime: the oracle is still correct, just single-threaded.
        subprocess.run(base + [src, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``ppf_oracle.c`` into ``libppf_oracle.so`` and ``ppf_cpu_radix2.c``
    into ``libppf_cpu_radix2.so`` (gcc -O2, no fast-math, no FMA contraction)."""
    for src, lib in ((_SRC2, _LIB2), (_SRC, _LIB)):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(src):
            _compile(src, lib)
    return _LIB


def to_complex128(x) -> np.ndarray:
    """Exact conversion of stored samples to complex128.

    Accepts complex64/complex128 arrays, or real arrays whose last axis holds
    (I, Q) pairs (float16 or int8 storage).
    """
    x = np.asarray(x)
    if np.iscomplexobj(x):
        return np.ascontiguousarray(x, dtype=np.complex128)
    if x.shape[-1] != 2:
        raise ValueError("real input must have a trailing (I, Q) axis of length 2")
    xd = x.astype(np.float64)
    return np.ascontiguousarray(xd[..., 0] + 1j * xd[..., 1])


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _prep(x, h, N, T, n_spectra, window_stride):
    xc = to_complex128(x).reshape(-1)
    hd = np.ascontiguousarray(np.asarray(h, dtype=np.float32).astype(np.float64).reshape(-1))
    if hd.size != N * T:
        raise ValueError("h must hold N*T coefficients")
    stride = N if window_stride is None else int(window_stride)
    if n_spectra is None:
        n_spectra = (xc.size - T * N) // stride + 1 if xc.size >= T * N else 0
    n_spectra = int(n_spectra)
    if n_spectra > 0 and (n_spectra - 1) * stride + T * N > xc.size:
        raise ValueError("input too short for the requested spectra")
    return xc, hd, stride, max(n_spectra, 0)


class Oracle:
    """ctypes view of one compiled oracle library."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        dp = ctypes.POINTER(ctypes.c_double)
        for name in ("ppf_oracle_fir", "ppf_oracle_ppf"):
            fn = getattr(lib, name)
            fn.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, dp]
            fn.restype = ctypes.c_int
        lib.ppf_oracle_dft.argtypes = [dp, ctypes.c_int, ctypes.c_int64, dp]
        lib.ppf_oracle_dft.restype = ctypes.c_int
        lib.ppf_oracle_threads.argtypes = []
        lib.ppf_oracle_threads.restype = ctypes.c_int
        self.lib = lib

    def threads(self) -> int:
        return int(self.lib.ppf_oracle_threads())

    def fir(self, x, h, N, T, n_spectra=None, window_stride=None):
        """FIR stage (Eq. 1 / Algorithm 1) -> complex128 [n_spectra, N]."""
        xc, hd, stride, n = _prep(x, h, N, T, n_spectra, window_stride)
        y = np.empty((n, N), dtype=np.complex128)
        if n and self.lib.ppf_oracle_fir(_dptr(xc.view(np.float64)), stride, _dptr(hd), N, T, n,
                                         _dptr(y.view(np.float64))) != 0:
            raise ValueError("ppf_oracle_fir: invalid arguments")
        return y

    def dft(self, y, N):
        """Naive forward DFT of each row -> complex128 [rows, N]."""
        yc = np.ascontiguousarray(np.asarray(y, dtype=np.complex128).reshape(-1, N))
        Y = np.empty_like(yc)
        if yc.shape[0] and self.lib.ppf_oracle_dft(_dptr(yc.view(np.float64)), N, yc.shape[0],
                                                   _dptr(Y.view(np.float64))) != 0:
            raise ValueError("ppf_oracle_dft: invalid arguments")
        return Y

    def ppf(self, x, h, N, T, n_spectra=None, window_stride=None):
        """Whole PPF (FIR then DFT) -> complex128 [n_spectra, N]."""
        xc, hd, stride, n = _prep(x, h, N, T, n_spectra, window_stride)
        Y = np.empty((n, N), dtype=np.complex128)
        if n and self.lib.ppf_oracle_ppf(_dptr(xc.view(np.float64)), stride, _dptr(hd), N, T, n,
                                         _dptr(Y.view(np.float64))) != 0:
            raise ValueError("ppf_oracle_ppf: invalid arguments")
        return Y

    def ppf_rows(self, x_stored, h, N, T, rows):
        """PPF of selected spectra ``rows`` of a contiguous stored input stream.

        Only the T input rows each spectrum reads are converted, so this works
        on inputs far larger than host FP64 memory would allow.  ``x_stored`` is
        the stored stream (complex64 1-D, or [..., 2] float16/int8 I/Q pairs).
        """
        rows = np.asarray(rows, dtype=np.int64).reshape(-1)
        xs = np.asarray(x_stored)
        flat = xs.reshape(-1) if np.iscomplexobj(xs) else xs.reshape(-1, 2)
        if rows.size == 0:
            return np.empty((0, N), dtype=np.complex128)
        windows = np.stack([flat[r * N:(r + T) * N] for r in rows])
        return self.ppf(windows, h, N, T, n_spectra=rows.size, window_stride=T * N)


class Radix2(Oracle):
    """ctypes view of the second CPU path (FIR + iterative radix-2 FFT)."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        dp = ctypes.POINTER(ctypes.c_double)
        for name in ("ppf_cpu2_fir", "ppf_cpu2_ppf"):
            fn = getattr(lib, name)
            fn.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int64, dp]
            fn.restype = ctypes.c_int
        lib.ppf_cpu2_fft.argtypes = [dp, ctypes.c_int, ctypes.c_int64, dp]
        lib.ppf_cpu2_fft.restype = ctypes.c_int
        lib.ppf_cpu2_threads.argtypes = []
        lib.ppf_cpu2_threads.restype = ctypes.c_int
        # the oracle's method names, bound to this library's functions
        lib.ppf_oracle_fir = lib.ppf_cpu2_fir
        lib.ppf_oracle_ppf = lib.ppf_cpu2_ppf
        lib.ppf_oracle_dft = lib.ppf_cpu2_fft
        lib.ppf_oracle_threads = lib.ppf_cpu2_threads
        self.lib = lib


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def radix2() -> Radix2:
    """The second CPU path (FIR + radix-2 FFT), with the oracle's methods."""
    global _radix2
    with _lock:
        if _radix2 is None:
            build()
            _radix2 = Radix2(_LIB2)
    return _radix2


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return default().threads()


def fir(x, h, N, T, n_spectra=None, window_stride=None):
    return default().fir(x, h, N, T, n_spectra, window_stride)


def dft(y, N):
    return default().dft(y, N)


def ppf(x, h, N, T, n_spectra=None, window_stride=None):
    return default().ppf(x, h, N, T, n_spectra, window_stride)


def ppf_rows(x_stored, h, N, T, rows):
    return default().ppf_rows(x_stored, h, N, T, rows)
