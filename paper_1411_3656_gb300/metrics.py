"""Throughput metrics of the polyphase filter bank (Section 3 of arXiv 1411.3656).

* Multiples of real time (Section 3, Eq. 2): M = (one second of data) / (time
  taken to process it).  With a batch of data worth ``data_seconds`` processed
  in ``elapsed_s``, M = data_seconds / elapsed_s.  M_c excludes host<->device
  transfers (data already in device memory), M_b includes them.
* The real-time rate is 6.5 GB/s (Section 1, Section 3); with complex64
  samples that is 8.125e8 samples per second.
* Algorithmic bytes of one fused launch: every input sample read once, every
  output written once, coefficients read once:
  (S+T-1)*N*in_bytes + S*N*8 + N*T*coef_bytes.
* Arithmetic per output sample: 4*T flops of FIR (a real coefficient times a
  complex sample is two multiply-adds) plus about 5*log2(N) flops of FFT.
"""
from __future__ import annotations

import math

REALTIME_BYTES_PER_S = 6.5e9
REALTIME_SAMPLES_PER_S = REALTIME_BYTES_PER_S / 8.0
IN_BYTES = {"c32": 8, "c16": 4, "ci8": 2}
COEF_BYTES = {"c32": 4, "c16": 2, "ci8": 2}


def realtime_multiple(data_seconds: float, elapsed_s: float) -> float:
    """Eq. 2: multiples of real time M = data_seconds / elapsed_s."""
    if elapsed_s <= 0:
        raise ValueError("elapsed time must be positive")
    return data_seconds / elapsed_s


def data_seconds(n_input_samples: int, samples_per_s: float = REALTIME_SAMPLES_PER_S) -> float:
    """Seconds of the 6.5 GB/s stream that n_input_samples complex samples represent."""
    return n_input_samples / samples_per_s


def algorithmic_bytes(N: int, T: int, S: int, dtype: str = "c32", out_bytes: int = 8) -> int:
    """Bytes one fused launch must move: input once, output once (8 bytes per
    complex64 bin, 4 for FP16 pairs), coefficients once."""
    if S <= 0:
        return 0
    return (S + T - 1) * N * IN_BYTES[dtype] + S * N * out_bytes + N * T * COEF_BYTES[dtype]


def flops(N: int, T: int, S: int) -> float:
    """Nominal flops: 4T (FIR) + 5 log2 N (FFT) per output sample."""
    return S * N * (4.0 * T + 5.0 * math.log2(N))


def pcie_gbs_single_mode(m_b: float, rate_gbs: float = 6.5) -> float:
    """Host-link traffic implied by M_b when output volume equals input volume: 2*rate*M_b."""
    return 2.0 * rate_gbs * m_b
