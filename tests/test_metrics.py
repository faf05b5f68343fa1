"""Metric helpers against the numbers the paper prints (tests/golden)."""
import os

import pytest

from paper_1411_3656_gb300 import metrics

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_section3_metric.txt")


def _rows():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


def test_eq2_worked_example():
    (name, ds, el, want), = [r for r in _rows() if r[0] == "eq2_example"]
    assert metrics.realtime_multiple(float(ds), float(el)) == pytest.approx(float(want))


@pytest.mark.parametrize("row", [r for r in _rows() if r[0].startswith("table2_")], ids=lambda r: r[0])
def test_table2_link_usage(row):
    _, m_b, gbs = row
    assert abs(metrics.pcie_gbs_single_mode(float(m_b)) - float(gbs)) <= 0.06


def test_realtime_rate_and_bytes():
    assert metrics.REALTIME_SAMPLES_PER_S == 8.125e8
    # one second of complex64 at N=1024, T=8: S = floor(8.125e8/1024) - 7
    N, T = 1024, 8
    S = int(8.125e8) // N - T + 1
    b = metrics.algorithmic_bytes(N, T, S)
    assert b == (S + T - 1) * N * 8 + S * N * 8 + N * T * 4
    assert abs(b / 13.0e9 - 1) < 1e-3
    assert metrics.algorithmic_bytes(N, T, 0) == 0
    assert metrics.flops(256, 8, 1) == 256 * 72
