"""Planted mistakes in a copy of the oracle must fail at least one pin.

Each mutant is the oracle's C source with one plausible error planted (a
dropped tap, a reversed tap order, a transposed coefficient index, a flipped
DFT sign, a wrong angle index, a dropped cross term).  It is compiled into a
temporary library on the CPU and run through every pin; a mutant that passes
all pins would mean the pins cannot tell a wrong oracle from the right one.
"""
import os
import tempfile

import pytest

import oracle
from tests import oracle_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "ppf_oracle.c")

MUTANTS = {
    "dropped_last_tap": ("for (int t = 0; t < T; ++t) {", "for (int t = 0; t < T - 1; ++t) {"),
    "reversed_taps": ("xw + 2 * ((int64_t)t * N + c)", "xw + 2 * ((int64_t)(T - 1 - t) * N + c)"),
    "transposed_h": ("h[(int64_t)t * N + c]", "h[(int64_t)c * T + t]"),
    "flipped_dft_sign": ("re += yw[2 * c] * cr + yw[2 * c + 1] * si;\n                im += yw[2 * c + 1] * cr - yw[2 * c] * si;",
                         "re += yw[2 * c] * cr - yw[2 * c + 1] * si;\n                im += yw[2 * c + 1] * cr + yw[2 * c] * si;"),
    "wrong_angle_index": ("(((int64_t)k * c) % N)", "(((int64_t)k * (c + 1)) % N)"),
    "dropped_cross_term": ("im += yw[2 * c + 1] * cr - yw[2 * c] * si;", "im += yw[2 * c + 1] * cr;"),
    "channel_shift": ("const double coeff = h[(int64_t)t * N + c];",
                      "const double coeff = h[(int64_t)t * N + (c + 1) % N];"),
}


def _run_pins(orc):
    failed = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(orc)
        except AssertionError:
            failed.append(pin.__name__)
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "mutant.c")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        lib = oracle._compile(path, os.path.join(d, "libmutant.so"))
        failed = _run_pins(oracle.Oracle(lib))
    assert failed, f"no pin catches the planted mistake '{name}'"
