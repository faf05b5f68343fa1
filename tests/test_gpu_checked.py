"""The bounds-checked build (stand-in for a memory checker, which this GPU pool
does not offer).

libppf_checked.so is the library built with -DPPF_CHECKED: the ring, gather
and general kernels test the index of every shared-memory and global access
they make (ring and FFT buffers, distributed-shared-memory stores, bulk-copy
destinations, spectrum stores) against the buffer's size, count a violation
and skip the access instead of making it.  Every compiled tile shape of every
(N, T) of the real-time sweep, the FP16-output twins, small and maximal sizes
and the reduced input types run through it in a child process; the test
requires zero violations and outputs bitwise equal to the normal build's (the
checks change no arithmetic).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_no_violations_and_same_results(tmp_path):
    import torch
    from paper_1411_3656_gb300 import build, ppf
    lib = build.build(checked=True)
    build.build()
    ppf.load()
    assert ppf.load().ppf_check_violations(0) == -1  # the normal build has no checks
    out = tmp_path / "checked.npz"
    env = dict(os.environ, PPF_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py"), str(out)],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert "0 violations" in r.stdout
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import checked_cases
    got = np.load(out)
    cases = checked_cases.cases()
    assert set(got.files) == {c[0] for c in cases}
    for k, (name, N, T, dtype, kind, variant) in enumerate(cases):
        ref, kern = checked_cases.run_case(N, T, dtype, kind, variant, 9000 + k)
        assert np.array_equal(got[name], ref), (name, kern)
    torch.cuda.synchronize()
