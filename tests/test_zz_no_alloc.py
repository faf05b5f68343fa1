"""The no-allocation entry point against the plan-based one.

ppf_execute_noalloc serves callers that cannot allocate device memory when
they need a filter bank (inside CUDA graph capture, under a framework that
owns all device memory, on real-time threads that must not wait on the
allocator).  It keeps its FFT twiddle table in a static device array instead
of a plan.  This file is collected last so that a failure here, under -x,
comes after every other test has run; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1411_3656_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1411_3656_gb300 import build, ppf
    build.build()
    assert torch.cuda.is_available()
    return ppf.load()


def _case(N, T, S, seed):
    x = synth.stream(synth.samples_for(S, N, T), N, seed)
    h = np.random.default_rng(seed).standard_normal(N * T).astype(np.float32)
    return x, h


def test_noalloc_matches_ppf_execute_two_calls(lib):
    """Two calls in a row (different N, so the second rewrites the shared scratch)."""
    import torch
    from paper_1411_3656_gb300 import ppf
    sp = torch.cuda.current_stream().cuda_stream
    for N, T, S in [(1024, 8, 37), (256, 16, 91)]:
        x, h = _case(N, T, S, 700 + N)
        xd = torch.from_numpy(x).cuda()
        hd = torch.from_numpy(h).cuda()
        plan = ppf.Plan(N, T, h)
        ref = plan(xd, n_spectra=S)
        out = torch.empty((S, N), dtype=torch.complex64, device="cuda")
        st = lib.ppf_execute_noalloc(N, T, 0, hd.data_ptr(), xd.data_ptr(), out.data_ptr(), S, sp)
        assert st == 0, ppf.ppf_status_string(st)
        torch.cuda.synchronize()
        err = synth.rel_l2(out.cpu().numpy(), ref.cpu().numpy())
        assert err <= TOL32, (N, T, err)


def test_noalloc_rejects_beyond_scratch_and_bad_args(lib):
    import torch
    x = torch.zeros(64, dtype=torch.complex64, device="cuda")
    h = torch.zeros(64, dtype=torch.float32, device="cuda")
    y = torch.zeros(64, dtype=torch.complex64, device="cuda")
    assert lib.ppf_execute_noalloc(8192, 4, 0, h.data_ptr(), x.data_ptr(), y.data_ptr(), 1, None) == 2
    assert lib.ppf_execute_noalloc(256, 0, 0, h.data_ptr(), x.data_ptr(), y.data_ptr(), 1, None) == 2
    assert lib.ppf_execute_noalloc(16, 2, 0, None, x.data_ptr(), y.data_ptr(), 1, None) == 1
    assert lib.ppf_execute_noalloc(16, 2, 0, h.data_ptr(), x.data_ptr() + 8, y.data_ptr(), 1, None) == 3
