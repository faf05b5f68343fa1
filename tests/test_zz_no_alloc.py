"""The no-allocation entry point, against the plan-based one and the FP64 oracle.

ppf_execute_noalloc serves callers that cannot allocate device memory when
they need a filter bank: plug-ins under a framework that owns all device
memory, and real-time threads that must not wait on the allocator (cudaMalloc
and cudaFree can synchronise the whole device).  It keeps its FFT twiddle
table in a static device array instead of a plan, and takes FP32 coefficients
for every input type.  This file is collected last so that a failure here,
under -x, comes after every other test has run; it also passes alone in a
fresh process.

Tolerance: relative L2 <= 1e-5 against the oracle on the stored input values
with the same FP32 h (FP32 arithmetic on every input type).
"""
import numpy as np
import pytest

import oracle
from paper_1411_3656_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
DT = {"c32": 0, "c16": 1, "ci8": 2}


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_1411_3656_gb300 import build, ppf
    build.build()
    assert torch.cuda.is_available()
    return ppf.load()


def _case(N, T, S, seed, dtype="c32"):
    n = synth.samples_for(S, N, T)
    if dtype == "ci8":
        x = synth.int8_iq(n, seed)
    else:
        x = synth.stream(n, N, seed)
        if dtype == "c16":
            x = synth.to_fp16_iq(x)
    h = np.random.default_rng(seed).standard_normal(N * T).astype(np.float32)
    return x, h


def _noalloc(lib, N, T, S, x, h, dtype="c32"):
    import torch
    from paper_1411_3656_gb300 import ppf
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    hd = torch.from_numpy(h).cuda()
    out = torch.full((S, N), float("nan"), dtype=torch.complex64, device="cuda")
    sp = torch.cuda.current_stream().cuda_stream
    st = lib.ppf_execute_noalloc(N, T, DT[dtype], hd.data_ptr(), xd.data_ptr(), out.data_ptr(), S, sp)
    assert st == 0, ppf.ppf_status_string(st)
    torch.cuda.synchronize()
    return xd, out.cpu().numpy()


def _check(Y, ref, what):
    err = synth.rel_l2(Y, ref)
    worst = synth.worst_spectrum_rel_l2(Y, ref)
    assert err <= TOL32, (what, err, worst)


def test_noalloc_matches_ppf_execute_two_calls(lib):
    """Two calls in a row (different N, so the second rewrites the shared
    scratch): each equals ppf_execute and the FP64 oracle."""
    import torch
    from paper_1411_3656_gb300 import ppf
    for N, T, S in [(1024, 8, 37), (256, 16, 91)]:
        x, h = _case(N, T, S, 700 + N)
        xd, Y = _noalloc(lib, N, T, S, x, h)
        plan = ppf.Plan(N, T, h)
        ref = plan(xd, n_spectra=S)
        torch.cuda.synchronize()
        assert synth.rel_l2(Y, ref.cpu().numpy()) <= TOL32, (N, T)
        _check(Y, oracle.ppf(x, h, N, T, S), (N, T))
        plan.close()


@pytest.mark.parametrize("dtype", ["c16", "ci8"])
@pytest.mark.parametrize("N,T,S", [(1024, 8, 29), (8, 3, 40), (4, 5, 33)])
def test_noalloc_reduced_inputs_against_oracle(lib, dtype, N, T, S):
    """FP16 and int8 storage with FP32 coefficients: FP32 arithmetic on the
    stored values, so the 1e-5 gate against the oracle on those values."""
    x, h = _case(N, T, S, 900 + N + T, dtype)
    _, Y = _noalloc(lib, N, T, S, x, h, dtype)
    _check(Y, oracle.ppf(x, h, N, T, S), (dtype, N, T))


def test_noalloc_full_scratch_n4096(lib):
    """N = 4096 fills the whole twiddle array; T = 64 is the largest tap count."""
    N, T, S = 4096, 64, 5
    x, h = _case(N, T, S, 4096)
    _, Y = _noalloc(lib, N, T, S, x, h)
    _check(Y, oracle.ppf(x, h, N, T, S), (N, T))


def test_noalloc_rejects_beyond_scratch_and_bad_args(lib):
    import torch
    x = torch.zeros(64, dtype=torch.complex64, device="cuda")
    h = torch.zeros(64, dtype=torch.float32, device="cuda")
    y = torch.zeros(64, dtype=torch.complex64, device="cuda")
    assert lib.ppf_execute_noalloc(8192, 4, 0, h.data_ptr(), x.data_ptr(), y.data_ptr(), 1, None) == 2
    assert lib.ppf_execute_noalloc(256, 0, 0, h.data_ptr(), x.data_ptr(), y.data_ptr(), 1, None) == 2
    assert lib.ppf_execute_noalloc(16, 2, 0, None, x.data_ptr(), y.data_ptr(), 1, None) == 1
    assert lib.ppf_execute_noalloc(16, 2, 0, h.data_ptr(), x.data_ptr() + 8, y.data_ptr(), 1, None) == 3
    # coefficients inside the output buffer
    assert lib.ppf_execute_noalloc(16, 2, 0, y.data_ptr(), x.data_ptr(), y.data_ptr(), 1, None) == 3
