"""Failure detection on the device without a fault: a bounded wait made to run out.

ppf_check_timeout launches one warp that waits on an mbarrier nothing
completes, through the PPF kernels' own bounded wait, with a 1 ms limit.  The
wait must give up, report PPF_ERR_TIMEOUT through the mapped error word, and
leave the context usable for a normal PPF launch afterwards.
"""
import numpy as np
import pytest

import oracle
from paper_1411_3656_gb300 import synth

pytestmark = pytest.mark.gpu

PPF_OK, PPF_ERR_INVALID_ARG, PPF_ERR_TIMEOUT = 0, 1, 6


@pytest.fixture(scope="module")
def ppf():
    from paper_1411_3656_gb300 import build, ppf as mod
    build.build()
    mod.load()
    return mod


def test_bounded_wait_times_out_and_reports(ppf):
    import time
    import torch
    t0 = time.perf_counter()
    assert ppf.ppf_check_timeout(1000) == PPF_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    # the context is intact: a normal launch still matches the oracle
    x, h, N, T, S = synth.plain_config()
    plan = ppf.Plan(N, T, h)
    Y = plan(torch.from_numpy(x).cuda(), n_spectra=S)
    torch.cuda.synchronize()
    assert synth.rel_l2(Y.cpu().numpy(), oracle.ppf(x, h, N, T, S)) <= 1e-5, ("rel L2", "worst spectrum", synth.worst_spectrum_rel_l2(Y.cpu().numpy(), oracle.ppf(x, h, N, T, S)))
    plan.close()


def test_limit_out_of_range(ppf):
    assert ppf.ppf_check_timeout(0) == PPF_ERR_INVALID_ARG
    assert ppf.load().ppf_check_timeout(2000000, None) == PPF_ERR_INVALID_ARG
