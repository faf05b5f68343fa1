"""Batches of independent streams (ppf_batch_*): every job against the FP64
oracle (relative L2 <= 1e-5; reduced-precision jobs on their stored values
with the FP16 coefficients the device uses) and bitwise against one
ppf_execute per stream."""
import numpy as np
import pytest

import oracle
from paper_1411_3656_gb300 import synth

TOL32 = 1e-5

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ppf():
    import torch
    from paper_1411_3656_gb300 import build, ppf as mod
    build.build()
    mod.load()
    assert torch.cuda.is_available()
    return mod


def _jobs(ppf, specs, seed):
    """specs: (N, T, dtype, S[, kernel family]).  Each job gets its own seeded
    input and h; a job naming a kernel family runs that family's first compiled
    tile shape instead of the tuned default."""
    import torch
    out = []
    for i, spec in enumerate(specs):
        N, T, dt, S = spec[:4]
        flags = 0
        if len(spec) > 4:
            names = [ppf.ppf_variant_name(N, T, dt, v) for v in range(ppf.ppf_variant_count(N, T, dt))]
            flags = ppf.flag_variant(next(v for v, nm in enumerate(names) if nm.startswith(spec[4])))
        g = np.random.default_rng(seed + i)
        h = g.standard_normal(N * T).astype(np.float32)
        x = synth.stream(synth.samples_for(S, N, T), N, seed + 100 + i)
        if dt == "c16":
            x = synth.to_fp16_iq(x)
        elif dt == "ci8":
            x = synth.int8_iq(synth.samples_for(S, N, T), seed + 200 + i)
        plan = ppf.Plan(N, T, h, dt, flags)
        # what the oracle needs: the stored input and the coefficients the device uses
        plan.oracle_in = (x, h if dt == "c32" else h.astype(np.float16).astype(np.float32))
        xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        yd = torch.full((S, N), float("nan"), dtype=torch.complex64, device="cuda")
        out.append((plan, xd, yd, S))
    return out


def check_oracle(jobs, rows_per_job=None):
    """Each job's output (torch, complex64) against the oracle on its stored input."""
    for plan, xd, yd, S in jobs:
        if S == 0:
            continue
        x, h = plan.oracle_in
        got = yd.cpu().numpy()
        if rows_per_job is None or S <= rows_per_job:
            ref = oracle.ppf(x, h, plan.N, plan.T, S)
        else:
            rows = synth.sample_rows(S, rows_per_job)
            ref = oracle.ppf_rows(x, h, plan.N, plan.T, rows)
            got = got[rows]
        err = synth.rel_l2(got, ref)
        assert err <= TOL32, (plan.kernel, plan.N, plan.T, S, err, synth.worst_spectrum_rel_l2(got, ref))


SPECS = [(256, 8, "c32", 700), (256, 8, "c32", 1500), (1024, 8, "c32", 333), (4096, 16, "c32", 41),
         (4096, 16, "c32", 9), (2048, 32, "c32", 17, "gather:p4:nt256:rb2:nch6"), (2048, 32, "c32", 23),
         (64, 5, "c32", 90), (128, 4, "c32", 257),
         (1024, 16, "c16", 120), (512, 8, "ci8", 77), (256, 4, "c32", 0), (2048, 8, "c32", 1), (4, 3, "ci8", 50)]


@pytest.mark.parametrize("graph", [False, True])
def test_batch_equals_individual(ppf, graph):
    import torch
    jobs = _jobs(ppf, SPECS, 5000)
    batch = ppf.Batch(jobs, graph=graph)
    kernels = {p.kernel for p, _, _, _ in jobs}
    assert all(any(k.startswith(f) for k in kernels) for f in ("ring", "gather", "generic"))
    before = ppf.ppf_launch_count()
    batch.execute()
    torch.cuda.synchronize()
    if not graph:
        assert ppf.ppf_launch_count() - before == batch.launches
    check_oracle(jobs)
    for plan, xd, yd, S in jobs:
        ref = plan(xd, n_spectra=S)
        torch.cuda.synchronize()
        assert torch.equal(yd, ref), plan.kernel
    # the batch reads the inputs afresh each time (graph replay included)
    for plan, xd, yd, S in jobs:
        if xd.dtype == torch.complex64:
            xd.mul_(2)
    batch.execute()
    torch.cuda.synchronize()
    for plan, xd, yd, S in jobs:
        assert torch.equal(yd, plan(xd, n_spectra=S)), plan.kernel
    for plan, xd, yd, S in jobs:
        if xd.dtype == torch.complex64:
            plan.oracle_in = (plan.oracle_in[0] * np.complex64(2), plan.oracle_in[1])
    check_oracle(jobs)
    batch.close()


def test_batch_many_streams_in_few_launches(ppf):
    """64 streams of six shapes: one launch per specialised kernel, not per stream."""
    import torch
    g = np.random.default_rng(77)
    shapes = [(256, 8), (512, 4), (1024, 8), (2048, 8), (4096, 4), (128, 16)]
    specs = [(*shapes[i % len(shapes)], "c32", int(g.integers(10, 200))) for i in range(64)]
    jobs = _jobs(ppf, specs, 9000)
    batch = ppf.Batch(jobs)
    assert batch.launches <= len({p.kernel + str((p.N, p.T)) for p, _, _, _ in jobs})
    batch.execute()
    torch.cuda.synchronize()
    check_oracle(jobs)
    for plan, xd, yd, S in jobs:
        assert torch.equal(yd, plan(xd, n_spectra=S))


def test_batch_argument_errors(ppf):
    import ctypes
    lib = ppf.load()
    out = ctypes.c_void_p()
    assert lib.ppf_batch_create(None, None, 0, 0) == 1
    assert lib.ppf_batch_create(ctypes.byref(out), None, -1, 0) == 1
    assert lib.ppf_batch_create(ctypes.byref(out), None, 0, 8) == 1
    assert lib.ppf_batch_create(ctypes.byref(out), None, 0, 4) == 1
    assert lib.ppf_batch_create(ctypes.byref(out), None, 0, 0) == 0
    assert lib.ppf_batch_launches(out.value) == 0
    assert lib.ppf_batch_execute(out.value, None) == 0
    assert lib.ppf_batch_destroy(out.value) == 0
    assert lib.ppf_batch_execute(None, None) == 1


def test_batch_mixes_fp16_and_complex64_outputs(ppf):
    """Jobs whose plans write FP16 bins (PPF_FLAG_OUT_F16) share launches with
    complex64 jobs of the same kernel; each matches its own ppf_execute."""
    import torch
    specs = [(256, 8, 700), (256, 8, 310), (4096, 16, 41), (4096, 16, 12), (1024, 8, 333)]
    jobs = []
    for i, (N, T, S) in enumerate(specs):
        g = np.random.default_rng(7000 + i)
        h = g.standard_normal(N * T).astype(np.float32)
        x = synth.stream(synth.samples_for(S, N, T), N, 7100 + i)
        f16 = i % 2 == 0
        plan = ppf.Plan(N, T, h, "c32", ppf.FLAG_OUT_F16 if f16 else 0)
        xd = torch.from_numpy(x).cuda()
        yd = (torch.full((S, N, 2), float("nan"), dtype=torch.float16, device="cuda") if f16
              else torch.full((S, N), float("nan"), dtype=torch.complex64, device="cuda"))
        jobs.append((plan, xd, yd, S))
    batch = ppf.Batch(jobs)
    batch.execute()
    torch.cuda.synchronize()
    for plan, xd, yd, S in jobs:
        ref = plan(xd, n_spectra=S)
        torch.cuda.synchronize()
        assert torch.equal(yd, ref), (plan.kernel, plan.out_f16)


# (N, T) of every tile shape of the mixed-shape kernel (complex64, 128 <= N <= 2048, N*T <= 16K)
MIX_SHAPES = [(128, 4), (128, 8), (128, 16), (128, 32), (256, 4), (256, 8), (256, 16), (256, 32), (512, 4),
              (512, 8), (512, 16), (512, 32), (1024, 4), (1024, 8), (1024, 16), (2048, 4), (2048, 8)]


@pytest.mark.parametrize("graph", [False, True])
def test_batch_mixed_shapes_one_launch(ppf, graph):
    """Streams of every (N, T) the mixed-shape kernel takes, ragged lengths
    (several work items per stream for the long ones), in ONE persistent
    launch: every spectrum against the FP64 oracle and bitwise against the
    stream's own ppf_execute (tuned default kernel)."""
    import torch
    g = np.random.default_rng(31)
    specs = []
    for N, T in MIX_SHAPES:
        specs.append((N, T, "c32", int(g.integers(1, max(3, 24576 // N)))))
    specs += [(256, 8, "c32", 3001), (1024, 4, "c32", 613), (2048, 4, "c32", 1), (512, 32, "c32", 0)]
    jobs = _jobs(ppf, specs, 9500)
    batch = ppf.Batch(jobs, graph=graph)
    assert batch.launches == 1
    before = ppf.ppf_launch_count()
    batch.execute()
    torch.cuda.synchronize()
    if not graph:
        assert ppf.ppf_launch_count() - before == 1
    check_oracle(jobs)
    for plan, xd, yd, S in jobs:
        if S:
            assert torch.equal(yd, plan(xd, n_spectra=S)), (plan.N, plan.T, plan.kernel)
    # a second execution (graph replay) on new input
    for plan, xd, yd, S in jobs:
        xd.mul_(-0.5)
        plan.oracle_in = (plan.oracle_in[0] * np.complex64(-0.5), plan.oracle_in[1])
    batch.execute()
    torch.cuda.synchronize()
    check_oracle(jobs)
    batch.close()


def test_batch_mixed_ring_reaches_buffer_slot(ppf):
    """Streams whose ring reaches into the first FFT buffer slot (512x32,
    1024x16) alternate with streams whose buffer fills a whole slot (2048x4,
    512x8, 1024x8), so that CTAs cross from one to the other inside their
    segment and must wait for the FFT warps first: every spectrum against the
    oracle and bitwise against ppf_execute."""
    import torch
    specs = []
    for k in range(4):
        specs += [(2048, 4, "c32", 97 + k), (1024, 16, "c32", 61 + 3 * k), (512, 8, "c32", 203 + k),
                  (512, 32, "c32", 88 + k), (1024, 8, "c32", 45 + k)]
    jobs = _jobs(ppf, specs, 9800)
    batch = ppf.Batch(jobs)
    assert batch.launches == 1
    batch.execute()
    torch.cuda.synchronize()
    check_oracle(jobs)
    for plan, xd, yd, S in jobs:
        assert torch.equal(yd, plan(xd, n_spectra=S)), (plan.N, plan.T, plan.kernel)
    batch.close()


def test_batch_groups_beside_the_mixed_launch(ppf):
    """Cluster-kernel and 4096-channel jobs in their own group launches after
    the mixed launch (graph and eager): oracle and bitwise parity."""
    import torch
    specs = [(2048, 16, "c32", 150), (4096, 8, "c32", 77), (4096, 4, "c32", 64), (1024, 32, "c32", 90),
             (2048, 4, "c32", 400), (512, 8, "c32", 900), (256, 16, "c32", 1200), (128, 4, "c32", 3000)]
    jobs = _jobs(ppf, specs, 9900)
    for graph in (False, True):
        batch = ppf.Batch(jobs, graph=graph)
        assert batch.launches == 1 + len({p.kernel for p, _, _, _ in jobs if p.N * p.T > 16384 or p.N == 4096})
        for _, _, yd, _ in jobs:
            yd.fill_(float("nan"))
        batch.execute()
        torch.cuda.synchronize()
        check_oracle(jobs)
        for plan, xd, yd, S in jobs:
            assert torch.equal(yd, plan(xd, n_spectra=S)), (plan.N, plan.T, plan.kernel)
        batch.close()


def test_batch_per_kernel_flag(ppf):
    """PPF_BATCH_PER_KERNEL keeps one persistent launch per specialised kernel
    (the comparison form); results are those of the mixed launch, bitwise."""
    import torch
    specs = [(256, 8, "c32", 300), (1024, 8, "c32", 97), (2048, 4, "c32", 41), (512, 16, "c32", 128)]
    jobs = _jobs(ppf, specs, 9700)
    mixed = ppf.Batch(jobs)
    assert mixed.launches == 1
    mixed.execute()
    torch.cuda.synchronize()
    first = [yd.clone() for _, _, yd, _ in jobs]
    per = ppf.Batch(jobs, per_kernel=True)
    assert per.launches == len({p.kernel for p, _, _, _ in jobs})
    per.execute()
    torch.cuda.synchronize()
    for (plan, xd, yd, S), y0 in zip(jobs, first):
        assert torch.equal(yd, y0), plan.kernel
    check_oracle(jobs)
    mixed.close()
    per.close()
