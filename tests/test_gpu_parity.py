"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (relative L2 over the compared spectra, FP64):
  * complex64 input, FP32 arithmetic: <= 1e-5;
  * float16 / int8 storage against the oracle on the stored values with the
    caller's FP32 h: <= 3e-3 (covers the FP16 rounding of h), and <= 1e-5
    against the oracle run with the FP16-rounded h the device uses.
"""
import numpy as np
import pytest

import oracle
from paper_1411_3656_gb300 import synth

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL_REDUCED = 3e-3


@pytest.fixture(scope="module")
def ppf():
    import torch
    from paper_1411_3656_gb300 import build, ppf as mod
    build.build()
    mod.load()
    assert torch.cuda.is_available()
    return mod


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def _run(ppf, x, h, N, T, S, dtype="c32", flags=0):
    import torch
    plan = ppf.Plan(N, T, h, dtype, flags)
    xd = _dev(x)
    before = ppf.ppf_launch_count()
    Y = plan(xd, n_spectra=S)
    torch.cuda.synchronize()
    if S > 0:
        assert ppf.ppf_launch_count() > before
    return Y.cpu().numpy(), plan.kernel


def _rand(N, T, S, seed):
    x = synth.stream(synth.samples_for(S, N, T), N, seed)
    g = np.random.default_rng(seed)
    h = g.standard_normal(N * T).astype(np.float32)
    return x, h


def test_plain_config_n256_t8_s1024(ppf):
    """N=256, T=8, 1024 spectra, Hamming-sinc h, noise + 3 tones: the whole output."""
    x, h, N, T, S = synth.plain_config()
    Y, kern = _run(ppf, x, h, N, T, S)
    ref = oracle.ppf(x, h, N, T, S)
    err = synth.rel_l2(Y, ref)
    assert err <= TOL32, (kern, err)


SIZES = [(4, 1, 37), (4, 3, 50), (8, 2, 41), (16, 4, 33), (32, 5, 70), (64, 8, 39), (128, 4, 77),
         (256, 8, 45), (256, 1, 19), (512, 16, 21), (1024, 8, 19), (1024, 32, 9), (2048, 4, 11),
         (4096, 8, 7), (4096, 32, 5), (256, 64, 13), (128, 13, 29), (4096, 64, 3), (4, 64, 20)]


@pytest.mark.parametrize("N,T,S", SIZES)
@pytest.mark.parametrize("generic", [False, True])
def test_sizes_ragged(ppf, N, T, S, generic):
    x, h = _rand(N, T, S, 1000 + N + 7 * T)
    Y, kern = _run(ppf, x, h, N, T, S, flags=ppf.FLAG_GENERIC if generic else 0)
    if generic:
        assert kern == "generic"
    ref = oracle.ppf(x, h, N, T, S)
    assert synth.rel_l2(Y, ref) <= TOL32, (kern, "worst spectrum", synth.worst_spectrum_rel_l2(Y, ref))


# (N, T, S): the general kernel's FIR-only form (N = 16, T = 3) and the
# FIR-only kernel for every T it is built for, several bands per channel
# slice and ragged last blocks
FIR_CELLS = [(16, 3, 9), (256, 8, 31), (4096, 4, 3), (128, 4, 2203), (256, 32, 999), (512, 16, 1201),
             (1024, 8, 611), (2048, 32, 157), (4096, 16, 97), (4096, 32, 1)]


@pytest.mark.parametrize("N,T,S", FIR_CELLS)
def test_fir_only_hook(ppf, N, T, S):
    """PPF_FLAG_FIR_ONLY writes the filtered rows y (Section 2, Eq. 1) against
    the oracle's FIR; sizes with a FIR-only tile shape use the FIR-only kernel."""
    x, h = _rand(N, T, S, 77)
    Y, kern = _run(ppf, x, h, N, T, S, flags=ppf.FLAG_FIR_ONLY)
    if N >= 128 and T in (4, 8, 16, 32):
        assert kern.startswith("fir:"), kern
    ref = oracle.fir(x, h, N, T, S)
    assert synth.rel_l2(Y, ref) <= TOL32, ("rel L2", "worst spectrum", synth.worst_spectrum_rel_l2(Y, ref))


def test_impulse_on_device(ppf):
    """Impulse reproduces h on the GPU as well (convention check independent of tolerance)."""
    N, T, S = 64, 4, 10
    h = np.random.default_rng(5).standard_normal(N * T).astype(np.float32)
    x = np.zeros((S + T - 1) * N, dtype=np.complex64)
    r, c0 = 6, 9
    x[r * N + c0] = 1.0
    Y, _ = _run(ppf, x, h, N, T, S)
    k = np.arange(N)
    for s in range(S):
        t = r - s
        want = h[t * N + c0] * np.exp(-2j * np.pi * k * c0 / N) if 0 <= t < T else np.zeros(N)
        assert np.allclose(Y[s], want, atol=2e-6 * max(1.0, np.abs(h).max()))


def test_zero_and_single_spectrum(ppf):
    import torch
    N, T = 256, 8
    x, h = _rand(N, T, 1, 3)
    plan = ppf.Plan(N, T, h)
    xd = _dev(x)
    before = ppf.ppf_launch_count()
    out = torch.empty((0, N), dtype=torch.complex64, device="cuda")
    assert ppf.ppf_execute(plan.handle, xd.data_ptr(), out.data_ptr(), 0, 0) == 0
    assert ppf.ppf_launch_count() == before
    Y = plan(xd, n_spectra=1)
    torch.cuda.synchronize()
    assert synth.rel_l2(Y.cpu().numpy(), oracle.ppf(x, h, N, T, 1)) <= TOL32, ("rel L2", "worst spectrum", synth.worst_spectrum_rel_l2(Y.cpu().numpy(), oracle.ppf(x, h, N, T, 1)))


def test_argument_errors(ppf):
    import torch
    N, T = 256, 8
    h = np.ones(N * T, np.float32)
    plan = ppf.Plan(N, T, h)
    x = torch.zeros(N * (T + 4) + 4, dtype=torch.complex64, device="cuda")
    y = torch.zeros(16 * N + 2, dtype=torch.complex64, device="cuda")
    assert ppf.ppf_execute(plan.handle, x.data_ptr() + 8, y.data_ptr(), 4, 0) == 3  # misaligned in
    assert ppf.ppf_execute(plan.handle, x.data_ptr(), y.data_ptr() + 8, 4, 0) == 3  # misaligned out
    assert ppf.ppf_execute(plan.handle, x.data_ptr(), x.data_ptr() + 16 * N, 4, 0) == 3  # overlap
    assert ppf.ppf_execute(plan.handle, x.data_ptr(), y.data_ptr(), -1, 0) == 1


@pytest.mark.parametrize("dtype", ["c16", "ci8"])
def test_reduced_precision_n1024_t8(ppf, dtype):
    """FP16 / int8 I-Q storage at N=1024, T=8 (FP32 accumulation, FP16 h)."""
    N, T, S = 1024, 8, 64
    n = synth.samples_for(S, N, T)
    if dtype == "c16":
        xs = synth.to_fp16_iq(synth.stream(n, N, 4242))
    else:
        xs = synth.int8_iq(n, 4243)
    h = synth.hamming_sinc(N, T)
    Y, _ = _run(ppf, xs, h, N, T, S, dtype=dtype)
    err = synth.rel_l2(Y, oracle.ppf(xs, h, N, T, S))
    assert err <= TOL_REDUCED, err
    h16 = h.astype(np.float16).astype(np.float32)
    assert synth.rel_l2(Y, oracle.ppf(xs, h16, N, T, S)) <= TOL32, ("rel L2", "worst spectrum", synth.worst_spectrum_rel_l2(Y, oracle.ppf(xs, h16, N, T, S)))


@pytest.mark.parametrize("dtype", ["c16", "ci8"])
@pytest.mark.parametrize("N,T,S", [(4, 5, 33), (4, 1, 17), (8, 3, 40), (16, 2, 21), (32, 7, 19)])
def test_reduced_precision_small_n(ppf, dtype, N, T, S):
    """FP16 / int8 storage at the smallest sizes (N = 4 included for both):
    the oracle on the stored values with the device's FP16 h, gate 1e-5."""
    n = synth.samples_for(S, N, T)
    xs = synth.to_fp16_iq(synth.stream(n, N, 4300 + N)) if dtype == "c16" else synth.int8_iq(n, 4301 + N)
    h = np.random.default_rng(4302 + N + T).standard_normal(N * T).astype(np.float32)
    Y, kern = _run(ppf, xs, h, N, T, S, dtype=dtype)
    ref = oracle.ppf(xs, h.astype(np.float16).astype(np.float32), N, T, S)
    assert synth.rel_l2(Y, ref) <= TOL32, (kern, "worst spectrum", synth.worst_spectrum_rel_l2(Y, ref))


@pytest.mark.parametrize("N,T", [(256, 8), (1024, 16), (64, 3)])
def test_stream_equals_batch(ppf, N, T):
    """Pushing chunks of arbitrary length emits exactly the batch result."""
    import torch
    total = N * 57 + 13
    h = np.random.default_rng(31 + N).standard_normal(N * T).astype(np.float32)
    x = synth.stream(total, N, 31 + N)
    plan = ppf.Plan(N, T, h)
    batch = plan(_dev(x)).cpu().numpy()
    st = ppf.Stream(plan)
    g = np.random.default_rng(8)
    sizes = [1, N - 1, 3 * N + 5, 0, 2 * N, 7, N * 11 + 1]
    pos, i, outs = 0, 0, []
    while pos < total:
        n = sizes[i] if i < len(sizes) else int(g.integers(1, 4 * N))
        i += 1
        n = min(n, total - pos)
        chunk = _dev(x[pos:pos + n]) if n else None
        outs.append(st.push(chunk).cpu().numpy())
        pos += n
    torch.cuda.synchronize()
    got = np.concatenate(outs)
    assert got.shape == batch.shape
    assert np.array_equal(got, batch)
    assert st.position == (total, batch.shape[0])
    st.close()


@pytest.mark.parametrize("N,T,S,dtype", [(1024, 8, 40000, "c32"), (256, 16, 300000, "c32"),
                                         (4096, 32, 9000, "c16")])
def test_execute_host_equals_device(ppf, N, T, S, dtype):
    """ppf_execute_host (host buffers, the input cut into slices of 32 Mi
    samples whose copies overlap the kernels): bitwise the device-buffer
    result, and the spectra on both sides of every slice boundary, the ends
    and a seeded sample against the oracle."""
    import torch
    x, h = _rand(N, T, S, 55 + N)
    xs = _stored(x, dtype, 56 + N)
    plan = ppf.Plan(N, T, h, dtype)
    dev = plan(_dev(xs)).cpu()
    xh = torch.from_numpy(np.ascontiguousarray(xs)).pin_memory()
    host = plan.execute_host(xh)
    assert torch.equal(dev, host)
    per_slice = (32 << 20) // N
    edges = {r for b in range(per_slice, S, per_slice) for r in (b - 2, b - 1, b, b + 1)}
    rows = np.asarray(sorted(edges | set(synth.sample_rows(S, 256).tolist())), dtype=np.int64)
    hr = h if dtype == "c32" else h.astype(np.float16).astype(np.float32)
    ref = oracle.ppf_rows(xs, hr, N, T, rows)
    got = host.numpy()[rows]
    assert synth.rel_l2(got, ref) <= TOL32, ("worst spectrum", synth.worst_spectrum_rel_l2(got, ref))


@pytest.mark.parametrize("N,T", [(1024, 8)])
def test_full_size_realtime_second_sampled(ppf, N, T):
    """One second of 6.5 GB/s complex64 at (N, T), as the benchmark launches it.

    The whole stream runs in one ppf_execute; 1040 spectra (first 8, last 8,
    1024 seeded) are checked against the oracle.
    """
    import torch
    x, h, N, T, S = synth.realtime_second_config(N, T)
    plan = ppf.Plan(N, T, h)
    xd = _dev(x)
    Y = plan(xd)
    torch.cuda.synchronize()
    rows = synth.sample_rows(S)
    got = Y[torch.from_numpy(rows).to("cuda")].cpu().numpy()
    ref = oracle.ppf_rows(x, h, N, T, rows)
    assert synth.rel_l2(got, ref) <= TOL32, ("rel L2", "worst spectrum", synth.worst_spectrum_rel_l2(got, ref))
    del xd, Y
    torch.cuda.empty_cache()


VARIANT_CELLS = [(N, T) for N in (128, 256, 512, 1024, 2048, 4096) for T in (4, 8, 16, 32)]


def _stored(x, dtype, seed):
    if dtype == "c16":
        return synth.to_fp16_iq(x)
    if dtype == "ci8":
        return synth.int8_iq(x.shape[0], seed)
    return x


@pytest.mark.parametrize("N,T", VARIANT_CELLS)
@pytest.mark.parametrize("dtype", ["c32", "c16", "ci8"])
def test_every_variant(ppf, N, T, dtype):
    """Every compiled tile-shape variant of the specialised kernels matches the oracle.

    Reduced-precision inputs are compared with the oracle run on the stored
    values and the FP16-rounded coefficients the device uses.
    """
    n = ppf.ppf_variant_count(N, T, dtype)
    if n == 0:
        pytest.skip("no specialised variant for this size")
    S = max(3, 40960 // N) + 3
    x, h = _rand(N, T, S, 2000 + N + T)
    xs = _stored(x, dtype, 2100 + N + T)
    hr = h if dtype == "c32" else h.astype(np.float16).astype(np.float32)
    ref = oracle.ppf(xs, hr, N, T, S)
    for i in range(n):
        Y, kern = _run(ppf, xs, h, N, T, S, dtype=dtype, flags=ppf.flag_variant(i))
        assert kern == ppf.ppf_variant_name(N, T, dtype, i)
        assert synth.rel_l2(Y, ref) <= TOL32, (kern, "worst spectrum", synth.worst_spectrum_rel_l2(Y, ref))


# (N, T, S): S gives every persistent CTA (or cluster) of the default kernel
# about three blocks plus a ragged tail, so every band boundary and the
# partial last block are inside the compared output.
BAND_CELLS = [(512, 32, 3659), (2048, 8, 919), (4096, 8, 461), (4096, 32, 365), (1024, 32, 1831)]


@pytest.mark.parametrize("N,T,S", BAND_CELLS)
def test_default_kernel_every_band_boundary(ppf, N, T, S):
    """The tuned default kernel over several blocks per CTA: every spectrum
    against the oracle (band boundaries between CTAs, ring wrap-arounds and
    the ragged last block included)."""
    x, h = _rand(N, T, S, 3000 + N + T)
    Y, kern = _run(ppf, x, h, N, T, S)
    ref = oracle.ppf(x, h, N, T, S)
    assert synth.rel_l2(Y, ref) <= TOL32, (kern, "worst spectrum", synth.worst_spectrum_rel_l2(Y, ref))


SWEEP_CELLS = [(N, T) for N in (256, 512, 1024, 2048, 4096) for T in (4, 8, 16, 32)]


@pytest.fixture(scope="module")
def second_of_data():
    """One second of 6.5 GB/s complex64 (8.125e8 samples), shared by every sweep
    cell (each reads its prefix of (S+T-1)*N samples), on the host and the device."""
    x = synth.stream(int(synth.REALTIME_SAMPLES_PER_S), 1024, synth.BASE_SEED + 11)
    xd = _dev(x)
    yield x, xd
    del xd


@pytest.mark.parametrize("N,T", SWEEP_CELLS)
def test_full_size_sweep_cell_sampled(ppf, second_of_data, N, T):
    """Every cell of the real-time sweep at full size, with the tuned default
    kernel and launch configuration the benchmark times: 272 spectra (the first
    8, the last 8, 256 seeded) against the oracle."""
    import torch
    x, xd = second_of_data
    S = synth.spectra_for(x.shape[0], N, T)
    h = synth.hamming_sinc(N, T)
    plan = ppf.Plan(N, T, h)
    Y = plan(xd[: synth.samples_for(S, N, T)], n_spectra=S)
    torch.cuda.synchronize()
    rows = synth.sample_rows(S, count=256)
    got = Y[torch.from_numpy(rows).to("cuda")].cpu().numpy()
    kern = plan.kernel
    del Y
    plan.close()
    torch.cuda.empty_cache()
    ref = oracle.ppf_rows(x, h, N, T, rows)
    assert synth.rel_l2(got, ref) <= TOL32, (kern, "worst spectrum", synth.worst_spectrum_rel_l2(got, ref))


@pytest.mark.parametrize("N,T", VARIANT_CELLS + [(64, 3), (1024, 13)])
def test_fp16_output_every_variant(ppf, N, T):
    """PPF_FLAG_OUT_F16: a plan runs the FP16-output twin of the tile shape its
    complex64 counterpart runs (else the general kernel); its bins are that
    shape's complex64 bins rounded to nearest (bitwise), hence within FP16
    rounding (2^-11 relative per component; gate 1e-3 relative L2) of the oracle.
    Checked for the tuned default, the general kernel and every forced variant."""
    import torch
    S = max(3, 40960 // N) + 3
    x, h = _rand(N, T, S, 2200 + N + T)
    ref = oracle.ppf(x, h, N, T, S)
    xd = _dev(x)
    flags = [0, ppf.FLAG_GENERIC] + [ppf.flag_variant(i) for i in range(ppf.ppf_variant_count(N, T, "c32"))]
    default_twin = False
    for fl in flags:
        p16 = ppf.Plan(N, T, h, "c32", fl | ppf.FLAG_OUT_F16)
        p32 = ppf.Plan(N, T, h, "c32", fl)
        if p16.kernel == "generic:f16":
            p32 = ppf.Plan(N, T, h, "c32", ppf.FLAG_GENERIC)
        else:
            assert p16.kernel == p32.kernel + ":f16"
            default_twin = default_twin or fl == 0
        y32 = p32(xd, n_spectra=S)
        y16 = p16(xd, n_spectra=S)
        torch.cuda.synchronize()
        assert y16.dtype == torch.float16 and tuple(y16.shape) == (S, N, 2)
        assert torch.equal(y16, torch.view_as_real(y32).to(torch.float16)), p16.kernel
        got = y16.float().cpu().numpy().view(np.complex64)[..., 0]
        assert synth.rel_l2(got, ref) <= 1e-3, (p16.kernel, "worst spectrum", synth.worst_spectrum_rel_l2(got, ref))
    if (N, T) in VARIANT_CELLS and N >= 256:
        assert default_twin  # the tuned default of a sweep cell has an FP16 twin


def test_fp16_output_unsupported_paths(ppf):
    import torch
    N, T = 256, 8
    h = synth.hamming_sinc(N, T)
    with pytest.raises(ppf.PPFError):
        ppf.Plan(N, T, h, "c32", ppf.FLAG_OUT_F16 | ppf.FLAG_FIR_ONLY)
    plan = ppf.Plan(N, T, h, "c32", ppf.FLAG_OUT_F16)
    x = torch.zeros(16 * N, dtype=torch.complex64).pin_memory()
    y = torch.zeros(16 * N, dtype=torch.complex64).pin_memory()
    assert ppf.ppf_execute_host(plan.handle, x.data_ptr(), y.data_ptr(), 4, 0) == 2  # PPF_ERR_UNSUPPORTED
    import ctypes
    s = ctypes.c_void_p()
    assert ppf.load().ppf_stream_open(plan.handle, ctypes.byref(s)) == 2
