"""Stream checkpoint and resume through the C ABI (ppf_stream_save / _restore).

A stream saved after some pushes and restored into a new stream (on another
plan object with the same N, T and dtype) must go on exactly where it stopped:
the spectra of the first stream up to the save, followed by those of the
restored one, equal the batch result over the whole input (bitwise; the
stream path already equals the batch path bitwise), which is itself checked
against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1411_3656_gb300 import synth

pytestmark = pytest.mark.gpu

HEADER = 48


@pytest.fixture(scope="module")
def ppf():
    import torch
    from paper_1411_3656_gb300 import build, ppf as mod
    build.build()
    mod.load()
    assert torch.cuda.is_available()
    return mod


def _stored(x, dtype):
    if dtype == "c16":
        return synth.to_fp16_iq(x)
    return x


def _push_all(ppf, stream, x, cuts):
    import torch
    outs = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        outs.append(stream.push(torch.from_numpy(np.ascontiguousarray(x[a:b])).to("cuda")))
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("N,T,dtype", [(256, 8, "c32"), (64, 3, "c32"), (1024, 16, "c32"), (512, 8, "c16")])
def test_save_restore_equals_uninterrupted(ppf, N, T, dtype):
    import torch
    S = 3 * T + 41
    n = synth.samples_for(S, N, T)
    x = _stored(synth.stream(n, N, 7100 + N + T), dtype)
    h = synth.hamming_sinc(N, T)
    g = np.random.default_rng(N * 131 + T)
    # chunk edges that are not multiples of N; the save falls inside a row
    cuts = np.unique(np.concatenate([[0, n], g.integers(1, n, 9)])).tolist()
    k = len(cuts) // 2

    p1 = ppf.Plan(N, T, h, dtype)
    s1 = ppf.Stream(p1)
    first = _push_all(ppf, s1, x, cuts[:k + 1])
    pushed, emitted = s1.position
    state = s1.save()
    assert len(state) == HEADER + (pushed - emitted * N) * ppf.SAMPLE_BYTES[dtype]
    assert pushed - emitted * N < T * N
    s1.close()

    p2 = ppf.Plan(N, T, h, dtype)  # a new plan object, same N, T, dtype
    s2 = ppf.Stream.restore(p2, state)
    assert s2.position == (pushed, emitted)
    second = _push_all(ppf, s2, x, cuts[k:])
    s2.close()

    got = np.concatenate(first + second)
    batch = p1(torch.from_numpy(np.ascontiguousarray(x)).to("cuda"), n_spectra=S).cpu().numpy()
    torch.cuda.synchronize()
    assert got.shape == batch.shape == (S, N)
    assert np.array_equal(got, batch)
    assert synth.rel_l2(got, oracle.ppf(x, h, N, T, S)) <= (1e-5 if dtype == "c32" else 3e-3), ("rel L2", "worst spectrum", synth.worst_spectrum_rel_l2(got, oracle.ppf(x, h, N, T, S)))


def test_save_before_first_window_and_errors(ppf):
    import torch
    N, T = 128, 4
    h = synth.hamming_sinc(N, T)
    x = synth.stream(synth.samples_for(20, N, T), N, 7201)
    plan = ppf.Plan(N, T, h)
    s = ppf.Stream(plan)
    # fewer than T rows: nothing emitted yet, every sample held
    s.push(torch.from_numpy(x[:2 * N + 5]).to("cuda"))
    state = s.save()
    assert s.position == (2 * N + 5, 0)
    assert len(state) == HEADER + (2 * N + 5) * 8
    # the saved stream itself goes on
    rest = s.push(torch.from_numpy(x[2 * N + 5:]).to("cuda")).cpu().numpy()
    s.close()
    r = ppf.Stream.restore(ppf.Plan(N, T, h), state)
    again = r.push(torch.from_numpy(x[2 * N + 5:]).to("cuda")).cpu().numpy()
    r.close()
    assert np.array_equal(rest, again) and rest.shape == (20, N)

    # a plan of another shape or type, a truncated or corrupted state: refused
    for other in (ppf.Plan(N, T + 1, synth.hamming_sinc(N, T + 1)), ppf.Plan(2 * N, T, synth.hamming_sinc(2 * N, T)),
                  ppf.Plan(N, T, h, "c16")):
        st, handle = ppf.ppf_stream_restore(other.handle, np.frombuffer(state, np.uint8).ctypes.data, len(state))
        assert st == 1 and not handle
    buf = np.frombuffer(state, np.uint8).copy()
    st, _ = ppf.ppf_stream_restore(plan.handle, buf.ctypes.data, len(state) - 1)
    assert st == 1
    bad = buf.copy()
    bad[0] ^= 0xFF  # magic
    assert ppf.ppf_stream_restore(plan.handle, bad.ctypes.data, len(bad))[0] == 1
    bad = buf.copy()
    bad[24:32] = np.frombuffer(np.int64(5 * N).tobytes(), np.uint8)  # pushed inconsistent with held
    assert ppf.ppf_stream_restore(plan.handle, bad.ctypes.data, len(bad))[0] == 1
    # a save into a buffer that is too small
    s3 = ppf.Stream(plan)
    s3.push(torch.from_numpy(x[:N]).to("cuda"))
    small = np.empty(HEADER + N * 8 - 1, np.uint8)
    assert ppf.ppf_stream_save(s3.handle, small.ctypes.data, small.size) == 1
    s3.close()
