"""Host model of the shared-memory Stockham passes' addressing (ppf_device.cuh:
fft_radix_r, pad_slot, pad_stride; ppf_ring.cuh: fft_pass_ip).

Each pass reads butterfly j's R inputs at pad_slot(j) + r * pad_stride (the layout
the previous pass wrote), multiplies by its twiddles, takes an R-point DFT and writes
output q at pad_slot((j / NS) * NS * R + j % NS) + q * NS.  The model runs those
index formulas with numpy arithmetic for the padding divisors the kernels use (PD = 1:
one pad slot per 16 elements of a radix-16 first pass; PD = 2: one per 32, the
pipelined gather tiles) and for the radix-32 plans of the warp-specialised tiles
(512 = 32 x 16, 1024 = 32 x 32, one pad slot per 32 elements), and checks that every slot lies inside the row stride, that
no two outputs of a pass share a slot, and that the passes compute numpy's FFT.
Host-only: no GPU.
"""
import numpy as np
import pytest


def plan(N, R0=16, RC=16):
    out, n, p = [], N, 0
    while n > 1:
        cap = R0 if p == 0 else RC
        r = cap if n >= cap else n
        out.append(r)
        n //= r
        p += 1
    return out


def pad_slot(idx, NS, R, PD):
    if NS >= 16 or NS * R < 2:
        return idx
    return idx + NS * (idx // (PD * NS * R))


def pad_stride(NS, R, L, PD):
    if NS >= 16 or NS * R < 2:
        return L
    assert L % (PD * NS * R) == 0
    return L + L // (PD * R)


def row_stride(N, PD, RC=16):
    pad = N // (RC * PD)
    return N + (pad if pad > 2 else 2)


def run_passes(N, PD, RC):
    rng = np.random.default_rng(N + PD + RC)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    RS = row_stride(N, PD, RC)
    radices = plan(N, RC, RC)
    buf = np.zeros(RS, dtype=complex)
    buf[:N] = x                        # the FIR writes the row in natural order
    in_ns, in_r = 0, 1
    ns = 1
    for p, R in enumerate(radices):
        last = p == len(radices) - 1
        new = np.full(RS, np.nan + 0j)
        out = np.zeros(N, dtype=complex)
        written = set()
        L = N // R
        for j in range(N // R):
            if in_ns == 0:
                base, stride = j, L
            else:
                base, stride = pad_slot(j, in_ns, in_r, PD), pad_stride(in_ns, in_r, L, PD)
            slots = [base + r * stride for r in range(R)]
            assert max(slots) < RS
            v = buf[slots].copy()
            k = j % ns
            v = v * np.exp(-2j * np.pi * k * np.arange(R) / (ns * R))   # pass twiddles
            v = np.fft.fft(v)                                            # R-point DFT
            if last:
                for q in range(R):
                    out[j + q * ns] = v[q]
            else:
                o = pad_slot((j // ns) * ns * R + (j % ns), ns, R, PD)
                for q in range(R):
                    s = o + q * ns
                    assert s < RS and s not in written
                    written.add(s)
                    new[s] = v[q]
        if last:
            np.testing.assert_allclose(out, np.fft.fft(x), rtol=0, atol=1e-9 * np.sqrt(N))
        else:
            assert len(written) == N
            buf = new
            in_ns, in_r = ns, R
        ns *= R
    return radices


@pytest.mark.parametrize("N", [256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("PD", [1, 2])
def test_padded_stockham_passes_compute_the_dft(N, PD):
    if PD == 2 and (N // 16) % 32:
        pytest.skip("halved padding needs N/16 to span whole 32-element groups")
    run_passes(N, PD, 16)


@pytest.mark.parametrize("N,radices", [(512, [32, 16]), (1024, [32, 32])])
def test_radix32_plans_two_passes(N, radices):
    assert run_passes(N, 1, 32) == radices


def mul_w32_model(m, a):
    """The device's a * W_32^m (ppf_device.cuh mul_w32 and mul_w16), case by case."""
    C8, S8, R2 = np.cos(np.pi / 8), np.sin(np.pi / 8), np.sqrt(0.5)
    C16, S16, C316, S316 = np.cos(np.pi / 16), np.sin(np.pi / 16), np.cos(3 * np.pi / 16), np.sin(3 * np.pi / 16)
    m &= 31
    if m % 2 == 0:
        m16 = (m >> 1) & 15
        neg = m16 >= 8
        m16 -= 8 if neg else 0
        x, y = a.real, a.imag
        r = {0: (x, y), 1: (x * C8 + y * S8, y * C8 - x * S8), 2: ((x + y) * R2, (y - x) * R2),
             3: (x * S8 + y * C8, y * S8 - x * C8), 4: (y, -x), 5: (-x * S8 + y * C8, -y * S8 - x * C8),
             6: ((y - x) * R2, -(x + y) * R2), 7: (-x * C8 + y * S8, -y * C8 - x * S8)}[m16]
        v = complex(*r)
        return -v if neg else v
    q, rr = m >> 3, m & 7
    c, sn = {1: (C16, S16), 3: (C316, S316), 5: (S316, C316), 7: (S16, C16)}[rr]
    t = complex(a.real * c + a.imag * sn, a.imag * c - a.real * sn)
    for _ in range(q):
        t = complex(t.imag, -t.real)
    return t


def test_w32_twiddle_cases_match_the_root_of_unity():
    a = 0.3 - 1.7j
    for m in range(64):
        assert abs(mul_w32_model(m, a) - a * np.exp(-2j * np.pi * m / 32)) < 1e-12
