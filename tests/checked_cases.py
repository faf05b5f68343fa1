"""Cases run by the bounds-checked build test (tests/test_gpu_checked.py).

Run as a script with PPF_LIBRARY pointing at libppf_checked.so, it runs every
case through that build, requires ppf_check_violations() == 0 after each, and
saves the outputs to the .npz file named on the command line; imported, it
runs the same cases through whatever library is loaded.  Not collected by
pytest (no test_ prefix).
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SWEEP = [(n, t) for n in (256, 512, 1024, 2048, 4096) for t in (4, 8, 16, 32)]
SMALL = [(4, 3), (16, 4), (64, 8), (128, 13), (4096, 64)]


def cases():
    """(name, N, T, dtype, flags-kind, variant index or None)."""
    from paper_1411_3656_gb300 import ppf
    out = []
    for N, T in SWEEP:
        for i in range(ppf.ppf_variant_count(N, T, "c32")):
            out.append((f"{N}x{T}:c32:v{i}", N, T, "c32", "variant", i))
        out.append((f"{N}x{T}:c32:f16out", N, T, "c32", "f16", None))
    for N, T in SMALL:
        out.append((f"{N}x{T}:c32:default", N, T, "c32", "default", None))
        out.append((f"{N}x{T}:c32:generic", N, T, "c32", "generic", None))
    for dt in ("c16", "ci8"):
        for N, T in ((1024, 8), (4096, 16), (256, 32), (4096, 8), (2048, 16), (1024, 32)):
            for i in range(ppf.ppf_variant_count(N, T, dt)):
                out.append((f"{N}x{T}:{dt}:v{i}", N, T, dt, "variant", i))
    return out


def run_case(N, T, dtype, kind, variant, seed):
    import torch
    from paper_1411_3656_gb300 import ppf, synth
    S = max(3, 16384 // N) + 5  # several blocks of every tile and a ragged tail
    x = synth.stream(synth.samples_for(S, N, T), N, seed)
    if dtype == "c16":
        x = synth.to_fp16_iq(x)
    elif dtype == "ci8":
        x = synth.int8_iq(synth.samples_for(S, N, T), seed)
    h = synth.hamming_sinc(N, T)
    flags = {"variant": ppf.flag_variant(variant) if variant is not None else 0, "default": 0,
             "generic": ppf.FLAG_GENERIC, "f16": ppf.FLAG_OUT_F16}[kind]
    plan = ppf.Plan(N, T, h, dtype, flags)
    y = plan(torch.from_numpy(np.ascontiguousarray(x)).to("cuda"), n_spectra=S)
    torch.cuda.synchronize()
    out = y.cpu().numpy()
    name = plan.kernel
    plan.close()
    return out, name


def main(path):
    from paper_1411_3656_gb300 import ppf
    ppf.load()
    assert ppf.load().ppf_check_violations(1) == 0, "the loaded library is not the checked build"
    res = {}
    for k, (name, N, T, dtype, kind, variant) in enumerate(cases()):
        out, kern = run_case(N, T, dtype, kind, variant, 9000 + k)
        v = int(ppf.load().ppf_check_violations(1))
        if v != 0:
            print(f"VIOLATIONS {v} in {name} ({kern})", flush=True)
            return 1
        res[name] = out
    np.savez(path, **res)
    print(f"checked: {len(res)} cases, 0 violations", flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1]))
