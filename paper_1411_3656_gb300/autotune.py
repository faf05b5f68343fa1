"""Autotuner for the fused PPF kernels' tile shapes.

For every (N, T, dtype) it times each compiled variant of the specialised
kernels (``ppf_variant_count`` / ``PPF_FLAG_VARIANT``) on one second of
6.5 GB/s input with CUDA events, and writes the fastest into
``csrc/ppf_tuned.inc``, which ``ppf_select.cu`` compiles in as the default.
An entry whose variant name no longer matches the compiled list is ignored.

    python -m paper_1411_3656_gb300.autotune [--out PATH] [--cells N:T,...] [--dtype c32]
"""
from __future__ import annotations

import argparse
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "csrc", "ppf_tuned.inc")
SWEEP = [(n, t) for n in (128, 256, 512, 1024, 2048, 4096) for t in (4, 8, 16, 32)]


def time_variant(ppf, torch, N, T, dtype, flags, x, y, S, reps=10):
    from paper_1411_3656_gb300 import synth
    plan = ppf.Plan(N, T, synth.hamming_sinc(N, T), dtype, flags)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    for _ in range(3):
        st = ppf.ppf_execute(plan.handle, x.data_ptr(), y.data_ptr(), S, sp)
        if st != 0:
            raise ppf.PPFError(st, "ppf_execute")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        ppf.ppf_execute(plan.handle, x.data_ptr(), y.data_ptr(), S, sp)
    e1.record(stream)
    torch.cuda.synchronize()
    name = plan.kernel
    plan.close()
    return e0.elapsed_time(e1) / reps, name


def reindex_line(ppf, ln: str):
    """Re-resolve an entry's variant index from its name against the compiled
    variant lists (they change when variants are added); None if the name is gone."""
    import re
    m = re.match(r'PPF_TUNED\((\d+), (\d+), (\d+), (\d+), "([^"]+)"\)(.*)', ln)
    if not m:
        return None
    N, T, d, _, name, rest = int(m[1]), int(m[2]), int(m[3]), int(m[4]), m[5], m[6]
    dtype = {v: k for k, v in ppf.DTYPES.items()}[d]
    for i in range(ppf.ppf_variant_count(N, T, dtype)):
        if ppf.ppf_variant_name(N, T, dtype, i) == name:
            return f'PPF_TUNED({N}, {T}, {d}, {i}, "{name}"){rest}'
    return None


def reindex_file(path: str) -> int:
    """Host-only: rewrite a tuned table with every index re-resolved by name."""
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1411_3656_gb300 import build, ppf
    build.build()
    ppf.load()
    head, body = [], []
    for ln in open(path):
        ln = ln.rstrip("\n")
        if ln.startswith("PPF_TUNED("):
            new = reindex_line(ppf, ln)
            if new:
                body.append(new)
        else:
            head.append(ln)
    with open(path, "w") as f:
        for ln in head + body:
            f.write(ln + "\n")
    return len(body)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--json", default="")
    ap.add_argument("--cells", default="")
    ap.add_argument("--dtype", default="c32", choices=("c32", "c16", "ci8"))
    ap.add_argument("--seconds", type=float, default=1.0)
    ap.add_argument("--reindex", action="store_true",
                    help="only re-resolve the table's variant indices by name (no GPU needed)")
    args = ap.parse_args(argv)
    if args.reindex:
        print(f"{reindex_file(args.out)} entries", flush=True)
        return 0

    import numpy as np
    import torch
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1411_3656_gb300 import build, metrics, ppf, synth
    build.build()
    ppf.load()
    cells = SWEEP if not args.cells else [tuple(int(v) for v in c.split(":")) for c in args.cells.split(",")]
    n_total = int(synth.REALTIME_SAMPLES_PER_S * args.seconds)
    bps = metrics.IN_BYTES[args.dtype]
    # contents do not affect timing: random bytes of the right size
    x = torch.randint(-100, 100, (n_total * bps,), dtype=torch.int8, device="cuda")
    if args.dtype == "c32":
        x = (torch.randn(n_total, dtype=torch.complex64, device="cuda"))
    elif args.dtype == "c16":
        x = torch.randn(n_total, 2, dtype=torch.float16, device="cuda")
    else:
        x = x.view(-1, 2)
    y = torch.empty(n_total, dtype=torch.complex64, device="cuda")
    results, lines = [], []
    for N, T in cells:
        S = synth.spectra_for(n_total, N, T)
        nv = ppf.ppf_variant_count(N, T, args.dtype)
        rows = []
        for i in range(nv):
            ms, name = time_variant(ppf, torch, N, T, args.dtype, ppf.flag_variant(i), x, y, S)
            gbs = metrics.algorithmic_bytes(N, T, S, args.dtype) / (ms / 1e3) / 1e9
            rows.append({"variant": i, "name": name, "ms": ms, "GBs": gbs})
        gms, _ = time_variant(ppf, torch, N, T, args.dtype, ppf.FLAG_GENERIC, x, y, S)
        best = min(rows, key=lambda r: r["ms"]) if rows else None
        results.append({"N": N, "T": T, "dtype": args.dtype, "variants": rows, "generic_ms": gms,
                        "best": best})
        if best:
            lines.append(f'PPF_TUNED({N}, {T}, {ppf.DTYPES[args.dtype]}, {best["variant"]}, "{best["name"]}")'
                         f'  // {best["ms"]:.3f} ms, {best["GBs"]:.0f} GB/s')
        print(json.dumps(results[-1]), flush=True)
    old = []
    if os.path.exists(args.out):
        dt = ppf.DTYPES[args.dtype]
        keep = {(N, T) for N, T in cells}
        for ln in open(args.out):
            if ln.startswith("PPF_TUNED("):
                parts = ln[len("PPF_TUNED("):].split(",")
                n, t, d = int(parts[0]), int(parts[1]), int(parts[2])
                if not (d == dt and (n, t) in keep):
                    new = reindex_line(ppf, ln.rstrip("\n"))
                    if new:
                        old.append(new)
    with open(args.out, "w") as f:
        f.write("// Written by paper_1411_3656_gb300/autotune.py on a GB300: fastest variant per\n"
                "// (N, T, dtype) as PPF_TUNED(N, T, dtype, variant index, variant name).\n")
        for ln in old + lines:
            f.write(ln + "\n")
    if args.json:
        with open(args.json, "w") as f:
            json.dump(results, f, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
