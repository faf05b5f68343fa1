"""The C-ABI library loads and exports every entry point include/ppf.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(ppf_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1411_3656_gb300 import build, ppf
    build.build()
    return ppf.load()


def test_header_declares_entry_points():
    from paper_1411_3656_gb300 import ppf
    assert _declared() == set(ppf.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    from paper_1411_3656_gb300 import ppf
    for code, name in ppf.STATUS.items():
        assert ppf.ppf_status_string(code) == name


def test_unsupported_sizes_rejected_before_any_device_call(lib):
    import ctypes
    import numpy as np
    from paper_1411_3656_gb300 import ppf
    h = np.ones(4096 * 64, dtype=np.float32)
    hp = h.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    out = ctypes.c_void_p()
    for N, T, dt in [(3, 4, 0), (6, 4, 0), (8192, 4, 0), (2, 4, 0), (256, 0, 0), (256, 65, 0),
                     (2, 4, 2), (256, 8, 7)]:
        assert lib.ppf_plan_create(ctypes.byref(out), N, T, hp, dt, 0) == 2, (N, T, dt)
    assert lib.ppf_plan_create(None, 256, 8, hp, 0, 0) == 1
    assert lib.ppf_plan_create(ctypes.byref(out), 256, 8, None, 0, 0) == 1
    assert lib.ppf_plan_destroy(None) == 1
    assert lib.ppf_execute(None, None, None, 1, None) == 1
    assert lib.ppf_stream_push(None, None, 0, None, 0, None, None) == 1
    assert lib.ppf_stream_close(None) == 1
    assert lib.ppf_plan_kernel_name(None) is None
    assert ppf.ppf_launch_count() >= 0


def test_stream_state_and_checker_entry_points_without_a_device(lib):
    """Argument errors of the checkpoint entry points come back before any device
    call; the normal build reports that it has no bounds checks compiled in."""
    import ctypes
    n = ctypes.c_size_t(0)
    buf = (ctypes.c_ubyte * 64)()
    assert lib.ppf_stream_state_bytes(None, ctypes.byref(n)) == 1
    assert lib.ppf_stream_save(None, buf, 64) == 1
    out = ctypes.c_void_p()
    assert lib.ppf_stream_restore(None, buf, 64, ctypes.byref(out), None) == 1
    assert lib.ppf_check_violations(0) == -1


def test_tuned_table_names_compiled_variants(lib):
    """Every entry of the autotuned table (csrc/ppf_tuned.inc) names the compiled
    variant at its index (a stale entry would silently fall back to variant 0)."""
    import re
    from paper_1411_3656_gb300 import ppf
    path = os.path.join(ROOT, "paper_1411_3656_gb300", "csrc", "ppf_tuned.inc")
    dtypes = {v: k for k, v in ppf.DTYPES.items()}
    n = 0
    for ln in open(path):
        m = re.match(r'PPF_TUNED\((\d+), (\d+), (\d+), (\d+), "([^"]+)"\)', ln)
        if not m:
            continue
        N, T, d, i, name = int(m[1]), int(m[2]), int(m[3]), int(m[4]), m[5]
        assert ppf.ppf_variant_name(N, T, dtypes[d], i) == name, ln
        n += 1
    assert n >= 3 * 20


def test_fma_peak_argument_errors_without_a_device(lib):
    """The FP32 probe refuses bad arguments before touching the device."""
    from paper_1411_3656_gb300 import ppf
    bad = {v: k for k, v in ppf.STATUS.items()}["PPF_ERR_INVALID_ARG"]
    for blocks, iters in ((0, 10), (70000, 10), (4, 0), (4, 1 << 25)):
        st, n = ppf.ppf_fma_peak(blocks, iters, 0)
        assert st == bad, (blocks, iters, st)
