"""ctypes binding of libppf.so (declared in include/ppf.h).

Argument marshalling only: every step of the polyphase filter bank runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.  If the
library is missing or cannot be loaded, every call raises; there is no CPU
fallback.

Low-level functions carry the C names (``ppf_plan_create``, ``ppf_execute``,
``ppf_execute_host``, ``ppf_stream_open``, ``ppf_stream_push``,
``ppf_stream_close`` ...).  ``Plan`` and ``Stream`` wrap them for torch tensors.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# PPF_LIBRARY selects another build of the same library (the tests point it
# at the bounds-checked build, libppf_checked.so)
LIB_PATH = os.environ.get("PPF_LIBRARY") or os.path.join(HERE, "libppf.so")

PPF_OK = 0
STATUS = {0: "PPF_OK", 1: "PPF_ERR_INVALID_ARG", 2: "PPF_ERR_UNSUPPORTED", 3: "PPF_ERR_MISALIGNED",
          4: "PPF_ERR_OUT_OF_MEMORY", 5: "PPF_ERR_CUDA", 6: "PPF_ERR_TIMEOUT", 7: "PPF_ERR_BUSY"}
DTYPES = {"c32": 0, "c16": 1, "ci8": 2}
SAMPLE_BYTES = {"c32": 8, "c16": 4, "ci8": 2}
FLAG_FIR_ONLY = 1
FLAG_GENERIC = 2
FLAG_OUT_F16 = 4

#: every entry point declared in include/ppf.h
EXPORTS = ("ppf_plan_create", "ppf_plan_destroy", "ppf_execute", "ppf_execute_host",
           "ppf_stream_open", "ppf_stream_push", "ppf_stream_position", "ppf_stream_close",
           "ppf_stream_state_bytes", "ppf_stream_save", "ppf_stream_restore",
           "ppf_status_string", "ppf_plan_kernel_name", "ppf_launch_count", "ppf_variant_count",
           "ppf_variant_name", "ppf_execute_noalloc", "ppf_batch_create", "ppf_batch_execute",
           "ppf_batch_launches", "ppf_batch_destroy", "ppf_server_create", "ppf_server_admit",
           "ppf_server_release", "ppf_server_submit", "ppf_server_submit_many", "ppf_server_tick", "ppf_server_position",
           "ppf_server_info", "ppf_server_graph_ticks", "ppf_server_destroy", "ppf_design_coeffs", "ppf_check_timeout",
           "ppf_check_violations", "ppf_fma_peak")


class PPFJob(ctypes.Structure):
    """ppf_job_t: one stream of a batch."""
    _fields_ = [("plan", ctypes.c_void_p), ("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p),
                ("n_spectra", ctypes.c_int64)]


BATCH_GRAPH = 1
BATCH_PER_KERNEL = 2


class PPFError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}")
        self.status = status


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libppf.so and declare its signatures (no GPU needed for loading)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_1411_3656_gb300.build.build()")
        lib = ctypes.CDLL(p)
        vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        sig = {
            "ppf_plan_create": ([ctypes.POINTER(vp), i32, i32, ctypes.POINTER(ctypes.c_float), i32,
                                 ctypes.c_uint], i32),
            "ppf_plan_destroy": ([vp], i32),
            "ppf_execute": ([vp, vp, vp, i64, vp], i32),
            "ppf_execute_host": ([vp, vp, vp, i64, vp], i32),
            "ppf_stream_open": ([vp, ctypes.POINTER(vp)], i32),
            "ppf_stream_push": ([vp, vp, i64, vp, i64, ctypes.POINTER(i64), vp], i32),
            "ppf_stream_position": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64)], i32),
            "ppf_stream_close": ([vp], i32),
            "ppf_stream_state_bytes": ([vp, ctypes.POINTER(ctypes.c_size_t)], i32),
            "ppf_stream_save": ([vp, vp, ctypes.c_size_t], i32),
            "ppf_stream_restore": ([vp, vp, ctypes.c_size_t, ctypes.POINTER(vp), vp], i32),
            "ppf_status_string": ([i32], ctypes.c_char_p),
            "ppf_plan_kernel_name": ([vp], ctypes.c_char_p),
            "ppf_launch_count": ([], i64),
            "ppf_variant_count": ([i32, i32, i32], i32),
            "ppf_variant_name": ([i32, i32, i32, i32], ctypes.c_char_p),
            "ppf_execute_noalloc": ([i32, i32, i32, vp, vp, vp, i64, vp], i32),
            "ppf_batch_create": ([ctypes.POINTER(vp), ctypes.POINTER(PPFJob), i32, ctypes.c_uint], i32),
            "ppf_batch_execute": ([vp, vp], i32),
            "ppf_batch_launches": ([vp], i32),
            "ppf_batch_destroy": ([vp], i32),
            "ppf_server_create": ([ctypes.POINTER(vp), i32, ctypes.c_size_t], i32),
            "ppf_server_admit": ([vp, vp, i64, ctypes.POINTER(i32)], i32),
            "ppf_server_release": ([vp, i32], i32),
            "ppf_server_submit": ([vp, i32, vp, i64, vp, i64], i32),
            "ppf_server_submit_many": ([vp, i32, vp, vp, vp, vp, vp, vp], i32),
            "ppf_server_tick": ([vp, vp, ctypes.POINTER(i32)], i32),
            "ppf_server_position": ([vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)], i32),
            "ppf_server_info": ([vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
            "ppf_server_graph_ticks": ([vp], i64),
            "ppf_server_destroy": ([vp], i32),
            "ppf_design_coeffs": ([i32, i32, i32, ctypes.c_double, ctypes.POINTER(ctypes.c_float)], i32),
            "ppf_check_timeout": ([ctypes.c_uint, vp], i32),
            "ppf_check_violations": ([i32], i64),
            "ppf_fma_peak": ([i32, i32, vp, ctypes.POINTER(ctypes.c_double)], i32),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        if path is None:
            _lib = lib
        return lib


def _check(status: int, where: str):
    if status != PPF_OK:
        raise PPFError(status, where)


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# -- C-named entry points ----------------------------------------------------

def ppf_plan_create(N: int, T: int, h, dtype: str = "c32", flags: int = 0) -> int:
    import numpy as np
    hh = np.ascontiguousarray(np.asarray(h, dtype=np.float32).reshape(-1))
    if hh.size != N * T:
        raise ValueError("h must hold N*T coefficients")
    out = ctypes.c_void_p()
    st = load().ppf_plan_create(ctypes.byref(out), int(N), int(T),
                                hh.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), DTYPES[dtype], int(flags))
    _check(st, "ppf_plan_create")
    return out.value


def ppf_plan_destroy(plan: int):
    _check(load().ppf_plan_destroy(plan), "ppf_plan_destroy")


def ppf_execute(plan: int, d_in: int, d_out: int, n_spectra: int, stream: int = 0) -> int:
    return load().ppf_execute(plan, d_in, d_out, int(n_spectra), stream)


def ppf_execute_host(plan: int, h_in: int, h_out: int, n_spectra: int, stream: int = 0) -> int:
    return load().ppf_execute_host(plan, h_in, h_out, int(n_spectra), stream)


def ppf_stream_open(plan: int) -> int:
    out = ctypes.c_void_p()
    _check(load().ppf_stream_open(plan, ctypes.byref(out)), "ppf_stream_open")
    return out.value


def ppf_stream_push(stream_obj: int, d_chunk: int, n_samples: int, d_out: int, capacity: int,
                    cuda_stream: int = 0):
    n = ctypes.c_int64(0)
    st = load().ppf_stream_push(stream_obj, d_chunk, int(n_samples), d_out, int(capacity),
                                ctypes.byref(n), cuda_stream)
    return st, n.value


def ppf_stream_position(stream_obj: int):
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().ppf_stream_position(stream_obj, ctypes.byref(a), ctypes.byref(b)), "ppf_stream_position")
    return a.value, b.value


def ppf_stream_close(stream_obj: int):
    _check(load().ppf_stream_close(stream_obj), "ppf_stream_close")


def ppf_stream_state_bytes(stream_obj: int) -> int:
    n = ctypes.c_size_t(0)
    _check(load().ppf_stream_state_bytes(stream_obj, ctypes.byref(n)), "ppf_stream_state_bytes")
    return n.value


def ppf_stream_save(stream_obj: int, h_state: int, capacity: int) -> int:
    return load().ppf_stream_save(stream_obj, h_state, int(capacity))


def ppf_stream_restore(plan: int, h_state: int, nbytes: int, cuda_stream: int = 0):
    out = ctypes.c_void_p()
    st = load().ppf_stream_restore(plan, h_state, int(nbytes), ctypes.byref(out), cuda_stream)
    return st, out.value


def ppf_status_string(status: int) -> str:
    return load().ppf_status_string(int(status)).decode()


def ppf_plan_kernel_name(plan: int) -> str:
    r = load().ppf_plan_kernel_name(plan)
    return r.decode() if r else ""


def ppf_launch_count() -> int:
    return int(load().ppf_launch_count())


def ppf_variant_count(N: int, T: int, dtype: str = "c32") -> int:
    return int(load().ppf_variant_count(int(N), int(T), DTYPES[dtype]))


def ppf_variant_name(N: int, T: int, dtype: str, i: int) -> str | None:
    r = load().ppf_variant_name(int(N), int(T), DTYPES[dtype], int(i))
    return r.decode() if r else None


def ppf_execute_noalloc(N: int, T: int, dtype: str, d_h: int, d_in: int, d_out: int, n_spectra: int,
                        stream: int = 0) -> int:
    """No-allocation PPF (see include/ppf.h): coefficients as a device FP32 array."""
    return load().ppf_execute_noalloc(int(N), int(T), DTYPES[dtype], d_h, d_in, d_out, int(n_spectra), stream)


def ppf_check_timeout(limit_us: int = 1000, stream=None) -> int:
    """Run the device bounded-wait self-check; returns the status (PPF_ERR_TIMEOUT expected)."""
    return load().ppf_check_timeout(int(limit_us), _stream_ptr(stream))


def ppf_fma_peak(blocks: int, iters: int, stream=None):
    """Enqueue the FP32 packed-FMA probe; returns (status, scalar FMA lanes the launch executes)."""
    n = ctypes.c_double(0.0)
    st = load().ppf_fma_peak(int(blocks), int(iters), _stream_ptr(stream), ctypes.byref(n))
    return st, n.value


WINDOWS = {"hamming": 0, "kaiser": 1}


def ppf_design_coeffs(N: int, T: int, window: str = "kaiser", beta: float = 8.0):
    """Windowed-sinc prototype filter h[t*N + c] (float32 numpy array of N*T)."""
    import numpy as np
    if window not in WINDOWS:
        raise ValueError(f"window must be one of {sorted(WINDOWS)}")
    h = np.empty(max(0, int(N) * int(T)), dtype=np.float32)
    st = load().ppf_design_coeffs(int(N), int(T), WINDOWS[window], float(beta),
                                  h.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    _check(st, "ppf_design_coeffs")
    return h


def flag_variant(i: int) -> int:
    """PPF_FLAG_VARIANT(i): force specialised kernel variant i."""
    return ((int(i) + 1) & 0xFF) << 8


# -- torch-facing wrappers -----------------------------------------------------

def dtype_of(x) -> str:
    """Storage name of a torch input tensor: complex64 -> c32; float16 [...,2] -> c16; int8 [...,2] -> ci8."""
    import torch
    if x.dtype == torch.complex64:
        return "c32"
    if x.dtype == torch.float16:
        return "c16"
    if x.dtype == torch.int8:
        return "ci8"
    raise TypeError(f"unsupported input dtype {x.dtype}")


def n_samples_of(x) -> int:
    import torch
    if x.dtype == torch.complex64:
        return x.numel()
    return x.numel() // 2


class Plan:
    """A PPF plan: N channels, T taps, coefficients h[t*N + c] (float32)."""

    def __init__(self, N: int, T: int, h, dtype: str = "c32", flags: int = 0):
        self.N, self.T, self.dtype, self.flags = int(N), int(T), dtype, int(flags)
        self.handle = ppf_plan_create(N, T, h, dtype, flags)

    @property
    def kernel(self) -> str:
        return ppf_plan_kernel_name(self.handle)

    def close(self):
        if self.handle:
            ppf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def n_spectra(self, x) -> int:
        return max(0, n_samples_of(x) // self.N - self.T + 1)

    @property
    def out_f16(self) -> bool:
        return bool(self.flags & FLAG_OUT_F16)

    def execute(self, x, out=None, n_spectra: int | None = None, stream=None):
        """Run the PPF on device tensor ``x``; returns complex64 [n_spectra, N],
        or float16 [n_spectra, N, 2] (I, Q) for a plan made with FLAG_OUT_F16."""
        import torch
        if dtype_of(x) != self.dtype:
            raise TypeError(f"plan expects {self.dtype} input, got {dtype_of(x)}")
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("input must be a contiguous CUDA tensor")
        S = self.n_spectra(x) if n_spectra is None else int(n_spectra)
        if n_samples_of(x) < (S + self.T - 1) * self.N and S > 0:
            raise ValueError("input too short for n_spectra")
        if self.out_f16:
            if out is None:
                out = torch.empty((S, self.N, 2), dtype=torch.float16, device=x.device)
            elif out.numel() < 2 * S * self.N or out.dtype != torch.float16 or not out.is_contiguous():
                raise ValueError("out must be a contiguous float16 tensor of at least n_spectra*N*2")
        elif out is None:
            out = torch.empty((S, self.N), dtype=torch.complex64, device=x.device)
        elif out.numel() < S * self.N or out.dtype != torch.complex64 or not out.is_contiguous():
            raise ValueError("out must be a contiguous complex64 tensor of at least n_spectra*N")
        st = ppf_execute(self.handle, x.data_ptr(), out.data_ptr(), S, _stream_ptr(stream))
        _check(st, "ppf_execute")
        return out

    __call__ = execute

    def execute_host(self, x_host, out_host=None, n_spectra: int | None = None, stream=None):
        """Host-buffer PPF (copies inside).  ``x_host`` is a CPU tensor (pinned for speed)."""
        import torch
        S = self.n_spectra(x_host) if n_spectra is None else int(n_spectra)
        if out_host is None:
            out_host = torch.empty((S, self.N), dtype=torch.complex64, pin_memory=x_host.is_pinned())
        st = ppf_execute_host(self.handle, x_host.data_ptr(), out_host.data_ptr(), S, _stream_ptr(stream))
        _check(st, "ppf_execute_host")
        return out_host


class Stream:
    """Continuous stream on a plan; push chunks, receive completed spectra."""

    def __init__(self, plan: Plan):
        self.plan = plan
        self.handle = ppf_stream_open(plan.handle)

    def push(self, chunk, out=None, stream=None):
        import torch
        n = n_samples_of(chunk) if chunk is not None else 0
        pushed, emitted = ppf_stream_position(self.handle)
        total = pushed + n
        fresh = max(0, total // self.plan.N - self.plan.T + 1) - emitted
        if out is None:
            dev = chunk.device if chunk is not None else torch.device("cuda")
            out = torch.empty((max(fresh, 0), self.plan.N), dtype=torch.complex64, device=dev)
        cap = out.numel() // self.plan.N
        st, got = ppf_stream_push(self.handle, chunk.data_ptr() if n else 0, n,
                                  out.data_ptr() if out.numel() else 0, cap, _stream_ptr(stream))
        _check(st, "ppf_stream_push")
        return out[:got]

    @property
    def position(self):
        return ppf_stream_position(self.handle)

    def save(self) -> bytes:
        """The stream's state (position and held samples) as bytes; see ppf_stream_save."""
        import numpy as np
        n = ppf_stream_state_bytes(self.handle)
        buf = np.empty(n, dtype=np.uint8)
        _check(ppf_stream_save(self.handle, buf.ctypes.data, n), "ppf_stream_save")
        return buf.tobytes()

    @classmethod
    def restore(cls, plan: "Plan", state: bytes, stream=None) -> "Stream":
        """A new stream on ``plan`` that continues a saved one; see ppf_stream_restore."""
        import numpy as np
        buf = np.frombuffer(state, dtype=np.uint8)
        st, handle = ppf_stream_restore(plan.handle, buf.ctypes.data, buf.size, _stream_ptr(stream))
        _check(st, "ppf_stream_restore")
        obj = cls.__new__(cls)
        obj.plan = plan
        obj.handle = handle
        return obj

    def close(self):
        if self.handle:
            ppf_stream_close(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent streams (jobs) launched together; see ppf_batch_create.

    ``jobs`` is a list of (Plan, input tensor, output tensor, n_spectra).  The
    tensors must stay alive (and at the same addresses) as long as the batch.
    """

    def __init__(self, jobs, graph: bool = False, per_kernel: bool = False):
        self._keep = list(jobs)
        arr = (PPFJob * max(1, len(jobs)))()
        for i, (plan, x, y, n) in enumerate(jobs):
            arr[i] = PPFJob(plan.handle, x.data_ptr(), y.data_ptr(), int(n))
        out = ctypes.c_void_p()
        flags = (BATCH_GRAPH if graph else 0) | (BATCH_PER_KERNEL if per_kernel else 0)
        _check(load().ppf_batch_create(ctypes.byref(out), arr, len(jobs), flags), "ppf_batch_create")
        self.handle = out.value

    @property
    def launches(self) -> int:
        return int(load().ppf_batch_launches(self.handle))

    def execute(self, stream=None):
        _check(load().ppf_batch_execute(self.handle, _stream_ptr(stream)), "ppf_batch_execute")

    __call__ = execute

    def close(self):
        if self.handle:
            _check(load().ppf_batch_destroy(self.handle), "ppf_batch_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching of many streams on one GPU (ppf_server_*)."""

    def __init__(self, max_streams: int, memory_budget_bytes: int):
        out = ctypes.c_void_p()
        _check(load().ppf_server_create(ctypes.byref(out), int(max_streams), int(memory_budget_bytes)),
               "ppf_server_create")
        self.handle = out.value
        self.plans = {}

    def admit(self, plan: Plan, max_chunk_samples: int) -> int:
        """Slot id, or raises PPFError (PPF_ERR_OUT_OF_MEMORY / PPF_ERR_BUSY) when refused."""
        slot = ctypes.c_int(-1)
        _check(load().ppf_server_admit(self.handle, plan.handle, int(max_chunk_samples), ctypes.byref(slot)),
               "ppf_server_admit")
        self.plans[slot.value] = plan
        return slot.value

    def release(self, slot: int):
        _check(load().ppf_server_release(self.handle, int(slot)), "ppf_server_release")
        self.plans.pop(slot, None)

    def expected(self, slot: int, queued: int, n: int) -> int:
        """Spectra a chunk of n samples completes, after `queued` samples already queued."""
        plan = self.plans[slot]
        pushed, _ = self.position(slot)
        a = max(0, (pushed + queued) // plan.N - plan.T + 1)
        b = max(0, (pushed + queued + n) // plan.N - plan.T + 1)
        return b - a

    def submit(self, slot: int, chunk, out, n_samples: int | None = None) -> int:
        n = n_samples_of(chunk) if n_samples is None else int(n_samples)
        cap = out.numel() // self.plans[slot].N if out is not None else 0
        st = load().ppf_server_submit(self.handle, int(slot), chunk.data_ptr() if n else None, n,
                                      out.data_ptr() if (out is not None and out.numel()) else None, cap)
        return st

    def submit_many(self, slots, chunk_ptrs, n_samples, out_ptrs, caps):
        """Queue many chunks in one call; numpy arrays (int32 slots, int64 pointers/sizes).

        Returns the per-chunk status array.
        """
        import numpy as np
        slots = np.ascontiguousarray(slots, dtype=np.int32)
        chunk_ptrs = np.ascontiguousarray(chunk_ptrs, dtype=np.uint64)
        n_samples = np.ascontiguousarray(n_samples, dtype=np.int64)
        out_ptrs = np.ascontiguousarray(out_ptrs, dtype=np.uint64)
        caps = np.ascontiguousarray(caps, dtype=np.int64)
        st = np.zeros(slots.shape[0], dtype=np.int32)
        load().ppf_server_submit_many(self.handle, int(slots.shape[0]), slots.ctypes.data, chunk_ptrs.ctypes.data,
                                      n_samples.ctypes.data, out_ptrs.ctypes.data, caps.ctypes.data,
                                      st.ctypes.data)
        return st

    def tick(self, stream=None) -> int:
        n = ctypes.c_int(0)
        _check(load().ppf_server_tick(self.handle, _stream_ptr(stream), ctypes.byref(n)), "ppf_server_tick")
        return n.value

    def position(self, slot: int):
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(load().ppf_server_position(self.handle, int(slot), ctypes.byref(a), ctypes.byref(b)),
               "ppf_server_position")
        return a.value, b.value

    def info(self):
        r, n, l = ctypes.c_size_t(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(load().ppf_server_info(self.handle, ctypes.byref(r), ctypes.byref(n), ctypes.byref(l)),
               "ppf_server_info")
        return {"reserved_bytes": r.value, "streams": n.value, "last_tick_launches": l.value}

    @property
    def graph_ticks(self) -> int:
        """Ticks that ran as a replay of the server's captured CUDA graph."""
        return int(load().ppf_server_graph_ticks(self.handle))

    def close(self):
        if self.handle:
            _check(load().ppf_server_destroy(self.handle), "ppf_server_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
