"""Thin ctypes binding of ``libgbfft.so`` (C ABI in ``include/gbfft.h``).

Argument marshalling only: every transform runs in the library's CUDA kernels.
The functions keep the C names (``fft_plan_create``, ``fft_execute``, ...);
``Plan`` wraps them for torch tensors (torch is used for device memory and
streams only).  If the shared library has not been built the first call raises
``RuntimeError``; there is no other code path.
"""
from __future__ import annotations

import ctypes
import json
import os
from typing import Optional, Sequence

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgbfft.so")

FFT_OK = 0
FFT_ERR_INVALID_ARG = 1
FFT_ERR_UNSUPPORTED_SIZE = 2
FFT_ERR_OUT_OF_MEMORY = 3
FFT_ERR_CUDA = 4
FFT_ERR_TIMEOUT = 5
FFT_ERR_BAD_PLAN = 6
FFT_ERR_NOT_IMPLEMENTED = 7
STATUS_NAMES = {0: "FFT_OK", 1: "FFT_ERR_INVALID_ARG", 2: "FFT_ERR_UNSUPPORTED_SIZE",
                3: "FFT_ERR_OUT_OF_MEMORY", 4: "FFT_ERR_CUDA", 5: "FFT_ERR_TIMEOUT",
                6: "FFT_ERR_BAD_PLAN", 7: "FFT_ERR_NOT_IMPLEMENTED"}
FFT_FORWARD = -1
FFT_INVERSE = +1
FFT_PREC_FP32 = 0
FFT_PREC_TC_FP16 = 1
FFT_PREC_TC_BF16 = 2
FFT_PREC_TC_BF16X3 = 3
FFT_PREC_TC_FP16_C32 = 4  # FP16 tensor-core class with complex32 (FP16 pair) input and output


class GbfftError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class fft_plan_options_t(ctypes.Structure):
    _fields_ = [("autotune", ctypes.c_int), ("radix", ctypes.c_int),
                ("schedule", ctypes.c_uint32), ("max_block_log2", ctypes.c_int),
                ("tile", ctypes.c_int), ("generic", ctypes.c_int),
                ("variant", ctypes.c_int), ("epilogue", ctypes.c_int),
                ("split_log2", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class fft_filter_t(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("lines", ctypes.c_int64), ("scale", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class fft_server_options_t(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_size_t), ("streams", ctypes.c_int),
                ("max_group", ctypes.c_int), ("max_running", ctypes.c_int),
                ("fail_workspace_alloc", ctypes.c_int), ("strict_order", ctypes.c_int),
                ("large_group_log2", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


class fft_job_t(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("n", ctypes.c_int64 * 2), ("batch", ctypes.c_int64),
                ("direction", ctypes.c_int), ("precision", ctypes.c_int),
                ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class fft_job_result_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("latency_ms", ctypes.c_double),
                ("queue_ms", ctypes.c_double)]


class fft_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("groups", ctypes.c_uint64), ("coalesced_jobs", ctypes.c_uint64),
                ("workspace_allocations", ctypes.c_uint64),
                ("peak_bytes_in_flight", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("wall_s", ctypes.c_double), ("gflops", ctypes.c_double),
                ("backfilled_jobs", ctypes.c_uint64), ("host_launch_s", ctypes.c_double),
                ("group_stream_s", ctypes.c_double)]


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_SIGS = {
    "fft_plan_create": [ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.c_int, _i64, ctypes.c_int,
                        ctypes.c_int],
    "fft_plan_create_ex": [ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.c_int, _i64,
                           ctypes.c_int, ctypes.c_int, ctypes.POINTER(fft_plan_options_t)],
    "fft_execute": [_vp, _vp, _vp, _vp],
    "fft_execute_host": [_vp, _vp, _vp, _vp, _vp, _vp],
    "fft_execute_graph": [_vp, _vp, _vp, _vp],
    "fft_execute_noalloc": [_i64, _i64, ctypes.c_int, _vp, _vp, _vp],
    "fft_fill_uniform": [_vp, _i64, ctypes.c_uint64, ctypes.c_uint64, _vp],
    "fft_wait_selftest": [ctypes.c_uint32, ctypes.POINTER(ctypes.c_int)],
    "fft_plan_destroy": [_vp],
    "fft_plan_workspace_bytes": [_vp, ctypes.POINTER(ctypes.c_size_t)],
    "fft_plan_launch_count": [_vp, ctypes.POINTER(ctypes.c_int)],
    "fft_plan_describe": [_vp, ctypes.c_char_p, ctypes.c_size_t],
    "fft_plan_dry_run": [ctypes.POINTER(_i64), ctypes.c_int, _i64, ctypes.c_int, ctypes.c_int,
                         ctypes.POINTER(fft_plan_options_t), ctypes.c_int, ctypes.c_int,
                         ctypes.c_char_p, ctypes.c_size_t],
    "fft_plan_sync_status": [_vp, _vp],
    "fft_conv_plan_create": [ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.c_int, _i64,
                             ctypes.POINTER(fft_filter_t), ctypes.POINTER(fft_plan_options_t)],
    "fft_conv_plan_dry_run": [ctypes.POINTER(_i64), ctypes.c_int, _i64, ctypes.POINTER(fft_filter_t),
                              ctypes.POINTER(fft_plan_options_t), ctypes.c_int, ctypes.c_int,
                              ctypes.c_char_p, ctypes.c_size_t],
    "fft_server_create": [ctypes.POINTER(_vp), ctypes.POINTER(fft_server_options_t)],
    "fft_server_submit": [_vp, ctypes.POINTER(fft_job_t), ctypes.POINTER(ctypes.c_uint64)],
    "fft_server_wait": [_vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(fft_job_result_t)],
    "fft_server_drain": [_vp, ctypes.c_double],
    "fft_server_pause": [_vp, ctypes.c_int],
    "fft_server_stats": [_vp, ctypes.POINTER(fft_server_stats_t)],
    "fft_server_destroy": [_vp],
    "fft_queue_create": [ctypes.POINTER(_vp), _i64, _i64, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "fft_queue_submit": [_vp, _vp, _vp, _i64, ctypes.POINTER(ctypes.c_uint64)],
    "fft_queue_wait": [_vp, ctypes.c_uint64, ctypes.c_double],
    "fft_queue_info": [_vp, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_uint64)],
    "fft_queue_destroy": [_vp],
    "fft_schedule_count": [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                           ctypes.POINTER(ctypes.c_uint64)],
    "fft_schedule_shortest_path": [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_double)],
    "fft_schedule_path_cost": [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                               ctypes.c_int, ctypes.POINTER(ctypes.c_double)],
}


def load():
    """Open libgbfft.so (built by ``paper_1505_08067_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.fft_last_error.argtypes = []
    lib.fft_last_error.restype = ctypes.c_char_p
    lib.fft_bandwidth_bound_gflops.argtypes = [_i64, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double]
    lib.fft_bandwidth_bound_gflops.restype = ctypes.c_double
    _lib = lib
    return lib


def fft_last_error() -> str:
    return load().fft_last_error().decode()


def _check(status: int) -> None:
    if status != FFT_OK:
        raise GbfftError(status, fft_last_error())


def _shape(n) -> tuple:
    return tuple(int(v) for v in (n if isinstance(n, (tuple, list)) else (n,)))


def _options(opts: dict) -> fft_plan_options_t:
    o = fft_plan_options_t()
    for k, v in opts.items():
        if k not in ("autotune", "radix", "schedule", "max_block_log2", "tile", "generic",
                     "variant", "epilogue", "split_log2"):
            raise TypeError(f"unknown plan option {k!r}")
        setattr(o, k, int(v))
    return o


# ------------------------------------------------------------ C-named API --

def fft_plan_create(n, batch: int, direction: int = FFT_FORWARD,
                    precision: int = FFT_PREC_FP32, **options) -> int:
    """Returns the opaque plan handle (an integer)."""
    shape = _shape(n)
    arr = (_i64 * len(shape))(*shape)
    h = _vp()
    if options:
        o = _options(options)
        _check(load().fft_plan_create_ex(ctypes.byref(h), arr, len(shape), int(batch), direction,
                                         precision, ctypes.byref(o)))
    else:
        _check(load().fft_plan_create(ctypes.byref(h), arr, len(shape), int(batch), direction,
                                      precision))
    return h.value


def fft_execute(plan: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().fft_execute(plan, in_ptr, out_ptr, stream))


def fft_execute_graph(plan: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().fft_execute_graph(plan, in_ptr, out_ptr, stream))


def fft_execute_host(plan: int, host_in: int, host_out: int, dev_in: int, dev_out: int,
                     stream: int = 0) -> None:
    _check(load().fft_execute_host(plan, host_in, host_out, dev_in, dev_out, stream))


def fft_execute_noalloc(n: int, batch: int, direction: int, in_ptr: int, out_ptr: int,
                        stream: int = 0) -> None:
    """Plan-free transform that allocates no device memory (see include/gbfft.h)."""
    _check(load().fft_execute_noalloc(int(n), int(batch), direction, in_ptr, out_ptr, stream))


class Queue:
    """Persistent work queue for batched 1D FP32 transforms of one length (see
    fft_queue_* in include/gbfft.h): submit(x, out, batch) returns a ticket,
    wait(ticket) blocks until that job's output is complete."""

    def __init__(self, n: int, max_batch: int, direction: int = FFT_FORWARD, slots: int = 0,
                 blocks: int = 0):
        self.n, self.max_batch = int(n), int(max_batch)
        h = _vp()
        _check(load().fft_queue_create(ctypes.byref(h), self.n, self.max_batch, direction,
                                       int(slots), int(blocks)))
        self.handle: Optional[int] = h.value

    def submit_ptr(self, in_ptr: int, out_ptr: int, batch: int) -> int:
        t = ctypes.c_uint64()
        _check(load().fft_queue_submit(self.handle, in_ptr, out_ptr, int(batch), ctypes.byref(t)))
        return t.value

    def submit(self, x, out, batch: Optional[int] = None) -> int:
        """Queue the transform of CUDA complex64 tensor x into out (batch
        defaults to x.numel() // n); both must stay alive until the job ends."""
        import torch
        for t, name in ((x, "input"), (out, "output")):
            if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.complex64:
                raise TypeError(f"{name} must be a CUDA complex64 tensor")
        b = x.numel() // self.n if batch is None else int(batch)
        if b * self.n > min(x.numel(), out.numel()):
            raise ValueError("batch x n exceeds the tensors")
        return self.submit_ptr(x.data_ptr(), out.data_ptr(), b)

    def wait(self, ticket: int, timeout_s: float = -1.0) -> None:
        _check(load().fft_queue_wait(self.handle, int(ticket), float(timeout_s)))

    def info(self) -> dict:
        launches, completed = _i64(), ctypes.c_uint64()
        _check(load().fft_queue_info(self.handle, ctypes.byref(launches), ctypes.byref(completed)))
        return {"worker_launches": launches.value, "completed": completed.value}

    def close(self) -> None:
        if self.handle:
            _check(load().fft_queue_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fft_fill_uniform(out_ptr: int, count: int, seed: int, first: int = 0, stream: int = 0) -> None:
    """Device buffer out_ptr[0 .. count) <- complex64 values with parts uniform in
    [-1, 1), values first .. first + count - 1 of the seeded counter-based
    sequence (synth.uniform_hash computes the same values on the host)."""
    _check(load().fft_fill_uniform(out_ptr, int(count), int(seed) & (2 ** 64 - 1),
                                   int(first), stream))


def fft_wait_selftest(polls: int) -> int:
    """Run the kernels' bounded mbarrier wait on a barrier nothing completes,
    limited to `polls` polls; 1 if it gave up (the expected result)."""
    g = ctypes.c_int(0)
    _check(load().fft_wait_selftest(ctypes.c_uint32(int(polls) & 0xFFFFFFFF), ctypes.byref(g)))
    return g.value


def fft_plan_destroy(plan: int) -> None:
    _check(load().fft_plan_destroy(plan))


def fft_plan_workspace_bytes(plan: int) -> int:
    v = ctypes.c_size_t()
    _check(load().fft_plan_workspace_bytes(plan, ctypes.byref(v)))
    return v.value


def fft_plan_launch_count(plan: int) -> int:
    v = ctypes.c_int()
    _check(load().fft_plan_launch_count(plan, ctypes.byref(v)))
    return v.value


def fft_plan_describe(plan: int) -> dict:
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().fft_plan_describe(plan, buf, len(buf)))
    return json.loads(buf.value.decode())


def fft_plan_dry_run(n, batch: int, direction: int = FFT_FORWARD, precision: int = FFT_PREC_FP32,
                     sm_count: int = 152, smem_optin_bytes: int = 232448, **options) -> dict:
    shape = _shape(n)
    arr = (_i64 * len(shape))(*shape)
    o = _options(options)
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().fft_plan_dry_run(arr, len(shape), int(batch), direction, precision,
                                   ctypes.byref(o), sm_count, smem_optin_bytes, buf, len(buf)))
    return json.loads(buf.value.decode())


def fft_plan_sync_status(plan: int, stream: int = 0) -> None:
    _check(load().fft_plan_sync_status(plan, stream))


def _filters(filters) -> ctypes.Array:
    """[(device pointer or None, lines, scale)] per dimension -> fft_filter_t[]."""
    arr = (fft_filter_t * max(1, len(filters)))()
    for i, (ptr, lines, scale) in enumerate(filters):
        arr[i].h = ptr
        arr[i].lines = int(lines)
        arr[i].scale = float(scale)
    return arr


def fft_conv_plan_create(n, batch: int, filters, **options) -> int:
    """Fast-convolution plan (include/gbfft.h); filters = [(h_ptr, lines, scale)]
    per dimension.  Returns the plan handle."""
    shape = _shape(n)
    arr = (_i64 * len(shape))(*shape)
    h = _vp()
    o = _options(options) if options else None
    _check(load().fft_conv_plan_create(ctypes.byref(h), arr, len(shape), int(batch),
                                       _filters(filters), ctypes.byref(o) if o else None))
    return h.value


def fft_conv_plan_dry_run(n, batch: int, filters, sm_count: int = 152,
                          smem_optin_bytes: int = 232448, **options) -> dict:
    """Convolution plan description for a described device; filters =
    [(lines, scale)] per dimension."""
    shape = _shape(n)
    arr = (_i64 * len(shape))(*shape)
    o = _options(options)
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().fft_conv_plan_dry_run(arr, len(shape), int(batch),
                                        _filters([(None, l, sc) for l, sc in filters]),
                                        ctypes.byref(o), sm_count, smem_optin_bytes, buf, len(buf)))
    return json.loads(buf.value.decode())


def _cost_arrays(log2n, radix_logs, cost):
    rl = (ctypes.c_int * len(radix_logs))(*radix_logs)
    flat = [float(cost[j][s]) if s < len(cost[j]) else -1.0
            for j in range(len(radix_logs)) for s in range(log2n)]
    return rl, (ctypes.c_double * len(flat))(*flat)


def fft_schedule_count(log2n: int, radix_logs: Sequence[int]) -> int:
    rl = (ctypes.c_int * len(radix_logs))(*radix_logs)
    v = ctypes.c_uint64()
    _check(load().fft_schedule_count(log2n, rl, len(radix_logs), ctypes.byref(v)))
    return v.value


def fft_schedule_shortest_path(log2n: int, radix_logs: Sequence[int], cost):
    """cost[j][s]: cost of radix 2**radix_logs[j] starting at stage s (None/-1 = no edge).
    Returns (list of radices in stage order, total cost)."""
    rl, c = _cost_arrays(log2n, radix_logs, [[-1.0 if v is None else v for v in row] for row in cost])
    path = (ctypes.c_int * 64)()
    ln = ctypes.c_int()
    tot = ctypes.c_double()
    _check(load().fft_schedule_shortest_path(log2n, rl, len(radix_logs), c, path, 64,
                                             ctypes.byref(ln), ctypes.byref(tot)))
    return [1 << path[i] for i in range(ln.value)], tot.value


def fft_schedule_path_cost(log2n: int, radix_logs: Sequence[int], cost, radices: Sequence[int]):
    rl, c = _cost_arrays(log2n, radix_logs, [[-1.0 if v is None else v for v in row] for row in cost])
    logs = [int(r).bit_length() - 1 for r in radices]
    p = (ctypes.c_int * len(logs))(*logs)
    tot = ctypes.c_double()
    _check(load().fft_schedule_path_cost(log2n, rl, len(radix_logs), c, p, len(logs),
                                         ctypes.byref(tot)))
    return tot.value


def fft_bandwidth_bound_gflops(n: int, gbs: float, bytes_per_sample: float = 8.0,
                               passes: float = 1.0) -> float:
    return load().fft_bandwidth_bound_gflops(int(n), gbs, bytes_per_sample, passes)


# ------------------------------------------------------- torch convenience --

def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """A plan for ``batch`` transforms of shape ``n`` (int for 1D, (rows, cols) for 2D)."""

    def __init__(self, n, batch: int, direction: int = FFT_FORWARD,
                 precision: int = FFT_PREC_FP32, **options):
        self.shape = _shape(n)
        self.batch = int(batch)
        self.direction = direction
        self.precision = precision
        self.handle: Optional[int] = fft_plan_create(self.shape, self.batch, direction, precision,
                                                     **options)

    @property
    def elements(self) -> int:
        e = self.batch
        for v in self.shape:
            e *= v
        return e

    def _check_tensor(self, t, name):
        import torch
        want = torch.complex32 if self.precision == FFT_PREC_TC_FP16_C32 else torch.complex64
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != want:
            raise TypeError(f"{name} must be a CUDA {str(want).split('.')[-1]} tensor")
        if not t.is_contiguous() or t.numel() != self.elements:
            raise ValueError(f"{name} must be contiguous with {self.elements} elements")

    def execute(self, x, out=None, stream=None):
        """Enqueue the transform of tensor ``x`` into ``out`` (allocated if None)."""
        import torch
        self._check_tensor(x, "input")
        if out is None:
            out = torch.empty_like(x)
        self._check_tensor(out, "output")
        fft_execute(self.handle, x.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def execute_graph(self, x, out=None, stream=None):
        """Like execute, replayed from a CUDA graph cached for (x, out)."""
        import torch
        self._check_tensor(x, "input")
        if out is None:
            out = torch.empty_like(x)
        self._check_tensor(out, "output")
        fft_execute_graph(self.handle, x.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def execute_host(self, host_in, host_out, dev_in, dev_out, stream=None):
        """Host -> device -> transform -> host, pipelined in chunks (torch tensors)."""
        fft_execute_host(self.handle, host_in.data_ptr(), host_out.data_ptr(), dev_in.data_ptr(),
                         dev_out.data_ptr(), _stream_handle(stream))

    def describe(self) -> dict:
        return fft_plan_describe(self.handle)

    @property
    def workspace_bytes(self) -> int:
        return fft_plan_workspace_bytes(self.handle)

    @property
    def launch_count(self) -> int:
        return fft_plan_launch_count(self.handle)

    def close(self) -> None:
        if self.handle:
            fft_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ConvPlan(Plan):
    """Fast convolution (matched filtering) of ``batch`` lines / frames of
    shape ``n`` with ``filters`` = [(h, lines, scale)] per dimension, h a CUDA
    complex64 tensor holding the filter spectrum (kept alive by the plan).
    ``execute`` computes scale * IDFT(H . DFT(x)) along every dimension."""

    def __init__(self, n, batch: int, filters, **options):
        import torch
        self.shape = _shape(n)
        self.batch = int(batch)
        self.direction = FFT_FORWARD
        self.precision = FFT_PREC_FP32
        self.handle = None
        self.filters = []
        spec = []
        for h, lines, scale in filters:
            if not isinstance(h, torch.Tensor) or not h.is_cuda or h.dtype != torch.complex64:
                raise TypeError("filters must be CUDA complex64 tensors")
            if not h.is_contiguous():
                raise ValueError("filters must be contiguous")
            self.filters.append(h)
            spec.append((h.data_ptr(), lines, scale))
        self.handle = fft_conv_plan_create(self.shape, self.batch, spec, **options)


# ----------------------------------------------------------------- serving --

def fft_server_create(memory_budget_bytes: int = 0, streams: int = 0, max_group: int = 0,
                      max_running: int = 0, fail_workspace_alloc: int = 0,
                      strict_order: int = 0, large_group_log2: int = 0) -> int:
    o = fft_server_options_t(memory_budget_bytes, streams, max_group, max_running,
                             fail_workspace_alloc, strict_order, large_group_log2)
    h = _vp()
    _check(load().fft_server_create(ctypes.byref(h), ctypes.byref(o)))
    return h.value


def fft_server_submit(server: int, n, batch: int, direction: int, precision: int, in_ptr: int,
                      out_ptr: int) -> int:
    shape = _shape(n)
    j = fft_job_t(len(shape), (ctypes.c_int64 * 2)(*shape, *([1] * (2 - len(shape)))), int(batch),
                  direction, precision, in_ptr, out_ptr)
    t = ctypes.c_uint64()
    _check(load().fft_server_submit(server, ctypes.byref(j), ctypes.byref(t)))
    return t.value


def fft_server_wait(server: int, ticket: int, timeout_s: float = -1.0) -> dict:
    """Waits for a job.  Returns its status (FFT_OK or the job's error, or
    FFT_ERR_TIMEOUT if it is still running); raises for a bad ticket/server."""
    r = fft_job_result_t()
    r.status = -1
    st = load().fft_server_wait(server, ticket, timeout_s, ctypes.byref(r))
    if st == FFT_ERR_TIMEOUT:
        return {"status": st, "latency_ms": -1.0, "queue_ms": -1.0}
    if st != FFT_OK and r.status == -1:
        raise GbfftError(st, fft_last_error())
    return {"status": r.status, "latency_ms": r.latency_ms, "queue_ms": r.queue_ms}


def fft_server_pause(server: int, paused: bool) -> None:
    _check(load().fft_server_pause(server, 1 if paused else 0))


def fft_server_drain(server: int, timeout_s: float = -1.0) -> None:
    _check(load().fft_server_drain(server, timeout_s))


def fft_server_stats(server: int) -> dict:
    s = fft_server_stats_t()
    _check(load().fft_server_stats(server, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in fft_server_stats_t._fields_}


def fft_server_destroy(server: int) -> None:
    _check(load().fft_server_destroy(server))
