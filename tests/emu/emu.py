"""Loader for the CPU replay harness (test infrastructure, see emu_harness.cpp)."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_1505_08067_gb300", "csrc")
LIB = os.path.join(HERE, "_emu.so")
SRCS = [os.path.join(HERE, "emu_harness.cpp"), os.path.join(CSRC, "planner.cpp")]
DEPS = SRCS + [os.path.join(CSRC, f) for f in ("fft_core.h", "fft_stage.h", "fft_split.h", "planner.h", "kernel_shapes.h",
                                    "tc_stage.h", "umma_stage.h", "tc_stage.h", "queue_ring.h")] + \
    [os.path.join(ROOT, "include", "gbfft.h")]
_lib = None


class Options(ctypes.Structure):
    _fields_ = [("autotune", ctypes.c_int), ("radix", ctypes.c_int), ("schedule", ctypes.c_uint32),
                ("max_block_log2", ctypes.c_int), ("tile", ctypes.c_int),
                ("generic", ctypes.c_int), ("variant", ctypes.c_int),
                ("epilogue", ctypes.c_int), ("split_log2", ctypes.c_int),
                ("reserved", ctypes.c_int * 4)]


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(p) for p in DEPS):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-shared", "-fPIC",
                        "-Wno-unknown-pragmas", "-I" + CSRC, "-I" + os.path.join(ROOT, "include"),
                        "-o", tmp] + SRCS, check=True)
        os.replace(tmp, LIB)
    lib = ctypes.CDLL(LIB)
    lib.emu_run.restype = ctypes.c_int64
    lib.emu_run.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int64,
                            ctypes.c_int, ctypes.c_int, ctypes.POINTER(Options), ctypes.c_int,
                            ctypes.c_int,
                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t,
                            ctypes.POINTER(ctypes.c_int64)]
    lib.emu_conv_run.restype = ctypes.c_int64
    lib.emu_conv_run.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int64,
                                 ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64),
                                 ctypes.POINTER(Options), ctypes.c_int, ctypes.c_int,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p,
                                 ctypes.c_size_t, ctypes.POINTER(ctypes.c_int64)]
    lib.emu_ring_replay.restype = ctypes.c_int
    lib.emu_ring_replay.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_char_p, ctypes.c_size_t]
    _lib = lib
    return lib


def ring_replay(seed: int, slots: int, jobs: int, exact: bool = False) -> str:
    """Replay the work queue's ring bookkeeping against a model; '' if every
    check held, else the first failure."""
    buf = ctypes.create_string_buffer(256)
    r = load().emu_ring_replay(seed, slots, jobs, 1 if exact else 0, buf, 256)
    return "" if r == 0 else buf.value.decode()


def run(x: np.ndarray, shape, direction=-1, smem_optin=232448, specialised=True, stats=None,
        precision=0, **opts):
    """Replay the planned passes for complex64 input x of shape (batch, *shape).
    With specialised=True a pass whose shape the library compiles with fixed
    parameters replays that instantiation (as the GPU would run it)."""
    lib = load()
    x = np.ascontiguousarray(x, dtype=np.complex64)
    dims = len(shape)
    n = (ctypes.c_int64 * 2)(*shape, *([1] * (2 - dims)))
    batch = x.size // int(np.prod(shape)) if np.prod(shape) else 0
    out = np.zeros_like(x)
    o = Options()
    for k, v in opts.items():
        setattr(o, k, v)
    msg = ctypes.create_string_buffer(512)
    sp = ctypes.c_int64(0)
    nerr = lib.emu_run(n, dims, batch, direction, precision, ctypes.byref(o), smem_optin,
                       1 if specialised else 0, x.ctypes.data, out.ctypes.data, msg, 512,
                       ctypes.byref(sp))
    if stats is not None:
        stats["special_passes"] = sp.value % 1000
        stats["staged_passes"] = sp.value // 1000
    return out, int(nerr), msg.value.decode()


def run_conv(x: np.ndarray, shape, filters, specialised=True, stats=None, smem_optin=232448,
             **opts):
    """Replay a fast-convolution plan: filters = [(h, lines, scale)] per
    dimension (h complex64, laid out as fft_filter_t describes)."""
    lib = load()
    x = np.ascontiguousarray(x, dtype=np.complex64)
    dims = len(shape)
    n = (ctypes.c_int64 * 2)(*shape, *([1] * (2 - dims)))
    batch = x.size // int(np.prod(shape))
    out = np.zeros_like(x)
    hs = [np.ascontiguousarray(f[0], dtype=np.complex64) for f in filters]
    lines = (ctypes.c_int64 * 2)(*[int(f[1]) for f in filters], *([1] * (2 - dims)))
    scale = (ctypes.c_float * 2)(*[float(f[2]) for f in filters], *([1.0] * (2 - dims)))
    ptrs = (ctypes.c_void_p * 2)(*[h.ctypes.data for h in hs], *([None] * (2 - dims)))
    lens = (ctypes.c_int64 * 2)(*[h.size for h in hs], *([0] * (2 - dims)))
    o = Options()
    for k, v in opts.items():
        setattr(o, k, v)
    msg = ctypes.create_string_buffer(512)
    sp = ctypes.c_int64(0)
    nerr = lib.emu_conv_run(n, dims, batch, lines, scale, ptrs, lens, ctypes.byref(o), smem_optin,
                            1 if specialised else 0, x.ctypes.data, out.ctypes.data, msg, 512,
                            ctypes.byref(sp))
    if stats is not None:
        stats["special_passes"] = sp.value % 1000
        stats["staged_passes"] = sp.value // 1000
    return out, int(nerr), msg.value.decode()
