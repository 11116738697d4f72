"""FP64 CPU oracle for the batched complex FFT -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this module.  The product path never imports it
and shares no code with it (the arithmetic lives in ``oracle.c``, compiled here
with gcc; nothing of the CUDA library is used).

It computes the DFT exactly as defined in Bergach et al., Sec. 2.1
(``X(k) = sum_n x(n) w_N^{nk}``, ``w_N = exp(-2 pi i / N)``, backward by
flipping the exponent's sign, read here as unnormalised).  ``dft`` evaluates the
definition directly (O(N^2)); ``fft`` / ``fft2d`` use textbook recursive radix-2
decimation in time, which reaches the same sum up to rounding.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FORWARD = -1
BACKWARD = +1


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` beside it (gcc, FP64,
    no FMA contraction so x86 and Arm round the same way)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
           "-D_GNU_SOURCE", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            i64 = ctypes.c_int64
            lib.oracle_dft.argtypes = [dp, dp, i64, ctypes.c_int]
            lib.oracle_fft.argtypes = [dp, dp, i64, i64, ctypes.c_int, ctypes.c_int]
            lib.oracle_fft2d.argtypes = [dp, dp, i64, i64, i64, ctypes.c_int, ctypes.c_int]
            lib.oracle_fft_select.argtypes = [dp, dp, i64, ctypes.POINTER(i64), i64,
                                              ctypes.c_int, ctypes.c_int]
            lib.oracle_unit_root.argtypes = [i64, i64, ctypes.c_int, dp]
            lib.oracle_num_threads.argtypes = [ctypes.c_int]
            for f in (lib.oracle_dft, lib.oracle_fft, lib.oracle_fft2d,
                      lib.oracle_fft_select, lib.oracle_unit_root, lib.oracle_num_threads):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c128(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _check_sign(sign: int) -> None:
    if sign not in (FORWARD, BACKWARD):
        raise ValueError("sign must be -1 (forward) or +1 (backward)")


def dft(x, sign: int = FORWARD) -> np.ndarray:
    """Direct O(N^2) DFT of a 1D sequence (any length >= 1)."""
    _check_sign(sign)
    xi = _c128(x).reshape(-1)
    out = np.empty_like(xi)
    if _load().oracle_dft(_ptr(xi.view(np.float64)), _ptr(out.view(np.float64)),
                          xi.size, sign) != 0:
        raise ValueError("oracle_dft rejected its arguments")
    return out


def fft(x, sign: int = FORWARD, threads: int = 0) -> np.ndarray:
    """Batched 1D FFT along the last axis (power-of-two length)."""
    _check_sign(sign)
    xi = _c128(x)
    n = xi.shape[-1]
    batch = xi.size // n if n else 0
    out = np.empty_like(xi)
    if _load().oracle_fft(_ptr(xi.view(np.float64)), _ptr(out.view(np.float64)),
                          n, batch, sign, threads) != 0:
        raise ValueError("oracle_fft rejected its arguments (length must be 2^k)")
    return out


def fft2d(x, sign: int = FORWARD, threads: int = 0) -> np.ndarray:
    """Batched 2D FFT over the last two axes of row-major frames."""
    _check_sign(sign)
    xi = _c128(x)
    rows, cols = xi.shape[-2], xi.shape[-1]
    batch = xi.size // (rows * cols)
    out = np.empty_like(xi)
    if _load().oracle_fft2d(_ptr(xi.view(np.float64)), _ptr(out.view(np.float64)),
                            rows, cols, batch, sign, threads) != 0:
        raise ValueError("oracle_fft2d rejected its arguments")
    return out


def fft_select(x, indices, sign: int = FORWARD) -> np.ndarray:
    """FFT of selected transforms ``x[indices]`` of a batch ``x`` (batch, n),
    without converting the whole batch to FP64 twice."""
    _check_sign(sign)
    xi = np.asarray(x)
    n = xi.shape[-1]
    idx = np.ascontiguousarray(np.asarray(indices, dtype=np.int64))
    sub = _c128(xi.reshape(-1, n)[idx])
    pos = np.ascontiguousarray(np.arange(idx.size, dtype=np.int64))
    out = np.empty_like(sub)
    if _load().oracle_fft_select(_ptr(sub.view(np.float64)), _ptr(out.view(np.float64)),
                                 n, pos.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 idx.size, sign, 1) != 0:
        raise ValueError("oracle_fft_select rejected its arguments")
    return out


def conv(x, h, scale: float, threads: int = 0) -> np.ndarray:
    """Fast convolution of every line along the last axis, as the library's
    convolution plans define it: ``scale * IDFT(H . DFT(x))`` with the
    unnormalised inverse (exponent sign +1, Sec. 2.1).  ``h`` is the filter
    spectrum, broadcast against ``x`` (shape (n,) for one filter shared by every
    line, or one row per line).  With ``h = DFT(c)`` and ``scale = 1/n`` this is
    the circular convolution of each line with ``c``; with ``h = conj(DFT(s))``
    it is the matched filter of ``s`` (circular cross-correlation), the range /
    azimuth compression step of the SAR processing chain (Sec. 2.2)."""
    X = fft(x, FORWARD, threads)
    Y = X * _c128(h)
    return fft(Y, BACKWARD, threads) * float(scale)


def conv2d(x, h_rows, scale_rows: float, h_cols, scale_cols: float,
           threads: int = 0) -> np.ndarray:
    """Fast convolution of row-major frames (..., rows, cols): every row
    (range line, length cols) with ``h_rows`` first, then every column
    (azimuth line, length rows) with ``h_cols``.  ``h_rows`` is (cols,) or
    (rows, cols) with row r's filter in row r; ``h_cols`` is (rows,) or
    (rows, cols) with column c's filter in column c (frame layout)."""
    y = conv(x, h_rows, scale_rows, threads)
    hc = _c128(h_cols)
    hc = hc if hc.ndim == 1 else hc.T
    yt = np.ascontiguousarray(np.swapaxes(y, -1, -2))
    return np.ascontiguousarray(np.swapaxes(conv(yt, hc, scale_cols, threads), -1, -2))


def unit_root(m: int, n: int, sign: int = FORWARD) -> complex:
    """The oracle's FP64 value of w_n^m (sign -1) or its conjugate (sign +1)."""
    buf = np.zeros(2, dtype=np.float64)
    if _load().oracle_unit_root(m, n, sign, _ptr(buf)) != 0:
        raise ValueError("bad root arguments")
    return complex(buf[0], buf[1])


def num_threads(threads: int = 0) -> int:
    """Threads the oracle uses for a given ``threads`` argument (0 = all cores)."""
    return int(_load().oracle_num_threads(threads))


def rel_l2(y, ref, axis=-1) -> np.ndarray:
    """Relative L2 error ||y - ref|| / ||ref|| per transform (along ``axis``),
    accumulated in FP64."""
    y = np.asarray(y, dtype=np.complex128)
    ref = np.asarray(ref, dtype=np.complex128)
    num = np.sqrt(np.sum(np.abs(y - ref) ** 2, axis=axis))
    den = np.sqrt(np.sum(np.abs(ref) ** 2, axis=axis))
    return num / np.where(den == 0, 1.0, den)
