"""Checks that pin fast convolution (matched filtering) to facts fixed by
mathematics, not by the oracle itself.

A convolution plan computes ``scale * IDFT(H . DFT(x))`` per line, IDFT
unnormalised (Bergach et al. Sec. 2.1 conventions).  The convolution theorem
turns that into sums that need no transform at all:

  - with ``H = DFT(c)`` and ``scale = 1/N``: the circular convolution
    ``y[n] = sum_m x[m] c[(n - m) mod N]``;
  - with ``H = conj(DFT(s))`` and ``scale = 1/N``: the circular
    cross-correlation ``r[n] = sum_m x[(m + n) mod N] conj(s[m])`` -- the
    matched filter of the SAR range / azimuth compression step (Sec. 2.2),
    whose output for an echo of ``s`` delayed by d peaks at n = d with the
    value sum |s|^2.

The spectra H are computed here by the DFT matrix written out in NumPy, and
the expected outputs by the sums above, element by element.  Each check takes
the function under test and raises AssertionError on a violation.
"""
from __future__ import annotations

import numpy as np


def _rand(seed, *shape):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)


def dft_matrix(n):
    """W[k, j] = exp(-2 pi i jk / n), the exponent reduced as an integer."""
    jk = np.outer(np.arange(n), np.arange(n)) % n
    return np.exp(-2j * np.pi * jk / n)


def spectrum(c):
    """DFT of each row of c (or of c itself) by the matrix product."""
    c = np.asarray(c, complex)
    return c @ dft_matrix(c.shape[-1]).T


def circ_conv(x, c):
    """y[..., n] = sum_m x[..., m] c[..., (n - m) mod N], term by term."""
    x = np.asarray(x, complex)
    c = np.asarray(c, complex)
    n = x.shape[-1]
    m = np.arange(n)
    y = np.zeros(np.broadcast_shapes(x.shape, c.shape), complex)
    for k in range(n):
        y[..., k] = np.sum(x * c[..., (k - m) % n], axis=-1)
    return y


def circ_corr(x, s):
    """r[..., n] = sum_m x[..., (m + n) mod N] conj(s[..., m])."""
    x = np.asarray(x, complex)
    s = np.asarray(s, complex)
    n = x.shape[-1]
    m = np.arange(n)
    r = np.zeros(np.broadcast_shapes(x.shape, s.shape), complex)
    for k in range(n):
        r[..., k] = np.sum(x[..., (m + k) % n] * np.conj(s), axis=-1)
    return r


def lfm(n, length, bandwidth_frac=0.8):
    """Linear FM chirp of `length` samples sweeping bandwidth_frac of the
    sampling rate, zero-padded to n."""
    t = np.arange(length) - length / 2
    k = bandwidth_frac / length  # chirp rate, cycles / sample^2
    s = np.zeros(n, complex)
    s[:length] = np.exp(1j * np.pi * k * t * t)
    return s


def _close(y, ref, tol, what):
    err = np.max(np.abs(np.asarray(y) - ref)) / max(1e-300, np.max(np.abs(ref)))
    assert err <= tol, f"{what}: max error {err:.3e} > {tol:.1e}"


def check_convolution(conv, n, tol=1e-12):
    """Shared filter, H = DFT(c), scale 1/N: circular convolution with c."""
    x = _rand(11 + n, 3, n)
    c = _rand(12 + n, n)
    _close(conv(x, spectrum(c), 1.0 / n), circ_conv(x, c), tol, f"convolution n={n}")


def check_matched_filter(conv, n, tol=1e-12):
    """H = conj(DFT(s)): circular cross-correlation with s, and an echo of s
    delayed by d compresses to a peak of sum |s|^2 at d."""
    s = lfm(n, max(1, (3 * n) // 4))
    x = _rand(13 + n, 2, n)
    h = np.conj(spectrum(s))
    _close(conv(x, h, 1.0 / n), circ_corr(x, s), tol, f"matched filter n={n}")
    d = (5 * n) // 7
    echo = np.roll(s, d)[None, :]
    y = conv(echo, h, 1.0 / n)[0]
    energy = float(np.sum(np.abs(s) ** 2))
    assert abs(y[d] - energy) <= tol * energy * 10, f"peak value {y[d]} != {energy}"
    if n >= 8:
        assert int(np.argmax(np.abs(y))) == d, "compressed echo does not peak at its delay"


def check_per_line(conv, n, tol=1e-12):
    """One filter per line (rows of h), and scale 1: N times the circular
    convolution of each line with its own kernel."""
    x = _rand(14 + n, 3, n)
    c = _rand(15 + n, 3, n)
    _close(conv(x, spectrum(c), 1.0), n * circ_conv(x, c), tol, f"per-line filters n={n}")


def conv2d_reference(x, c_rows, c_cols):
    """Rows convolved with c_rows (one kernel or one per row), then columns
    with c_cols (one kernel, or one per column given as c_cols[:, col])."""
    y = circ_conv(x, c_rows)
    yt = np.swapaxes(y, -1, -2)
    ct = c_cols if np.ndim(c_cols) == 1 else np.asarray(c_cols).T
    return np.swapaxes(circ_conv(yt, ct), -1, -2)


def check_conv2d_separable(conv2d, rows, cols, tol=1e-12):
    """Shared filters: the 2D circular convolution with the separable kernel
    c_cols[r] * c_rows[c], summed over the whole frame term by term."""
    x = _rand(16 + rows, 2, rows, cols)
    c_r = _rand(17 + cols, cols)
    c_a = _rand(18 + rows, rows)
    y = conv2d(x, spectrum(c_r), 1.0 / cols, spectrum(c_a), 1.0 / rows)
    ref = np.zeros_like(x)
    r_i = np.arange(rows)[:, None]
    c_i = np.arange(cols)[None, :]
    for r in range(rows):
        for c in range(cols):
            k = c_a[(r - r_i) % rows] * c_r[(c - c_i) % cols]
            ref[..., r, c] = np.sum(x * k, axis=(-2, -1))
    _close(y, ref, tol, f"2D separable {rows}x{cols}")


def check_conv2d_per_line(conv2d, rows, cols, tol=1e-12):
    """Per-row range filters (row r's in row r) and per-column azimuth filters
    laid out like the frame (column c's filter in column c)."""
    x = _rand(19 + rows, 2, rows, cols)
    c_r = _rand(20 + cols, rows, cols)       # kernel of row r: c_r[r]
    c_a = _rand(21 + rows, rows, cols)       # kernel of column c: c_a[:, c]
    h_r = spectrum(c_r)
    h_a = spectrum(c_a.T).T                  # spectrum of each column, in column layout
    y = conv2d(x, h_r, 1.0 / cols, h_a, 1.0 / rows)
    _close(y, conv2d_reference(x, c_r, c_a), tol, f"2D per-line {rows}x{cols}")


LINE_CHECKS = [check_convolution, check_matched_filter, check_per_line]
FRAME_CHECKS = [check_conv2d_separable, check_conv2d_per_line]
