"""Checks that pin a batched FFT to facts fixed by mathematics, not by itself.

Each check takes ``fft(x, sign)`` -- a batched transform along the last axis,
sign -1 forward, +1 backward (unnormalised) -- and raises AssertionError on a
violation.  They are applied to the FP64 oracle (test_oracle_pins.py) and to
deliberately broken variants of it (test_oracle_mutants.py), which must each
fail at least one of them.

Sources of truth: the DFT definition of Bergach et al. Sec. 2.1 through its
closed forms (impulse, shifted impulse, tone), Parseval's theorem, linearity,
the shift theorem, the unnormalised inverse (read from "changing the sign of
the exponent", same section), and NumPy's independent pocketfft.
"""
from __future__ import annotations

import numpy as np


def _rand(seed, batch, n):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, (batch, n)) + 1j * rng.uniform(-1, 1, (batch, n))


def _root_table(n, sign):
    """exp(sign 2 pi i j / n) via numpy, with j reduced mod n as an integer."""
    j = np.arange(n)
    ang = 2.0 * np.pi * (j % n) / n
    return np.cos(ang) + sign * 1j * np.sin(ang)


def check_impulse(fft, n, tol=1e-14):
    """delta[j] -> all ones; delta[j - n0] -> w^{n0 k}."""
    x = np.zeros((2, n), complex)
    x[0, 0] = 1.0
    n0 = (n // 3) | 1 if n > 2 else n - 1
    x[1, n0] = 1.0
    X = fft(x, -1)
    assert np.max(np.abs(X[0] - 1.0)) <= tol, "impulse at 0 must map to ones"
    k = np.arange(n)
    expect = _root_table(n, -1)[(n0 * k) % n]
    assert np.max(np.abs(X[1] - expect)) <= tol * max(1, np.log2(n)), \
        "shifted impulse must map to w^(n0 k)"


def check_tone(fft, n, tol=1e-12):
    """exp(+2 pi i k0 j / n) -> n * delta[k - k0] (forward)."""
    k0s = np.unique(np.array([0, 1, n // 2, n - 1, (5 * n) // 7]) % n)
    x = np.stack([_root_table(n, +1)[(k0 * np.arange(n)) % n] for k0 in k0s])
    X = fft(x, -1)
    for row, k0 in zip(X, k0s):
        expect = np.zeros(n, complex)
        expect[k0] = n
        assert np.max(np.abs(row - expect)) <= tol * n, f"tone at {k0} must be n delta"


def check_parseval(fft, n, tol=1e-12):
    x = _rand(11 + n, 3, n)
    X = fft(x, -1)
    lhs = np.sum(np.abs(x) ** 2, axis=-1)
    rhs = np.sum(np.abs(X) ** 2, axis=-1) / n
    assert np.max(np.abs(lhs - rhs) / lhs) <= tol, "Parseval"


def check_linearity(fft, n, tol=1e-12):
    x, y = _rand(21 + n, 2, n)
    a, b = 0.75 - 0.5j, -1.25 + 2.0j
    lhs = fft(np.stack([a * x + b * y]), -1)[0]
    X = fft(np.stack([x, y]), -1)
    rhs = a * X[0] + b * X[1]
    assert np.linalg.norm(lhs - rhs) <= tol * np.linalg.norm(rhs), "linearity"


def check_roundtrip(fft, n, tol=1e-12):
    """backward(forward(x)) = n x with the unnormalised inverse."""
    x = _rand(31 + n, 3, n)
    y = fft(fft(x, -1), +1)
    assert np.linalg.norm(y - n * x) <= tol * n * np.linalg.norm(x), "round trip"


def check_shift(fft, n, tol=1e-12):
    """x[j - s] -> w^{s k} X[k]."""
    x = _rand(41 + n, 1, n)
    s = (n // 5) + 1 if n > 1 else 0
    xs = np.roll(x, s, axis=-1)
    X, Xs = fft(np.concatenate([x, xs]), -1)
    k = np.arange(n)
    expect = _root_table(n, -1)[(s * k) % n] * X
    assert np.linalg.norm(Xs - expect) <= tol * np.linalg.norm(X), "shift theorem"


def check_numpy(fft, n, batch=3, tol=1e-13):
    """Against NumPy's pocketfft (an independent implementation), both signs."""
    x = _rand(51 + n, batch, n)
    f = fft(x, -1)
    fr = np.fft.fft(x, axis=-1)
    b = fft(x, +1)
    br = np.fft.ifft(x, axis=-1) * n
    scale = max(1.0, np.log2(max(n, 2)))
    assert np.linalg.norm(f - fr) <= tol * scale * np.linalg.norm(fr), "forward vs pocketfft"
    assert np.linalg.norm(b - br) <= tol * scale * np.linalg.norm(br), "backward vs pocketfft"


ALL = [check_impulse, check_tone, check_parseval, check_linearity, check_roundtrip,
       check_shift, check_numpy]
