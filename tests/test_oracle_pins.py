"""Pins of the FP64 oracle to facts outside itself (CPU only).

The oracle follows the DFT definition of Bergach et al. Sec. 2.1; these tests
check it against closed forms, invariants, brute force on tiny inputs, exact
symbolic values (sympy) and NumPy's independent pocketfft.
"""
import numpy as np
import pytest

import pins


POW2 = [2 ** e for e in range(0, 13)]


@pytest.mark.parametrize("n", POW2)
@pytest.mark.parametrize("check", pins.ALL, ids=lambda c: c.__name__)
def test_oracle_fft_pins(oracle, n, check):
    check(oracle.fft, n)


@pytest.mark.parametrize("n", [2 ** 16, 2 ** 20])
@pytest.mark.parametrize("check", [pins.check_impulse, pins.check_tone, pins.check_parseval,
                                   pins.check_roundtrip, pins.check_numpy],
                         ids=lambda c: c.__name__)
def test_oracle_fft_pins_large(oracle, n, check):
    check(oracle.fft, n)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8, 12, 16, 31, 64, 100, 256])
def test_dft_matches_pocketfft(oracle, n):
    """The O(N^2) definition, any length, against pocketfft."""
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    for sign, ref in ((-1, np.fft.fft(x)), (+1, np.fft.ifft(x) * n)):
        y = oracle.dft(x, sign)
        assert np.linalg.norm(y - ref) <= 1e-13 * max(1, n) * np.linalg.norm(ref)


@pytest.mark.parametrize("n", [2 ** e for e in range(0, 9)])
def test_fft_equals_brute_force_dft(oracle, n):
    """Recursive radix-2 and the direct sum agree (brute force on tiny sizes)."""
    rng = np.random.default_rng(100 + n)
    x = rng.uniform(-1, 1, (2, n)) + 1j * rng.uniform(-1, 1, (2, n))
    for sign in (-1, +1):
        f = oracle.fft(x, sign)
        for b in range(2):
            d = oracle.dft(x[b], sign)
            assert np.linalg.norm(f[b] - d) <= 1e-13 * np.linalg.norm(d)


def test_exact_symbolic_dft_n8(oracle):
    """DFT of the integers 1..8, exactly (sympy, 30 digits)."""
    sympy = pytest.importorskip("sympy")
    n = 8
    xs = list(range(1, n + 1))
    exact = []
    for k in range(n):
        s = sum(sympy.Integer(xs[j]) * sympy.exp(-2 * sympy.pi * sympy.I * j * k / n)
                for j in range(n))
        v = complex(sympy.N(sympy.expand_complex(s), 30))
        exact.append(v)
    y = oracle.fft(np.array(xs, complex), -1)
    assert np.max(np.abs(y - np.array(exact))) <= 1e-14 * 36


def test_unit_roots(oracle):
    """Quarter turns are exact; other roots match sympy to 1e-16."""
    sympy = pytest.importorskip("sympy")
    for n in (4, 8, 64, 2 ** 24):
        for q, val in enumerate((1, -1j, -1, 1j)):
            assert oracle.unit_root(q * n // 4, n, -1) == val
            assert oracle.unit_root(q * n // 4, n, +1) == np.conj(val)
    for m, n in ((1, 8), (3, 16), (5, 1024), (12345, 2 ** 20), (2 ** 24 - 1, 2 ** 24)):
        ang = 2 * sympy.pi * m / n
        ref = complex(sympy.N(sympy.cos(ang), 30)) - 1j * complex(sympy.N(sympy.sin(ang), 30))
        w = oracle.unit_root(m, n, -1)
        assert abs(w - ref) <= 2.3e-16
        assert oracle.unit_root(m + 7 * n, n, -1) == w          # integer reduction mod n


@pytest.mark.parametrize("rows,cols", [(8, 16), (16, 8), (1, 32), (32, 1), (64, 128)])
def test_fft2d_against_pocketfft(oracle, rows, cols):
    rng = np.random.default_rng(rows * 1000 + cols)
    x = rng.uniform(-1, 1, (2, rows, cols)) + 1j * rng.uniform(-1, 1, (2, rows, cols))
    for sign, ref in ((-1, np.fft.fft2(x)), (+1, np.fft.ifft2(x) * rows * cols)):
        y = oracle.fft2d(x, sign)
        assert np.linalg.norm(y - ref) <= 1e-13 * 8 * np.linalg.norm(ref)


def test_fft2d_closed_forms(oracle):
    """2D impulse -> ones; separable input -> outer product of 1D transforms;
    a 2D tone -> rows*cols at its bin."""
    rows, cols = 16, 32
    x = np.zeros((rows, cols), complex)
    x[0, 0] = 1
    assert np.max(np.abs(oracle.fft2d(x) - 1)) == 0
    rng = np.random.default_rng(7)
    a = rng.standard_normal(rows) + 1j * rng.standard_normal(rows)
    b = rng.standard_normal(cols) + 1j * rng.standard_normal(cols)
    sep = oracle.fft2d(np.outer(a, b))
    outer = np.outer(oracle.fft(a), oracle.fft(b))
    assert np.linalg.norm(sep - outer) <= 1e-13 * np.linalg.norm(outer)
    r0, c0 = 5, 27
    i = np.arange(rows)[:, None]
    j = np.arange(cols)[None, :]
    ang = 2 * np.pi * (((r0 * i) % rows) / rows + ((c0 * j) % cols) / cols)
    tone = np.exp(1j * ang)
    T = oracle.fft2d(tone)
    expect = np.zeros((rows, cols), complex)
    expect[r0, c0] = rows * cols
    assert np.max(np.abs(T - expect)) <= 1e-11 * rows * cols


def test_select_matches_batch(oracle):
    rng = np.random.default_rng(3)
    x = (rng.uniform(-1, 1, (10, 64)) + 1j * rng.uniform(-1, 1, (10, 64))).astype(np.complex64)
    idx = [9, 0, 4]
    full = oracle.fft(x)
    sub = oracle.fft_select(x, idx)
    assert np.array_equal(sub, full[idx])


def test_threads_do_not_change_results(oracle):
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, (37, 256)) + 1j * rng.uniform(-1, 1, (37, 256))
    assert np.array_equal(oracle.fft(x, threads=1), oracle.fft(x, threads=5))


def test_argument_errors(oracle):
    with pytest.raises(ValueError):
        oracle.fft(np.zeros((2, 12), complex))           # not a power of two
    with pytest.raises(ValueError):
        oracle.fft(np.zeros((2, 8), complex), sign=0)
    assert oracle.fft(np.zeros((0, 8), complex)).shape == (0, 8)   # empty batch
