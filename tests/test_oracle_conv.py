"""Pins of the oracle's fast convolution (matched filtering), and planted
mistakes that must each fail one of them.  CPU only."""
import numpy as np
import pytest

import conv_pins


@pytest.mark.parametrize("n", [2, 4, 8, 16, 64, 256])
@pytest.mark.parametrize("check", conv_pins.LINE_CHECKS, ids=lambda c: c.__name__)
def test_oracle_conv_pins(oracle, n, check):
    check(oracle.conv, n)


@pytest.mark.parametrize("rows,cols", [(2, 2), (4, 8), (8, 4), (16, 8)])
@pytest.mark.parametrize("check", conv_pins.FRAME_CHECKS, ids=lambda c: c.__name__)
def test_oracle_conv2d_pins(oracle, rows, cols, check):
    check(oracle.conv2d, rows, cols)


def test_lfm_compression_sidelobes(oracle):
    """Range compression of an LFM echo: the main lobe stands well above every
    sample outside it (pulse compression gain), at the echo's delay."""
    n, length = 1024, 600
    s = conv_pins.lfm(n, length)
    x = np.roll(s, 300)[None, :]
    y = np.abs(oracle.conv(x, np.conj(np.fft.fft(s)), 1.0 / n)[0])
    assert int(np.argmax(y)) == 300
    y[300 - 3:300 + 4] = 0
    assert y.max() < 0.25 * length


def _line_mutants(o):
    def forward_twice(x, h, sc):       # inverse taken with the forward sign
        return o.fft(o.fft(x, -1) * h, -1) * sc

    def scale_dropped(x, h, sc):
        return o.conv(x, h, 1.0)

    def filter_conjugated(x, h, sc):
        return o.conv(x, np.conj(h), sc)

    def shifted_by_one(x, h, sc):
        return np.roll(o.conv(x, h, sc), 1, axis=-1)

    def first_line_filter(x, h, sc):   # per-line filters collapsed to line 0
        h = np.asarray(h)
        return o.conv(x, h if h.ndim == 1 else h[0], sc)

    def single_precision(x, h, sc):
        return o.conv(np.asarray(x, np.complex64), np.asarray(h, np.complex64),
                      sc).astype(np.complex64).astype(complex)

    return [forward_twice, scale_dropped, filter_conjugated, shifted_by_one,
            first_line_filter, single_precision]


def _frame_mutants(o):
    def column_filter_untransposed(x, hr, sr, hc, sc):
        hc = np.asarray(hc)
        y = o.conv(x, hr, sr)
        yt = np.swapaxes(y, -1, -2)
        hh = hc if hc.ndim == 1 else hc.reshape(hc.shape[1], hc.shape[0])
        return np.swapaxes(o.conv(yt, hh, sc), -1, -2)

    def rows_only(x, hr, sr, hc, sc):
        return o.conv(x, hr, sr)

    def row_filters_misindexed(x, hr, sr, hc, sc):  # per-row filters read column-major
        hr = np.asarray(hr)
        hh = hr if hr.ndim == 1 else np.ascontiguousarray(hr.T).reshape(hr.shape)
        return o.conv2d(x, hh, sr, hc, sc)

    return [column_filter_untransposed, rows_only, row_filters_misindexed]


def _caught(fn, checks, sizes):
    for size in sizes:
        for check in checks:
            try:
                check(fn, *size)
            except AssertionError:
                return True
    return False


@pytest.mark.parametrize("idx", range(6))
def test_line_mutant_is_caught(oracle, idx):
    m = _line_mutants(oracle)[idx]
    assert _caught(m, conv_pins.LINE_CHECKS, [(8,), (64,)]), m.__name__


@pytest.mark.parametrize("idx", range(3))
def test_frame_mutant_is_caught(oracle, idx):
    m = _frame_mutants(oracle)[idx]
    assert _caught(m, conv_pins.FRAME_CHECKS, [(4, 8), (8, 4)]), m.__name__


def test_real_oracle_passes(oracle):
    assert not _caught(oracle.conv, conv_pins.LINE_CHECKS, [(8,), (64,)])
    assert not _caught(oracle.conv2d, conv_pins.FRAME_CHECKS, [(4, 8), (8, 4)])
