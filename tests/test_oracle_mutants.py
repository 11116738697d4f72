"""The pins must catch plausible mistakes.  Each mutant wraps the FP64 oracle
with one planted error (on the CPU) and must fail at least one pin."""
import numpy as np
import pytest

import pins


def _fails_some_pin(fft, sizes=(1, 2, 8, 64, 1024)):
    for n in sizes:
        for check in pins.ALL:
            try:
                check(fft, n)
            except AssertionError:
                return True
    return False


def _mutants(o):
    def wrong_sign(x, s):            # exponent sign flipped
        return o.fft(x, -s)

    def reversed_output(x, s):       # index k read as (n - k) mod n ... on output order
        y = o.fft(x, s)
        return y[..., ::-1]

    def transposed_operand(x, s):    # input read in bit-reversed/transposed order
        n = x.shape[-1]
        if n < 4:
            return o.fft(x, s)[..., ::-1] * 2
        m = int(np.sqrt(n)) if int(np.sqrt(n)) ** 2 == n else n // 2
        return o.fft(np.asarray(x).reshape(*x.shape[:-1], m, n // m).swapaxes(-1, -2)
                     .reshape(x.shape), s)

    def dropped_term(x, s):          # last input sample ignored
        x = np.array(x, complex)
        x[..., -1] = 0
        return o.fft(x, s)

    def normalised_forward(x, s):    # 1/N applied on the forward side
        y = o.fft(x, s)
        return y / x.shape[-1] if s == -1 else y

    def twiddle_off_by_one(x, s):    # uses w_{2N} instead of w_N in a second half
        n = x.shape[-1]
        y = o.fft(x, s)
        if n >= 4:
            y[..., n // 2:] *= np.exp(s * 1j * np.pi / n)
        return y

    def single_precision(x, s):      # silently computing in FP32
        return o.fft(np.asarray(x, np.complex64), s).astype(np.complex64).astype(complex)

    return [wrong_sign, reversed_output, transposed_operand, dropped_term,
            normalised_forward, twiddle_off_by_one, single_precision]


@pytest.mark.parametrize("idx", range(7))
def test_mutant_is_caught(oracle, idx):
    mutant = _mutants(oracle)[idx]
    assert _fails_some_pin(mutant), f"planted mistake {mutant.__name__} passed every pin"


def test_real_oracle_passes_all(oracle):
    assert not _fails_some_pin(oracle.fft)
