"""The counter-based input generator (synth.uniform_hash, the host twin of the
library's on-device fft_fill_uniform), pinned to the published SplitMix64
sequence and checked for the properties the workloads rely on.  CPU only."""
import numpy as np

from paper_1505_08067_gb300 import synth

# The first outputs of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014; the
# values every implementation of the generator reproduces).
SPLITMIX64_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_pinned_to_splitmix64():
    x = synth.uniform_hash(0, 2)           # stream indices 0, 1 (element 0) and 2, 3
    want = [2.0 * (v >> 40) * 2.0 ** -24 - 1.0 for v in SPLITMIX64_SEED0]
    assert x[0].real == np.float32(want[0])
    assert x[0].imag == np.float32(want[1])
    assert x[1].real == np.float32(want[2])


def test_slices_and_range():
    a = synth.uniform_hash(12345, 4096)
    assert np.array_equal(a[1000:3000], synth.uniform_hash(12345, 2000, first=1000))
    assert np.all(np.abs(a.real) <= 1) and np.all(np.abs(a.imag) <= 1)
    assert not np.array_equal(a, synth.uniform_hash(12346, 4096))


def test_uniform_moments():
    x = synth.uniform_hash(2, 1 << 20)
    for part in (x.real, x.imag):
        assert abs(float(part.mean())) < 3e-3
        assert abs(float(part.var()) - 1.0 / 3.0) < 3e-3
    # real and imaginary parts uncorrelated
    assert abs(float(np.mean(x.real * x.imag))) < 3e-3
