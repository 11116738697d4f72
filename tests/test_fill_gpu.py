"""fft_fill_uniform, the on-device generator of the uniform-noise inputs: bit
for bit the values synth.uniform_hash computes on the host, for any slice of
the seeded sequence."""
import numpy as np
import pytest

from paper_1505_08067_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,count,first", [(2, 1, 0), (2, 1000003, 0), (99, 4096, 123457),
                                              (2 ** 63 + 5, 65536, 2 ** 33)])
def test_fill_matches_host_twin(gb, seed, count, first):
    y = torch.full((count,), float("nan"), dtype=torch.complex64, device="cuda")
    gb.fft_fill_uniform(y.data_ptr(), count, seed, first)
    torch.cuda.synchronize()
    ref = synth.uniform_hash(seed, count, first)
    assert np.array_equal(y.cpu().numpy().view(np.uint32), ref.view(np.uint32))


def test_fill_rejects_bad_arguments(gb):
    y = torch.zeros(16, dtype=torch.complex64, device="cuda")
    for ptr, count in ((y.data_ptr() + 4, 4), (0, 4), (y.data_ptr(), -1)):
        with pytest.raises(gb.GbfftError) as e:
            gb.fft_fill_uniform(ptr, count, 1)
        assert e.value.status == gb.FFT_ERR_INVALID_ARG
    gb.fft_fill_uniform(y.data_ptr(), 0, 1)        # nothing to do


def test_device_input_transform_against_oracle(gb, oracle):
    """The benchmark's inputs are generated on the device; the oracle checks
    the transform of such an input from the host twin's values."""
    n, batch = 4096, 256
    x = torch.empty(n * batch, dtype=torch.complex64, device="cuda")
    gb.fft_fill_uniform(x.data_ptr(), n * batch, 2, 0)
    with gb.Plan(n, batch, -1) as p:
        y = p.execute(x)
        torch.cuda.synchronize()
    xh = synth.uniform_hash(2, n * batch).reshape(batch, n)
    idx = np.array([0, 77, batch - 1])
    err = oracle.rel_l2(y.view(batch, n)[torch.from_numpy(idx).cuda()].cpu().numpy(),
                        oracle.fft_select(xh, idx, -1))
    assert np.max(err) <= 1e-6 * np.log2(n)
