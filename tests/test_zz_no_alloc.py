"""fft_execute_noalloc, the entry point for callers that may not allocate GPU
memory while they run (e.g. a real-time radar loop that reserves everything at
start-up).  It must give the same transform as the plan-based entry point, call
after call, while keeping its tables and workspace in the library's static
array.  Collected last on purpose: it runs after every other GPU test."""
import numpy as np
import pytest

from paper_1505_08067_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tol(n):
    return 1e-6 * max(1.0, np.log2(n))


def _rel_l2(a, b):
    a = a.astype(np.complex128)
    b = b.astype(np.complex128)
    return np.linalg.norm(a - b, axis=-1) / np.linalg.norm(b, axis=-1)


@pytest.mark.parametrize("n,batch,direction", [
    (2 ** 20, 8, -1),      # two passes, workspace of 2^23 elements: the largest allowed
    (2 ** 16, 5, +1),      # two passes, backward
    (2 ** 22, 2, -1),
    (2 ** 12, 64, -1),     # one pass: only the twiddle tables live in the static array
])
def test_noalloc_matches_plan_entry_point(gb, n, batch, direction):
    x = torch.from_numpy(synth.uniform(70000 + n, batch, n)).cuda()
    with gb.Plan(n, batch, direction) as plan:
        ref = plan.execute(x)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):                      # two calls in a row share the array
        y = torch.full_like(x, float("nan"))
        gb.fft_execute_noalloc(n, batch, direction, x.data_ptr(), y.data_ptr(), stream)
        torch.cuda.synchronize()
        err = _rel_l2(y.cpu().numpy(), ref)
        assert np.max(err) <= _tol(n), (call, float(np.max(err)))


def test_noalloc_rejects_sizes_beyond_its_array(gb):
    x = torch.zeros(2 ** 24, dtype=torch.complex64, device="cuda")
    with pytest.raises(gb.GbfftError) as e:
        gb.fft_execute_noalloc(2 ** 24, 1, -1, x.data_ptr(), x.data_ptr())
    assert e.value.status == gb.FFT_ERR_UNSUPPORTED_SIZE
    with pytest.raises(gb.GbfftError) as e:
        gb.fft_execute_noalloc(2 ** 20, 9, -1, x.data_ptr(), x.data_ptr())
    assert e.value.status == gb.FFT_ERR_UNSUPPORTED_SIZE
    assert "64 MiB" in gb.fft_last_error()
