"""fft_execute_noalloc, the entry point for callers that may not allocate GPU
memory while they run (e.g. a real-time radar loop that reserves everything at
start-up).  It keeps its twiddle tables and two-pass workspace in the
library's static array, so it is checked call after call: against the FP64
oracle at the FP32 tolerance, against the plan-based entry point, and with
shapes that alternate on a non-default stream (each call must rebuild what
the previous one left in the shared array).  The file sorts last so that a
run stopping at the first failure has already run every other GPU test; each
test also passes on its own in a fresh process."""
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


def _noalloc(gb, x, n, batch, direction, stream):
    y = torch.full_like(x, float("nan"))
    gb.fft_execute_noalloc(n, batch, direction, x.data_ptr(), y.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("n,batch,direction", [
    (2 ** 20, 8, -1),      # two passes, workspace of 2^23 elements: the largest allowed
    (2 ** 16, 5, +1),      # two passes, backward
    (2 ** 22, 2, -1),
    (2 ** 12, 64, -1),     # one pass: only the twiddle tables live in the static array
])
def test_noalloc_matches_oracle_and_plan(gb, oracle, n, batch, direction):
    xh = synth.uniform(70000 + n, batch, n)
    x = torch.from_numpy(xh).cuda()
    with gb.Plan(n, batch, direction) as plan:
        ref_plan = plan.execute(x)
    torch.cuda.synchronize()
    ref_plan = ref_plan.cpu().numpy()
    ref = oracle.fft(xh, direction)
    stream = torch.cuda.current_stream()
    for call in range(2):                      # two calls in a row share the array
        y = _noalloc(gb, x, n, batch, direction, stream)
        err = _rel_l2(y, ref)
        assert np.max(err) <= _tol(n), (call, float(np.max(err)))
        assert np.max(_rel_l2(y, ref_plan)) <= _tol(n), call


def test_noalloc_alternating_shapes_on_a_side_stream(gb, oracle):
    """A smaller call after a larger one, a one-pass call between two-pass
    calls and a backward call in between, all on one non-default stream: the
    tables and status word each call leaves behind must not leak into the
    next."""
    side = torch.cuda.Stream()
    shapes = [(2 ** 20, 4, -1), (2 ** 12, 16, -1), (2 ** 16, 8, +1), (2 ** 20, 4, -1),
              (2 ** 12, 16, -1)]
    inputs = {}
    for k, (n, batch, d) in enumerate(shapes):
        if (n, batch) not in inputs:
            xh = synth.uniform(71000 + k, batch, n)
            inputs[(n, batch)] = (xh, torch.from_numpy(xh).cuda())
        xh, x = inputs[(n, batch)]
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            y = _noalloc(gb, x, n, batch, d, side)
        err = _rel_l2(y, oracle.fft(xh, d))
        assert np.max(err) <= _tol(n), (k, n, batch, d, float(np.max(err)))


def test_noalloc_rejects_sizes_beyond_its_array(gb):
    x = torch.zeros(2 ** 24, dtype=torch.complex64, device="cuda")
    with pytest.raises(gb.GbfftError) as e:
        gb.fft_execute_noalloc(2 ** 24, 1, -1, x.data_ptr(), x.data_ptr())
    assert e.value.status == gb.FFT_ERR_UNSUPPORTED_SIZE
    with pytest.raises(gb.GbfftError) as e:
        gb.fft_execute_noalloc(2 ** 20, 9, -1, x.data_ptr(), x.data_ptr())
    assert e.value.status == gb.FFT_ERR_UNSUPPORTED_SIZE
    assert "64 MiB" in gb.fft_last_error()
    with pytest.raises(gb.GbfftError) as e:
        gb.fft_execute_noalloc(2 ** 10, 1, 0, x.data_ptr(), x.data_ptr())
    assert e.value.status == gb.FFT_ERR_INVALID_ARG
