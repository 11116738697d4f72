"""Guard words around every buffer a plan reads or writes: the kernels write
exactly the output's bytes and leave the input of an out-of-place call as it
was.  Each buffer sits inside a larger allocation whose margins (4 KiB on each
side) hold a fixed bit pattern (an FP32 NaN payload no kernel produces); after
the call every margin word is compared, and the input is compared with a copy.

Cases cover each kernel family: register and staged single-pass kernels, the
two-pass and 2D plans (staged column and transposing passes), the fast
convolution (range lines and the staged azimuth columns with per-column
filters), the tcgen05 tensor-core classes (staged 4096-element tiles, 2^13,
2^14, six-step) with complex64 and complex32 storage, in place and out of
place."""
import numpy as np
import pytest

from paper_1505_08067_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MARGIN = 4096  # bytes on each side
PATTERN = 0x7FC0BEEF  # FP32 quiet NaN with a payload


def _guarded(nbytes):
    """A buffer of margin + nbytes + margin bytes, the margins filled with
    PATTERN, and a view of the middle (byte offset MARGIN: 16-byte aligned)."""
    words = (2 * MARGIN + nbytes) // 4
    buf = torch.full((words,), PATTERN, dtype=torch.int32, device="cuda")
    mid = buf.view(torch.uint8)[MARGIN:MARGIN + nbytes]
    return buf, mid


def _margins_intact(buf, nbytes):
    """Both margins still hold PATTERN (nbytes is a multiple of 4)."""
    words = buf.numel()
    lo = buf[:MARGIN // 4]
    hi = buf[(MARGIN + nbytes) // 4:words]
    return bool(torch.all(lo == PATTERN)) and bool(torch.all(hi == PATTERN))


def _run_case(gb, shape, batch, precision=0, in_place=False, conv=None, **opts):
    c32 = precision == 4
    esz = 4 if c32 else 8
    n = int(np.prod(shape))
    nbytes = batch * n * esz
    x_np = synth.uniform(4242 + n + batch, batch, n)
    if c32:
        h16 = np.stack([x_np.real, x_np.imag], axis=-1).astype(np.float16)
        src = torch.from_numpy(np.ascontiguousarray(h16)).view(torch.uint8).reshape(-1).cuda()
    else:
        src = torch.from_numpy(np.ascontiguousarray(x_np)).view(torch.uint8).reshape(-1).cuda()
    ibuf, xin = _guarded(nbytes)
    xin.copy_(src)
    if in_place:
        obuf, yout = ibuf, xin
    else:
        obuf, yout = _guarded(nbytes)
    st = torch.cuda.current_stream().cuda_stream
    arg = tuple(shape) if len(shape) > 1 else shape[0]
    if conv is None:
        plan = gb.Plan(arg, batch, -1, precision, **opts)
    else:
        plan = gb.ConvPlan(arg, batch, conv, **opts)
    with plan as p:
        gb.fft_execute(p.handle, xin.data_ptr(), yout.data_ptr(), st)
        gb.fft_plan_sync_status(p.handle, st)
    torch.cuda.synchronize()
    assert _margins_intact(ibuf, nbytes), "input margins written"
    if not in_place:
        assert _margins_intact(obuf, nbytes), "output margins written"
        assert torch.equal(xin, src), "input of an out-of-place call changed"
    # the output is finite (no element left unwritten with the margin pattern)
    y = yout.view(torch.float16 if c32 else torch.float32)
    assert bool(torch.isfinite(y).all())


@pytest.mark.parametrize("shape,batch", [((1,), 7), ((16,), 33), ((1024,), 129), ((4096,), 65),
                                         ((8192,), 17), ((16384,), 9), ((2 ** 16,), 3),
                                         ((2 ** 20,), 2), ((2 ** 22,), 1), ((2 ** 24,), 1),
                                         ((4096, 64), 2), ((256, 512), 3)])
@pytest.mark.parametrize("in_place", [False, True])
def test_fp32_plans_write_only_their_output(gb, shape, batch, in_place):
    _run_case(gb, shape, batch, in_place=in_place)


@pytest.mark.parametrize("shape,batch", [((4096,), 65), ((8192,), 9), ((16384,), 5), ((2 ** 20,), 1)])
@pytest.mark.parametrize("precision", [1, 2, 3, 4])
def test_tensor_core_plans_write_only_their_output(gb, shape, batch, precision):
    _run_case(gb, shape, batch, precision=precision)
    _run_case(gb, shape, batch, precision=precision, in_place=True)


def test_convolution_plans_write_only_their_output(gb):
    rows, cols = 4096, 64
    ha = torch.ones(rows * cols, dtype=torch.complex64, device="cuda")
    hr = torch.ones(cols, dtype=torch.complex64, device="cuda")
    # per-column azimuth filters (staged by tile) and a shared range filter
    _run_case(gb, (rows, cols), 2, conv=[(ha, cols, 1.0 / rows), (hr, 1, 1.0 / cols)])
    _run_case(gb, (rows, cols), 2, conv=[(ha, cols, 1.0 / rows), (hr, 1, 1.0 / cols)],
              in_place=True)
    h1 = torch.ones(8192, dtype=torch.complex64, device="cuda")
    _run_case(gb, (8192,), 33, conv=[(h1, 1, 1.0 / 8192)])
