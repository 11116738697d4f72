"""GPU parity of the fast-convolution plans (matched filtering; SAR range and
azimuth compression) through the C ABI against the FP64 oracle.  Tolerance
(relative L2 per line, or per frame): 2e-6 * log2(N), twice the single-FFT
bound, since each line goes through a forward and an inverse transform."""
import ctypes

import numpy as np
import pytest

from paper_1505_08067_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tol(n):
    return 2e-6 * max(1.0, np.log2(n))


def _filters(oracle, shape, batch, per_line, seed):
    """Filter spectra as the oracle's FP64 DFT of seeded kernels (complex64)."""
    if len(shape) == 1:
        n = shape[0]
        c = synth.uniform(seed, batch if per_line[0] else 1, n)
        h = oracle.fft(c).astype(np.complex64)
        return [(h if per_line[0] else h[0], batch if per_line[0] else 1, 1.0 / n)]
    rows, cols = shape
    cr = synth.uniform(seed, rows if per_line[1] else 1, cols)
    hr = oracle.fft(cr).astype(np.complex64)
    ca = synth.uniform(seed + 1, cols if per_line[0] else 1, rows)
    ha = oracle.fft(ca).astype(np.complex64)
    return [(np.ascontiguousarray(ha.T) if per_line[0] else ha[0], cols if per_line[0] else 1,
             1.0 / rows),
            (hr if per_line[1] else hr[0], rows if per_line[1] else 1, 1.0 / cols)]


def _reference(oracle, x, shape, filters):
    if len(shape) == 1:
        h, _, sc = filters[0]
        return oracle.conv(x, h.astype(np.complex128), sc)
    (ha, _, sa), (hr, _, sr) = filters
    return oracle.conv2d(x, hr.astype(np.complex128), sr, ha.astype(np.complex128), sa)


def _gpu_conv(gb, x_np, shape, filters, in_place=False, graph=False, **opts):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    hs = [(torch.from_numpy(np.ascontiguousarray(h)).cuda(), lines, sc) for h, lines, sc in filters]
    n = shape if len(shape) > 1 else shape[0]
    with gb.ConvPlan(n, x_np.shape[0], hs, **opts) as p:
        if in_place:
            y = x.clone()
            p.execute(y, y)
        elif graph:
            y = torch.empty_like(x)
            for _ in range(2):
                p.execute_graph(x, y)
        else:
            y = p.execute(x)
        torch.cuda.synchronize()
        desc = p.describe()
    return y.cpu().numpy(), desc


def _check(gb, oracle, shape, batch, per_line=(False, False), seed=21, **kw):
    n = int(np.prod(shape))
    x = synth.uniform(seed, batch, n).reshape((batch,) + tuple(shape))
    filters = _filters(oracle, shape, batch, per_line, seed + 100)
    y, desc = _gpu_conv(gb, x, shape, filters, **kw)
    ref = _reference(oracle, x, shape, filters)
    err = oracle.rel_l2(y.reshape(batch, -1), ref.reshape(batch, -1))
    assert np.max(err) <= _tol(max(shape)), (shape, batch, per_line, float(np.max(err)))
    return desc


@pytest.mark.parametrize("logn", range(1, 15))
@pytest.mark.parametrize("batch", [1, 5])
@pytest.mark.parametrize("per_line", [False, True])
def test_conv_lines(gb, oracle, logn, batch, per_line):
    _check(gb, oracle, (2 ** logn,), batch, (per_line, False))


@pytest.mark.parametrize("logn", [12, 13, 14])
def test_conv_specialised_and_generic(gb, oracle, logn):
    n = 2 ** logn
    _check(gb, oracle, (n,), 2 ** 17 // n)
    _check(gb, oracle, (n,), 2 ** 17 // n, generic=1)


@pytest.mark.parametrize("shape", [(2, 2), (8, 16), (16, 8), (64, 128), (4, 8192), (4096, 8)])
@pytest.mark.parametrize("per_line", [(False, False), (True, True), (True, False), (False, True)])
def test_conv_frames(gb, oracle, shape, per_line):
    _check(gb, oracle, shape, 2, per_line)


@pytest.mark.parametrize("shape,batch,per_line", [((8192,), 700, (True, False)),
                                                  ((4096, 8192), 1, (True, False)),
                                                  ((1024, 512), 3, (True, True))])
def test_conv_prefetch_variant(gb, oracle, shape, batch, per_line):
    """Persistent grid with L2 prefetch of the next tile (variant 3)."""
    _check(gb, oracle, shape, batch, per_line, variant=3)


@pytest.mark.parametrize("variant", [0, 1])
def test_conv_azimuth_staged_filters(gb, oracle, variant):
    """4096-row frames with one filter per column: the staged column kernel
    copies each tile's filters into shared memory after its data (variant 0;
    the first pass's kernel kind is reported as staged), the register kernel
    reads them from global memory (variant 1); both against the oracle, in
    place and from a replayed graph too."""
    desc = _check(gb, oracle, (4096, 64), 3, (True, False), variant=variant)
    kinds = [k["kernel"] for k in desc["kernels"]]
    assert kinds[1] == ("staged" if variant == 0 else "compile_time"), kinds
    _check(gb, oracle, (4096, 32), 2, (True, True), variant=variant, in_place=True)
    _check(gb, oracle, (4096, 16), 1, (True, False), variant=variant, graph=True)


def test_conv_azimuth_filter_not_16_byte_aligned(gb, oracle):
    """A per-column filter frame that starts 8 bytes off a 16-byte boundary
    cannot be copied by tensor-map boxes: the staged kernel reads it from
    global memory instead, with the same result."""
    rows, cols, batch = 4096, 32, 2
    x = synth.uniform(77, batch, rows * cols).reshape(batch, rows, cols)
    filters = _filters(oracle, (rows, cols), batch, (True, False), 177)
    ref = _reference(oracle, x, (rows, cols), filters)
    xt = torch.from_numpy(x).cuda()
    ha = torch.from_numpy(np.ascontiguousarray(filters[0][0]).reshape(-1)).cuda()
    hbuf = torch.zeros(ha.numel() + 1, dtype=torch.complex64, device="cuda")
    hbuf[1:].copy_(ha)
    hr = torch.from_numpy(np.ascontiguousarray(filters[1][0])).cuda()
    outs = []
    for h in (ha, hbuf[1:]):
        with gb.ConvPlan((rows, cols), batch, [(h, cols, filters[0][2]), (hr, 1, filters[1][2])]) as p:
            y = p.execute(xt)
            torch.cuda.synchronize()
        outs.append(y)
        err = oracle.rel_l2(y.cpu().numpy().reshape(batch, -1), ref.reshape(batch, -1))
        assert np.max(err) <= _tol(rows), float(np.max(err))
    assert torch.allclose(outs[0], outs[1], rtol=0, atol=1e-5 * float(torch.max(torch.abs(outs[0]))))


def test_conv_in_place_and_graph(gb, oracle):
    _check(gb, oracle, (256, 512), 2, (True, False), in_place=True)
    _check(gb, oracle, (1024,), 33, (True, False), graph=True)


@pytest.mark.parametrize("radix,tile", [(4, 0), (8, 2), (2, 4)])
def test_conv_forced_radix_and_tile(gb, oracle, radix, tile):
    _check(gb, oracle, (1024,), 7, (True, False), radix=radix, tile=tile)


def test_conv_host_execution_chunks_per_line_filters(gb, oracle):
    """fft_execute_host splits 1D batches into chunks: per-line filters must
    follow the chunk offsets (8192-point lines, 512 lines per 32 MiB chunk)."""
    n, batch = 8192, 1100
    x = synth.uniform(31, batch, n)
    filters = _filters(oracle, (n,), batch, (True, False), 131)
    h = torch.from_numpy(filters[0][0]).cuda()
    hin = torch.from_numpy(x).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    din = torch.empty(x.shape, dtype=torch.complex64, device="cuda")
    dout = torch.empty_like(din)
    with gb.ConvPlan(n, batch, [(h, batch, 1.0 / n)]) as p:
        p.execute_host(hin, hout, din, dout)
        torch.cuda.synchronize()
    idx = np.array([0, 1, 511, 512, 513, 1023, 1024, 1099])
    ref = oracle.conv(x[idx], filters[0][0][idx].astype(np.complex128), 1.0 / n)
    err = oracle.rel_l2(hout.numpy()[idx], ref)
    assert np.max(err) <= _tol(n), float(np.max(err))


def test_sar_compression_full_frame(gb, oracle):
    """Range then azimuth compression of a 4096 x 8192 raw frame with
    per-range-bin azimuth filters: the whole frame against the oracle, and
    every scatterer compressed to a peak at its own position."""
    rows, cols = 4096, 8192
    frame, rr, az, pos = synth.sar_raw(7, rows, cols)
    hr = np.conj(oracle.fft(rr)).astype(np.complex64)
    ha = np.ascontiguousarray(np.conj(oracle.fft(np.ascontiguousarray(az.T))).T).astype(np.complex64)
    filters = [(ha, cols, 1.0 / rows), (hr, 1, 1.0 / cols)]
    y, desc = _gpu_conv(gb, frame[None], (rows, cols), filters)
    assert len(desc["passes"]) == 2 and all(p["conv"] == 1 for p in desc["passes"])
    ref = _reference(oracle, frame[None], (rows, cols), filters)
    err = oracle.rel_l2(y.reshape(1, -1), ref.reshape(1, -1))
    assert np.max(err) <= _tol(rows * cols), float(np.max(err))
    a = np.abs(y[0])
    med = float(np.median(a))
    for r, c in pos:
        win = a[np.ix_(np.arange(r - 2, r + 3) % rows, np.arange(c - 2, c + 3) % cols)]
        assert win[2, 2] == win.max(), (r, c)
        assert win[2, 2] > 100 * med, (r, c, win[2, 2], med)


def test_conv_empty_batch(gb):
    h = torch.ones(64, dtype=torch.complex64, device="cuda")
    x = torch.empty(0, 64, dtype=torch.complex64, device="cuda")
    with gb.ConvPlan(64, 0, [(h, 1, 1.0)]) as p:
        p.execute(x, torch.empty_like(x))
        assert p.launch_count == 0


def test_conv_argument_errors(gb):
    h = torch.ones(64, dtype=torch.complex64, device="cuda")
    with pytest.raises(gb.GbfftError) as e:
        gb.fft_conv_plan_create((64,), 4, [(None, 1, 1.0)])
    assert e.value.status == gb.FFT_ERR_INVALID_ARG
    host = np.ones(64, np.complex64)
    with pytest.raises(gb.GbfftError) as e:
        gb.fft_conv_plan_create((64,), 4, [(host.ctypes.data, 1, 1.0)])
    assert e.value.status == gb.FFT_ERR_INVALID_ARG and "device" in str(e.value)
    with pytest.raises(gb.GbfftError) as e:
        gb.fft_conv_plan_create((64,), 4, [(h.data_ptr(), 3, 1.0)])
    assert e.value.status == gb.FFT_ERR_INVALID_ARG
    with pytest.raises(gb.GbfftError) as e:
        gb.fft_conv_plan_create((2 ** 15,), 1, [(h.data_ptr(), 1, 1.0)])
    assert e.value.status == gb.FFT_ERR_NOT_IMPLEMENTED
    with pytest.raises(gb.GbfftError) as e:
        gb.fft_conv_plan_create((64,), 4, [(h.data_ptr() + 4, 1, 1.0)])
    assert e.value.status == gb.FFT_ERR_INVALID_ARG
