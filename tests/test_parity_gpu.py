"""GPU parity: the CUDA kernels, called through the C ABI, against the FP64
oracle on the same seeded inputs.  Tolerance (relative L2 per transform):
1e-6 * log2(N) for the FP32 path (log2(rows*cols) for 2D).  Full-size
workloads are checked on sampled transforms the oracle computes one by one,
plus whole-array invariants."""
import numpy as np
import pytest

from paper_1505_08067_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tol(n):
    return 1e-6 * max(1.0, np.log2(n))


def _run(gb, x_np, shape, direction=-1, out_in_place=False, **opts):
    x = torch.from_numpy(np.ascontiguousarray(x_np)).cuda()
    batch = x_np.shape[0]
    with gb.Plan(shape if len(shape) > 1 else shape[0], batch, direction, **opts) as p:
        if out_in_place:
            y = x.clone()
            p.execute(y, y)
        else:
            y = p.execute(x)
        torch.cuda.synchronize()
    return y.cpu().numpy()


def _compare(oracle, y, x, shape, direction=-1):
    batch = x.shape[0]
    ref = oracle.fft(x, direction) if len(shape) == 1 else oracle.fft2d(x, direction)
    err = oracle.rel_l2(y.reshape(batch, -1), ref.reshape(batch, -1))
    n = int(np.prod(shape))
    assert np.max(err) <= _tol(n), (shape, float(np.max(err)))
    return float(np.max(err))


@pytest.mark.parametrize("logn", range(0, 15))
@pytest.mark.parametrize("batch", [1, 3, 64])
@pytest.mark.parametrize("direction", [-1, 1])
def test_single_pass_sweep(gb, oracle, logn, batch, direction):
    n = 2 ** logn
    x = synth.uniform(1000 + logn, batch, n)
    y = _run(gb, x, (n,), direction)
    _compare(oracle, y, x, (n,), direction)


@pytest.mark.parametrize("logn", range(15, 21))
@pytest.mark.parametrize("direction", [-1, 1])
def test_four_step_sweep(gb, oracle, logn, direction):
    n = 2 ** logn
    batch = max(1, 2 ** 20 // n)
    x = synth.uniform(2000 + logn, batch, n)
    y = _run(gb, x, (n,), direction)
    _compare(oracle, y, x, (n,), direction)


@pytest.mark.parametrize("logn,bmax", [(6, 3), (10, 5), (12, 6), (14, 7), (16, 8), (13, 12)])
def test_forced_splits(gb, oracle, logn, bmax):
    x = synth.uniform(3000 + logn, 5, 2 ** logn)
    y = _run(gb, x, (2 ** logn,), max_block_log2=bmax)
    _compare(oracle, y, x, (2 ** logn,))


def _schedules(total, parts=(1, 2, 3, 4)):
    if total == 0:
        yield []
        return
    for p in parts:
        if p <= total:
            for rest in _schedules(total - p, parts):
                yield [p] + rest


def test_every_radix_schedule_n1024(gb, oracle):
    """All radix-{2,4,8,16} schedules of a 1024-point transform agree."""
    x = synth.uniform(4000, 7, 1024)
    ref = oracle.fft(x)
    worst = 0.0
    scheds = [s for s in _schedules(10) if len(s) <= 8]
    for s in scheds:
        code = 0
        for i, lg in enumerate(s):
            code |= lg << (4 * i)
        y = _run(gb, x, (1024,), schedule=code, radix=1 << max(s))
        worst = max(worst, float(np.max(oracle.rel_l2(y, ref))))
    assert len(scheds) > 100 and worst <= _tol(1024)


@pytest.mark.parametrize("radix", [2, 4, 8, 16])
@pytest.mark.parametrize("logn", [5, 9, 13])
def test_register_radix(gb, oracle, radix, logn):
    x = synth.uniform(4100 + logn, 9, 2 ** logn)
    y = _run(gb, x, (2 ** logn,), radix=radix)
    _compare(oracle, y, x, (2 ** logn,))


@pytest.mark.parametrize("tile", [1, 2, 4, 16, 64])
def test_tiles_ragged_batch(gb, oracle, tile):
    x = synth.uniform(4200, 37, 256)
    _compare(oracle, _run(gb, x, (256,), tile=tile), x, (256,))


@pytest.mark.parametrize("shape", [(2 ** 12,), (2 ** 18,), (64, 32), (4096, 64), (1024, 256)])
def test_in_place(gb, oracle, shape):
    n = int(np.prod(shape))
    x = synth.uniform(4300, 3, n).reshape((3,) + shape)
    y = _run(gb, x, shape, out_in_place=True)
    _compare(oracle, y, x, shape)


@pytest.mark.parametrize("shape", [(8, 16), (16, 8), (1, 64), (64, 1), (1, 1), (256, 512),
                                   (2 ** 14, 4), (4, 2 ** 14)])
@pytest.mark.parametrize("direction", [-1, 1])
def test_2d(gb, oracle, shape, direction):
    n = int(np.prod(shape))
    x = synth.uniform(4400 + n, 2, n).reshape((2,) + shape)
    _compare(oracle, _run(gb, x, shape, direction), x, shape, direction)


def test_tones_closed_form(gb, oracle):
    """A unit tone at bin k0 maps to N at k0: the peak lands exactly there."""
    for n in (256, 4096, 2 ** 14, 2 ** 20):
        batch = 4
        x = synth.tones(4500 + n, batch, n, 1)
        bins = synth.tone_bins(4500 + n, batch, n, 1)[:, 0]
        y = _run(gb, x, (n,))
        assert np.array_equal(np.argmax(np.abs(y), axis=1), bins)
        peak = y[np.arange(batch), bins]
        assert np.max(np.abs(peak - n)) <= 1e-5 * n
        _compare(oracle, y, x, (n,))


@pytest.mark.parametrize("n", [512, 8192, 2 ** 14, 2 ** 22])
def test_multi_tone_closed_form(gb, oracle, n):
    """Four unit tones per transform: the spectrum is N at each tone bin and
    zero elsewhere (closed form of the DFT of a sum of exponentials)."""
    batch = 3
    x = synth.tones(4600 + n, batch, n, 4)
    bins = synth.tone_bins(4600 + n, batch, n, 4)
    y = _run(gb, x, (n,))
    expect = np.zeros((batch, n), dtype=np.complex128)
    for b in range(batch):
        expect[b, bins[b]] = n
    err = np.linalg.norm(y - expect, axis=1) / np.linalg.norm(expect, axis=1)
    assert np.max(err) <= _tol(n), float(np.max(err))
    _compare(oracle, y, x, (n,))


def test_impulse_and_roundtrip(gb, oracle):
    n = 4096
    x = np.zeros((2, n), np.complex64)
    x[0, 0] = 1
    x[1, 17] = 1
    y = _run(gb, x, (n,))
    assert np.max(np.abs(y[0] - 1)) <= 1e-6
    _compare(oracle, y, x, (n,))
    z = synth.uniform(4600, 3, n)
    back = _run(gb, _run(gb, z, (n,)), (n,), +1)
    assert np.max(oracle.rel_l2(back, n * z.astype(np.complex128))) <= 2 * _tol(n)


def test_empty_batch_and_errors(gb):
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    with gb.Plan(8, 0) as p:
        assert p.launch_count == 0
        gb.fft_execute(p.handle, 0, 0)          # batch 0: nothing to do
    with gb.Plan(8, 1) as p:
        with pytest.raises(gb.GbfftError) as e:
            gb.fft_execute(p.handle, x.data_ptr() + 4, x.data_ptr())
        assert e.value.status == gb.FFT_ERR_INVALID_ARG
        h = p.handle
    with pytest.raises(gb.GbfftError) as e:
        gb.fft_plan_create(12, 1)
    assert e.value.status == gb.FFT_ERR_UNSUPPORTED_SIZE
    with pytest.raises(gb.GbfftError) as e:
        gb.fft_plan_create(2 ** 25, 1)
    assert e.value.status == gb.FFT_ERR_UNSUPPORTED_SIZE
    del h


def test_execute_host_matches_device(gb, oracle):
    # 2^22 x 3 and 2^20 x 40 split into several ~32 MiB chunks, each running
    # the staged column and transposing passes on a sub-batch
    for shape, batch in (((4096,), 300), ((2 ** 18,), 6), ((64, 128), 3), ((2 ** 22,), 3),
                         ((2 ** 20,), 40)):
        n = int(np.prod(shape))
        x = synth.uniform(4700 + n, batch, n).reshape((batch,) + shape)
        host_in = torch.from_numpy(x).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        dev_in = torch.empty(host_in.shape, dtype=torch.complex64, device="cuda")
        dev_out = torch.empty_like(dev_in)
        with gb.Plan(shape if len(shape) > 1 else shape[0], batch) as p:
            p.execute_host(host_in, host_out, dev_in, dev_out)
            torch.cuda.synchronize()
            ref = p.execute(dev_in).cpu().numpy()
        assert np.array_equal(host_out.numpy(), ref)
        _compare(oracle, host_out.numpy(), x, shape)


# ------------------------------------------------ full-size workloads ------

def _full(gb, oracle, n, batch, seed, direction=-1, samples=6):
    x_np = synth.uniform(seed, batch, n)
    x = torch.from_numpy(x_np).cuda()
    with gb.Plan(n, batch, direction) as p:
        y = p.execute(x)
        torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    idx = np.unique(np.concatenate([[0, batch - 1], rng.integers(0, batch, samples)]))
    ys = y[torch.from_numpy(idx).cuda()].cpu().numpy()
    ref = oracle.fft_select(x_np, idx, direction)
    err = oracle.rel_l2(ys, ref)
    assert np.max(err) <= _tol(n), (n, batch, float(np.max(err)))
    # whole-array invariant (Parseval): sum |X|^2 = N sum |x|^2
    ex = torch.sum(torch.abs(x.to(torch.complex128)) ** 2).item()
    ey = torch.sum(torch.abs(y.to(torch.complex128)) ** 2).item()
    assert abs(ey / (n * ex) - 1) <= 1e-5


@pytest.mark.parametrize("logn", range(8, 15))
@pytest.mark.parametrize("direction", [-1, 1])
def test_full_size_batched_sweep(gb, oracle, logn, direction):
    """N = 2^8..2^14, N * batch = 2^27 (1 GiB in), as timed by the benchmark."""
    _full(gb, oracle, 2 ** logn, 2 ** (27 - logn), 5000 + logn, direction)


@pytest.mark.parametrize("logn,batch", [(20, 64), (22, 16), (24, 4)])
def test_full_size_multipass(gb, oracle, logn, batch):
    _full(gb, oracle, 2 ** logn, batch, 6000 + logn, samples=1)


def test_two_pass_sub_batches(gb, oracle):
    """N = 2^22 x 65 runs as sub-batches of 64 and 1 transforms sharing one
    sub-batch of workspace: the transforms on both sides of the boundary, and
    the same plan replayed from a CUDA graph."""
    n, batch = 2 ** 22, 65
    x_np = synth.uniform(6500, batch, n)
    x = torch.from_numpy(x_np).cuda()
    with gb.Plan(n, batch, -1) as p:
        assert p.describe()["chunk_batch"] == 64
        assert p.workspace_bytes == 8 * 64 * n
        y = p.execute(x)
        y2 = torch.empty_like(x)
        p.execute_graph(x, y2)
        torch.cuda.synchronize()
    idx = np.array([0, 63, 64])
    ys = y[torch.from_numpy(idx).cuda()].cpu().numpy()
    ref = oracle.fft_select(x_np, idx, -1)
    assert np.max(oracle.rel_l2(ys, ref)) <= _tol(n)
    assert torch.equal(y, y2)


def test_sar_frame(gb, oracle):
    """The 4096 azimuth x 8192 range chirp frame, whole, against the oracle."""
    frame = synth.sar_frame(7000)[None]
    y = _run(gb, frame, (4096, 8192))
    err = _compare(oracle, y, frame, (4096, 8192))
    assert err <= _tol(2 ** 25)


def test_buried_tone_n4096(gb, oracle):
    """N = 4096, batch 32768: uniform noise plus a 1e-3 tone; FP32 path."""
    x, bins = synth.buried_tone(8000, 32768, 4096)
    xt = torch.from_numpy(x).cuda()
    with gb.Plan(4096, 32768) as p:
        y = p.execute(xt)
        torch.cuda.synchronize()
    idx = np.arange(0, 32768, 997)
    ys = y[torch.from_numpy(idx).cuda()].cpu().numpy()
    ref = oracle.fft_select(x, idx)
    assert np.max(oracle.rel_l2(ys, ref)) <= _tol(4096)
    tone_err = np.abs(ys[np.arange(idx.size), bins[idx]] - ref[np.arange(idx.size), bins[idx]])
    assert np.max(tone_err) / (4096 * 1e-3) <= 1e-3


@pytest.mark.parametrize("logn", range(8, 15))
def test_generic_and_specialised_kernels_agree(gb, oracle, logn):
    """The benchmark's batch shapes select compile-time kernels; forcing the
    run-time-parameter kernel on the same plan gives the same transform."""
    n = 2 ** logn
    batch = 2 ** 18 // n
    x = synth.uniform(9000 + logn, batch, n)
    for d in (-1, 1):
        ys = _run(gb, x, (n,), d)
        yg = _run(gb, x, (n,), d, generic=1)
        ref = oracle.fft_select(x, np.arange(0, batch, 7), d)
        for y in (ys, yg):
            assert np.max(oracle.rel_l2(y[::7], ref)) <= _tol(n)
        assert np.max(np.abs(ys - yg)) <= 1e-5 * np.sqrt(n)


@pytest.mark.parametrize("logn", [12, 13, 14])
def test_staged_kernel_and_unaligned_fallback(gb, oracle, logn):
    """Contiguous 2^12..2^14 batches run the TMA-staged kernel when the input
    is 16-byte aligned; an input that is only 8-byte aligned takes the
    register kernel.  An output that is only 8-byte aligned does not change
    the staged kernel's result.  Every combination agrees with the oracle."""
    n = 2 ** logn
    batch = 40
    x_np = synth.uniform(9100 + logn, batch, n)
    buf = torch.zeros(batch * n + 1, dtype=torch.complex64, device="cuda")
    obuf = torch.zeros(batch * n + 1, dtype=torch.complex64, device="cuda")
    staged = []
    # 1 complex64 = 8 bytes: breaks 16-byte alignment
    for shift, oshift in ((0, 0), (1, 0), (0, 1)):
        xin = buf[shift:shift + batch * n]
        xin.copy_(torch.from_numpy(x_np.reshape(-1)))
        out = obuf[oshift:oshift + batch * n]
        out.zero_()
        with gb.Plan(n, batch, variant=2) as p:  # the staged kernel at 2^12 too
            gb.fft_execute(p.handle, xin.data_ptr(), out.data_ptr(),
                           torch.cuda.current_stream().cuda_stream)
            gb.fft_plan_sync_status(p.handle, torch.cuda.current_stream().cuda_stream)
        y = out.view(batch, n).cpu().numpy()
        assert np.max(oracle.rel_l2(y, oracle.fft(x_np))) <= _tol(n), (shift, oshift)
        if shift == 0:
            staged.append(y)
    assert np.array_equal(staged[0], staged[1])


@pytest.mark.parametrize("shape,batch,opts", [((4096, 64), 2, {}), ((2 ** 20,), 2, {"split_log2": 10}),
                                              ((2 ** 20,), 2, {"split_log2": 10, "tile": 8}),
                                              ((2 ** 22,), 1, {"split_log2": 11, "epilogue": 3}),
                                              ((2 ** 24,), 1, {"split_log2": 12, "epilogue": 3}),
                                              ((2 ** 22,), 1, {"split_log2": 11, "epilogue": 4}),
                                              ((2 ** 24,), 1, {"split_log2": 12, "epilogue": 4})])
@pytest.mark.parametrize("variant", [2, 4])
def test_staged_columns_and_unaligned_fallback(gb, oracle, shape, batch, opts, variant):
    """Column passes (2D, four-step first passes with G = 16 / 8 / 4 columns)
    run the staged column kernel from a 16-byte-aligned source (variant 2:
    tiles copied by tensor-map boxes; 4: by per-thread 16-byte row copies) and
    the register kernel from an 8-byte-aligned one; all match the oracle."""
    n = int(np.prod(shape))
    x_np = synth.uniform(9400 + int(np.log2(n)), batch, n)
    buf = torch.zeros(batch * n + 1, dtype=torch.complex64, device="cuda")
    dims = shape if len(shape) > 1 else shape[0]
    for shift in (0, 1):
        xin = buf[shift:shift + batch * n]
        xin.copy_(torch.from_numpy(x_np.reshape(-1)))
        out = torch.empty(batch * n, dtype=torch.complex64, device="cuda")
        with gb.Plan(dims, batch, variant=variant, **opts) as p:
            st = torch.cuda.current_stream().cuda_stream
            gb.fft_execute(p.handle, xin.data_ptr(), out.data_ptr(), st)
            gb.fft_plan_sync_status(p.handle, st)
        y = out.cpu().numpy().reshape(batch, n)
        if len(shape) == 1:
            ref = oracle.fft_select(x_np, np.arange(batch), -1)
        else:
            ref = oracle.fft2d(x_np.reshape((batch,) + shape)).reshape(batch, n)
        assert np.max(oracle.rel_l2(y, ref)) <= _tol(n), (shape, shift)


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("logn", [8, 11, 12, 13, 14])
def test_kernel_variants(gb, oracle, variant, logn):
    """Each contiguous-pass kernel variant, on a batch spanning several waves of
    the persistent grid and a ragged last tile."""
    n = 2 ** logn
    batch = 2 ** 21 // n + 3
    x = synth.uniform(9200 + logn, batch, n)
    for d in (-1, 1):
        y = _run(gb, x, (n,), d, variant=variant)
        idx = np.unique(np.r_[0, batch - 1, np.arange(1, batch, 97)])
        ref = oracle.fft_select(x, idx, d)
        assert np.max(oracle.rel_l2(y[idx], ref)) <= _tol(n)


@pytest.mark.parametrize("shape,batch", [((2 ** 16,), 5), ((2 ** 20,), 2), ((2 ** 22,), 1),
                                         ((512, 1024), 3), ((4096, 8192), 1)])
def test_prefetch_variant_strided_passes(gb, oracle, shape, batch):
    """Variant 3 on two-pass and 2D plans: persistent grids whose strided
    column tiles prefetch the next tile into L2 (a tile count that is not a
    multiple of the grid)."""
    n = int(np.prod(shape))
    x = synth.uniform(9300 + int(np.log2(n)), batch, n).reshape((batch,) + shape)
    for d in (-1, 1):
        y = _run(gb, x, shape, d, variant=3)
        if len(shape) == 1:
            idx = np.unique(np.r_[0, batch - 1])
            ref = oracle.fft_select(x, idx, d)
            assert np.max(oracle.rel_l2(y[idx], ref)) <= _tol(n)
        else:
            ref = oracle.fft2d(x, d)
            assert np.max(oracle.rel_l2(y.reshape(batch, -1), ref.reshape(batch, -1))) <= _tol(n)


@pytest.mark.parametrize("epilogue", [1, 2, 3, 4])
@pytest.mark.parametrize("logn", [16, 20, 22])
def test_four_step_twiddle_sources(gb, oracle, epilogue, logn):
    """The four sources of the four-step twiddle w_N^{n2 k1} (two small tables,
    one full table, sincospi of the exact angle, factored into a per-butterfly
    base and powers of a step) agree with the oracle."""
    n = 2 ** logn
    batch = max(1, 2 ** 22 // n)
    x = synth.uniform(9300 + logn, batch, n)
    for d in (-1, 1):
        y = _run(gb, x, (n,), d, epilogue=epilogue)
        idx = np.unique([0, batch - 1])
        assert np.max(oracle.rel_l2(y[idx], oracle.fft_select(x, idx, d))) <= _tol(n)


@pytest.mark.parametrize("shape,batch", [((1024,), 2048), ((2 ** 14,), 128), ((2 ** 20,), 4),
                                         ((256, 512), 2)])
def test_autotuned_plans(gb, oracle, shape, batch):
    """Autotuned plans: the report carries the stage-cost model (single pass)
    and the timed candidates; the chosen plan is correct; a second plan of the
    same shape reuses the choice."""
    n = int(np.prod(shape))
    x = synth.uniform(9400 + n, batch, n).reshape((batch,) + shape)
    arg = shape if len(shape) > 1 else shape[0]
    with gb.Plan(arg, batch, -1, autotune=1) as p:
        rep = p.describe()["tuning"]
        y = p.execute(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
    assert len(rep["candidates"]) >= 2
    assert all(c["ms"] > 0 for c in rep["candidates"] if c["ms"] >= 0)
    if len(shape) == 1 and n <= 2 ** 14:
        sched = rep["model"]["schedule"]
        assert int(np.prod(sched)) == n and rep["model"]["cost_ns_per_element"] > 0
    idx = np.unique([0, batch // 2, batch - 1])
    yr = y.cpu().numpy().reshape(batch, -1)[idx]
    ref = (oracle.fft(x[idx]) if len(shape) == 1 else oracle.fft2d(x[idx])).reshape(len(idx), -1)
    assert np.max(oracle.rel_l2(yr, ref)) <= _tol(n)
    with gb.Plan(arg, batch, -1, autotune=1) as p2:
        assert "cached" in p2.describe()["tuning"]


@pytest.mark.parametrize("shape,batch", [((1024,), 64), ((2 ** 18,), 3), ((64, 128), 2)])
def test_graph_execution_matches(gb, oracle, shape, batch):
    """fft_execute_graph: captured once per (in, out), replayed; identical to
    fft_execute and correct after the buffers' contents change."""
    n = int(np.prod(shape))
    x_np = synth.uniform(9600 + n, batch, n).reshape((batch,) + shape)
    x = torch.from_numpy(x_np).cuda()
    y1 = torch.empty_like(x)
    with gb.Plan(shape if len(shape) > 1 else shape[0], batch) as p:
        ref = p.execute(x)
        for _ in range(3):
            p.execute_graph(x, y1)
        torch.cuda.synchronize()
        assert torch.equal(ref, y1)
        x.mul_(-1)                                 # new contents, same buffers: replay
        p.execute_graph(x, y1)
        torch.cuda.synchronize()
        assert torch.equal(-ref, y1)


@pytest.mark.parametrize("shape,batch,kernels", [
    ((256,), 2 ** 19, ["compile_time"]), ((2048,), 2 ** 16, ["compile_time"]),
    ((4096,), 2 ** 15, ["compile_time"]), ((8192,), 2 ** 14, ["staged"]), ((16384,), 2 ** 13, ["staged"]),
    ((2 ** 20,), 4, ["staged", "staged"]), ((2 ** 22,), 1, ["staged", "staged"]),
    ((4096, 8192), 1, ["staged", "staged"]), ((512,), 2 ** 18, ["compile_time"]),
    ((512,), 3, ["generic"])])
def test_kernel_selection(gb, shape, batch, kernels):
    """The benchmarked shapes bind the intended kernels (2^12 the register
    kernel, 2^13 and 2^14 the staged one); a small batch whose tile has no
    compiled shape (4 transforms of 512 points) runs the generic kernel."""
    with gb.Plan(shape if len(shape) > 1 else shape[0], batch) as p:
        got = [k["kernel"] for k in p.describe()["kernels"]]
    assert got == kernels, got


def test_kernel_selection_conv_and_tc(gb):
    h = torch.ones(8192, dtype=torch.complex64, device="cuda")
    ha = torch.ones(4096 * 8192, dtype=torch.complex64, device="cuda")
    with gb.ConvPlan((4096, 8192), 1, [(ha, 8192, 1.0), (h, 1, 1.0)]) as p:
        ks = p.describe()["kernels"]
    assert [k["kernel"] for k in ks] == ["staged", "staged"] and all(k["conv"] for k in ks)
    with gb.Plan(4096, 64, -1, gb.FFT_PREC_TC_BF16) as p:
        ks = p.describe()["kernels"]
    assert ks[0]["kernel"] == "tensor_core_tcgen05" and ks[0]["persistent_grid"] > 0
    assert ks[0]["ctas_per_sm"] >= 1
    with gb.Plan(4096, 64, -1, gb.FFT_PREC_TC_BF16, variant=1) as p:
        ks = p.describe()["kernels"]
    assert ks[0]["kernel"] == "tensor_core_warp_mma" and ks[0]["persistent_grid"] > 0


def test_execute_argument_errors(gb):
    """Run-time argument checks of the execute entry points: null or
    misaligned device pointers, null host buffers, a description buffer that
    is too small.  Each returns FFT_ERR_INVALID_ARG and leaves the plan usable."""
    x = torch.zeros(2 * 1024, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    hx = torch.zeros(2 * 1024, dtype=torch.complex64).pin_memory()
    with gb.Plan(1024, 2) as p:
        for args in ((0, y.data_ptr()), (x.data_ptr(), 0), (x.data_ptr() + 4, y.data_ptr()),
                     (x.data_ptr(), y.data_ptr() + 2)):
            for fn in (gb.fft_execute, gb.fft_execute_graph):
                with pytest.raises(gb.GbfftError) as e:
                    fn(p.handle, *args)
                assert e.value.status == gb.FFT_ERR_INVALID_ARG
        with pytest.raises(gb.GbfftError) as e:
            gb.fft_execute_host(p.handle, 0, hx.data_ptr(), x.data_ptr(), y.data_ptr())
        assert e.value.status == gb.FFT_ERR_INVALID_ARG
        import ctypes
        buf = ctypes.create_string_buffer(16)
        st = gb.load().fft_plan_describe(p.handle, buf, len(buf))
        assert st == gb.FFT_ERR_INVALID_ARG and len(buf.value) == 15
        p.execute(x, y)                      # still usable
        gb.fft_plan_sync_status(p.handle)
        torch.cuda.synchronize()
