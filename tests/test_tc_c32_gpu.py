"""The FP16 tensor-core class with complex32 storage (FFT_PREC_TC_FP16_C32)
against the FP64 oracle.

Input and output are FP16 (re, im) pairs, 4 bytes per element.  The oracle
transforms the FP16 input exactly (every FP16 value is an FP64 value), so the
error measured is the kernel's: the FP16 stages of the FP16 class plus one more
rounding of each output to FP16.  Bound: the FP16 class's 2e-3 relative L2 per
transform."""
import numpy as np
import pytest

from paper_1505_08067_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C32 = 4
TOL = 2e-3


def _fp16_pairs(x):
    """complex128 values rounded to FP16 parts (round to nearest even), as a
    (..., 2) float16 array and as the complex128 values it holds."""
    h = np.stack([x.real, x.imag], axis=-1).astype(np.float16)
    return h, h[..., 0].astype(np.float64) + 1j * h[..., 1].astype(np.float64)


def _to_device(h):
    return torch.from_numpy(np.ascontiguousarray(h)).cuda().view(torch.complex32).reshape(h.shape[:-1])


def _to_numpy(y):
    f = y.reshape(-1).view(torch.float16).float().cpu().numpy().astype(np.float64)
    return (f[0::2] + 1j * f[1::2]).reshape(tuple(y.shape))


def _status(gb, p):
    gb.fft_plan_sync_status(p.handle, torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("logn", range(4, 15))
@pytest.mark.parametrize("direction", [-1, 1])
def test_c32_class(gb, oracle, logn, direction):
    """Every length of the tcgen05 kernel, five full tiles and a ragged one."""
    n = 2 ** logn
    batch = max(4096 // n, 1) * 5 + 3
    h, x = _fp16_pairs(synth.uniform(9900 + n, batch, n))
    xd = _to_device(h)
    with gb.Plan(n, batch, direction, C32) as p:
        y = p.execute(xd)
        _status(gb, p)
    err = oracle.rel_l2(_to_numpy(y), oracle.fft(x, direction))
    assert np.max(err) <= TOL, float(np.max(err))
    # the input buffer is never written
    assert np.array_equal(_to_numpy(xd), x)


@pytest.mark.parametrize("logn", [8, 12, 14])
def test_c32_in_place_and_graph(gb, oracle, logn):
    """in == out, and the graph-replayed launch, give the plain launch's bytes."""
    n = 2 ** logn
    batch = max(4096 // n, 1) * 3 + 1
    h, x = _fp16_pairs(synth.uniform(9950 + logn, batch, n))
    with gb.Plan(n, batch, -1, C32) as p:
        ref = p.execute(_to_device(h))
        xi = _to_device(h)
        p.execute(xi, xi)
        g = p.execute_graph(_to_device(h))
        g2 = p.execute_graph(_to_device(h))
        _status(gb, p)
    a = ref.view(torch.int16)
    assert torch.equal(a, xi.view(torch.int16))
    assert torch.equal(a, g.view(torch.int16)) and torch.equal(a, g2.view(torch.int16))
    err = oracle.rel_l2(_to_numpy(ref), oracle.fft(x, -1))
    assert np.max(err) <= TOL, float(np.max(err))


def test_c32_many_tiles_sampled(gb, oracle):
    """2^24 elements at N = 4096 (many tiles per CTA of the persistent grid),
    sampled transforms against the oracle, the rest against the round trip's
    scale: inverse(forward(x)) = N x within the class's bound."""
    n = 4096
    batch = (1 << 24) // n + 1
    h, x = _fp16_pairs(synth.uniform(9960, batch, n))
    xd = _to_device(h)
    with gb.Plan(n, batch, -1, C32) as f, gb.Plan(n, batch, 1, C32) as b:
        y = f.execute(xd)
        # the inverse's input: the forward output scaled by 1/N (exact in FP16
        # down to its subnormals) keeps the round trip's output near x
        ys = (y.view(torch.float16) * (1.0 / n)).view(torch.complex32)
        z = b.execute(ys)
        _status(gb, f)
        _status(gb, b)
    idx = np.unique(np.concatenate([[0, batch - 1], np.arange(1, batch, 331)]))
    yn = _to_numpy(y.view(torch.float16)[torch.from_numpy(idx).cuda()].view(torch.complex32))
    err = oracle.rel_l2(yn, oracle.fft_select(x, idx, -1))
    assert np.max(err) <= TOL, float(np.max(err))
    zn = _to_numpy(z)
    rt = np.linalg.norm(zn - x, axis=1) / np.linalg.norm(x, axis=1)
    assert np.max(rt) <= 2 * TOL, float(np.max(rt))


def test_c32_host_path(gb, oracle):
    """fft_execute_host moves 4 bytes per element each way."""
    n, batch = 1024, 200
    h, x = _fp16_pairs(synth.uniform(9970, batch, n))
    # FP16 views of the complex32 buffers (execute_host takes addresses only)
    hin = torch.from_numpy(np.ascontiguousarray(h)).reshape(batch, 2 * n).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    din = torch.empty(batch, 2 * n, dtype=torch.float16, device="cuda")
    dout = torch.empty_like(din)
    with gb.Plan(n, batch, -1, C32) as p:
        p.execute_host(hin, hout, din, dout)
        torch.cuda.synchronize()
        _status(gb, p)
        dev = p.execute(din.view(torch.complex32))
        torch.cuda.synchronize()
    assert torch.equal(hout.view(torch.int16), dev.view(torch.float16).cpu().view(torch.int16))
    err = oracle.rel_l2(_to_numpy(hout.view(torch.complex32)), oracle.fft(x, -1))
    assert np.max(err) <= TOL, float(np.max(err))


def test_c32_server_job(gb, oracle):
    """A complex32 job through the serving loop equals the plan's output."""
    n, batch = 2048, 37
    h, x = _fp16_pairs(synth.uniform(9980, batch, n))
    xd = _to_device(h)
    out = torch.empty_like(xd)
    with gb.Plan(n, batch, 1, C32) as p:
        ref = p.execute(xd)
        _status(gb, p)
    srv = gb.fft_server_create(memory_budget_bytes=256 << 20, streams=2)
    try:
        t = gb.fft_server_submit(srv, n, batch, 1, C32, xd.data_ptr(), out.data_ptr())
        r = gb.fft_server_wait(srv, t, 30.0)
        assert r["status"] == 0
        # an address that is not 4-byte aligned is refused at submission
        with pytest.raises(gb.GbfftError):
            gb.fft_server_submit(srv, n, batch, 1, C32, xd.data_ptr() + 2, out.data_ptr())
    finally:
        gb.fft_server_destroy(srv)
    torch.cuda.synchronize()
    assert torch.equal(ref.view(torch.int16), out.view(torch.int16))
    err = oracle.rel_l2(_to_numpy(out), oracle.fft(x, 1))
    assert np.max(err) <= TOL, float(np.max(err))


@pytest.mark.parametrize("logn,direction", [(15, -1), (18, 1), (21, -1), (24, 1)])
def test_c32_six_step(gb, oracle, logn, direction):
    """complex32 storage above 2^14: the six-step plan's transposes and
    workspace carry FP16 pairs too."""
    n = 2 ** logn
    h, x = _fp16_pairs(synth.uniform(9990 + logn, 2, n))
    with gb.Plan(n, 2, direction, C32) as p:
        y = p.execute(_to_device(h))
        _status(gb, p)
    err = oracle.rel_l2(_to_numpy(y), oracle.fft(x, direction))
    assert np.max(err) <= TOL, float(np.max(err))


@pytest.mark.parametrize("logn", [4, 6, 12, 13])
def test_c32_unaligned_input(gb, oracle, logn):
    """A complex32 input that is only 4-byte aligned (an odd element offset)
    is read from global memory directly instead of through the staging copy
    (tiles of 4096 elements); both within the class's bound, and the same
    bytes where the loader does no arithmetic (N a power of 16; 2^13 has no
    staging copy).  With an FP32 first stage (2^6) the two loaders are
    separately compiled code whose multiply-adds may be contracted
    differently."""
    n = 2 ** logn
    batch = max(4096 // n, 1) * 40 + 3
    h, x = _fp16_pairs(synth.uniform(9985 + logn, batch, n))
    buf = torch.zeros(2 * (batch * n + 1), dtype=torch.float16, device="cuda").view(torch.complex32)
    outs = []
    for shift in (0, 1):
        xin = buf[shift:shift + batch * n]
        xin.view(torch.float16).copy_(torch.from_numpy(np.ascontiguousarray(h).reshape(-1)).cuda())
        out = torch.empty(batch * n, dtype=torch.complex32, device="cuda")
        with gb.Plan(n, batch, -1, C32) as p:
            st = torch.cuda.current_stream().cuda_stream
            gb.fft_execute(p.handle, xin.data_ptr(), out.data_ptr(), st)
            gb.fft_plan_sync_status(p.handle, st)
        outs.append(out.view(torch.int16))
        err = oracle.rel_l2(_to_numpy(out.view(batch, n)), oracle.fft(x, -1))
        assert np.max(err) <= TOL, (shift, float(np.max(err)))
    if logn % 4 == 0 or logn > 12:
        assert torch.equal(outs[0], outs[1])


def test_c32_rejects(gb):
    """complex32 storage is the tcgen05 FP16 kernel's: no warp-MMA form, no
    lengths outside 2^4 .. 2^14, and buffers aligned to 4 bytes."""
    for n, variant in ((2 ** 25, 0), (8, 0), (4096, 1)):
        with pytest.raises(gb.GbfftError):
            gb.fft_plan_create(n, 4, -1, C32, variant=variant)
    with pytest.raises(gb.GbfftError):
        gb.fft_plan_create(1024, 4, -1, 5)
    x = torch.zeros(2 * (4 * 1024 + 1), dtype=torch.float16, device="cuda").view(torch.complex32)
    with gb.Plan(1024, 4, -1, C32) as p:
        with pytest.raises(gb.GbfftError):
            gb.fft_execute(p.handle, x.data_ptr() + 2, x.data_ptr(), 0)
        # 4-byte alignment suffices (an odd complex32 offset)
        gb.fft_execute(p.handle, x[1:].data_ptr(), x[1:].data_ptr(), 0)
        torch.cuda.synchronize()
